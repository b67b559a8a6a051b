"""GPU parity, batched path: one persistent launch over many matrices of uneven
sizes, each checked against the oracle at the same (m, s). Tolerances: 1e-12
relative Frobenius with binary64 storage; 1e-6 with binary32 storage (the
batched workload's tolerance; the oracle runs on the binary32-rounded input)."""
import numpy as np
import pytest

from gpu_util import rel_fro
from oracle import oracle as O
from paper_1710_10989_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_10989_gb300 import api as A
    return A


@pytest.fixture(scope="module")
def h(api):
    hh = api.Handle(0)
    hh.batch_reserve(256)
    yield hh
    hh.close()


def _run(h, api, mats, dtype):
    import torch
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    ins = [torch.from_numpy(A.astype(dtype)).cuda() for A in mats]
    outs = [torch.full_like(a, float("nan")) for a in ins]
    b = api.Batch(ins, outs)
    h.expm_batched(b)
    torch.cuda.synchronize()
    return [o.cpu().numpy().astype(np.float64) for o in outs], b.infos()


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_batch_matches_oracle(h, api, dtype):
    ns, norms = W.batch_spec(count=40, seed=3)
    ns[:6] = [1, 7, 8, 65, 255, 256]           # edge sizes, ragged tails
    mats = [W.batch_matrix(i, int(n), float(v), seed=3) for i, (n, v) in enumerate(zip(ns, norms))]
    outs, infos = _run(h, api, mats, dtype)
    tol = 1e-12 if dtype == np.float64 else 1e-6
    for A, E, inf in zip(mats, outs, infos):
        A = A.astype(dtype).astype(np.float64)
        want, oi = O.expm(A, "new")
        assert inf["status"] == 0, inf
        assert (inf["m"], inf["s"], inf["products"]) == (oi.m, oi.s, oi.products), (inf, oi)
        assert rel_fro(E, want) < tol, (A.shape, inf, rel_fro(E, want))


def test_batch_order_largest_first(api):
    assert api.batch_order([8, 256, 64, 256, 1]) == [1, 3, 2, 0, 4]


def test_batch_statuses(h, api):
    import torch
    bad = np.eye(12)
    bad[3, 3] = np.nan
    big = np.eye(9) * 900.0  # e^900 overflows binary32 and binary64
    mats = [np.eye(5) * 0.5, bad, big]
    ins = [torch.from_numpy(m.astype(np.float32)).cuda() for m in mats]
    outs = [torch.zeros_like(a) for a in ins]
    b = api.Batch(ins, outs)
    h.expm_batched(b)
    torch.cuda.synchronize()
    st = [i["status"] for i in b.infos()]
    assert st == [api.OK, api.NONFINITE_INPUT, api.OVERFLOW], st
    assert np.allclose(outs[0].cpu().numpy(), np.eye(5) * np.exp(0.5), rtol=1e-6)


def test_batch_rejects_oversize_per_matrix(api):
    import torch
    hh = api.Handle(0)
    hh.batch_reserve(32)
    ins = [torch.eye(16, dtype=torch.float64, device="cuda"), torch.eye(40, dtype=torch.float64, device="cuda")]
    outs = [torch.zeros_like(a) for a in ins]
    b = api.Batch(ins, outs)
    hh.expm_batched(b)
    torch.cuda.synchronize()
    st = [i["status"] for i in b.infos()]
    assert st == [api.OK, api.INVALID_ARG]
    assert torch.allclose(outs[0], torch.eye(16, dtype=torch.float64, device="cuda") * np.e)
    hh.close()


def test_batch_graph_capture_replay(h, api):
    import torch
    ns, norms = W.batch_spec(count=12, seed=4)
    mats = [W.batch_matrix(i, int(n), float(v), seed=4) for i, (n, v) in enumerate(zip(ns, norms))]
    ins = [torch.from_numpy(A).cuda() for A in mats]
    outs = [torch.zeros_like(a) for a in ins]
    b = api.Batch(ins, outs)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        h.expm_batched(b, stream=s)   # warm-up outside the capture
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            h.expm_batched(b, stream=s)
    for o in outs:
        o.zero_()
    g.replay()
    torch.cuda.synchronize()
    for A, o in zip(mats, outs):
        want, _ = O.expm(A, "new")
        assert rel_fro(o.cpu().numpy(), want) < 1e-12


def test_batch_split_precision_matches_oracle(api):
    """4-slice BF16 products (warp-level MMAs, exact group sums): the batched
    workload's tolerance (1e-6 against the oracle on the binary32-rounded input)."""
    import torch
    hh = api.Handle(0)
    hh.batch_reserve(256, api.PREC_OZAKI)
    ns, norms = W.batch_spec(count=48, seed=5)
    ns[:6] = [1, 7, 8, 65, 255, 256]
    mats = [W.batch_matrix(i, int(n), float(v), seed=5) for i, (n, v) in enumerate(zip(ns, norms))]
    outs, infos = None, None
    ins = [torch.from_numpy(A.astype(np.float32)).cuda() for A in mats]
    outs = [torch.full_like(a, float("nan")) for a in ins]
    b = api.Batch(ins, outs)
    hh.expm_batched(b, flags=api.PREC_OZAKI)
    torch.cuda.synchronize()
    worst = 0.0
    for A, o, inf in zip(mats, outs, b.infos()):
        A = A.astype(np.float32).astype(np.float64)
        want, oi = O.expm(A, "new")
        assert inf["status"] == 0 and (inf["m"], inf["s"]) == (oi.m, oi.s)
        worst = max(worst, rel_fro(o.cpu().numpy().astype(np.float64), want))
    assert worst < 1e-6, worst
    hh.close()


def test_batch_split_learned_all_three(api):
    """Split-precision products + learned selection in one launch; N > 256 falls
    back to FP64 products inside the same launch."""
    import torch
    from paper_1710_10989_gb300 import selector as SEL
    hh = api.Handle(0)
    hh.batch_reserve(512, api.PREC_OZAKI)
    SEL.install(hh)
    ns, norms = W.batch_spec(count=24, seed=6)
    ns[0], ns[1] = 300, 512
    mats = [W.batch_matrix(i, int(n), float(v), seed=6) for i, (n, v) in enumerate(zip(ns, norms))]
    ins = [torch.from_numpy(A).cuda() for A in mats]
    outs = [torch.zeros_like(a) for a in ins]
    b = api.Batch(ins, outs)
    hh.expm_batched(b, flags=api.PREC_OZAKI | api.SELECT_LEARNED)
    torch.cuda.synchronize()
    for A, o, inf in zip(mats, outs, b.infos()):
        assert inf["status"] == 0 and inf["selector"] in (2, 3, 4)
        want, _ = O.expm(A, "new")
        tol = 1e-12 if A.shape[0] > 256 else 1e-6
        assert rel_fro(o.cpu().numpy(), want) < tol, (A.shape, inf)
    hh.close()


def test_autotuner_choice_keeps_parity(api):
    """bbc_batch_tune times split against FP64 products per size bucket and the
    grid size; whatever it picks, the batch still matches the oracle."""
    import torch
    h = api.Handle(0)
    h.batch_reserve(64, api.PREC_OZAKI)
    mask, ctas = h.batch_tune(64)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert ctas in (sms, 2 * sms)
    assert mask >> 8 == (0xFFFFFFFF >> 8)          # buckets above max_n keep the default
    t16, t32, s16 = h.batch_get_shapes()
    assert (t16 | t32 | s16) >> 8 == 0             # shapes chosen only for the tuned buckets
    assert t16 & t32 == 0 and (t16 | t32) & mask == 0 and s16 & ~mask == 0  # one choice per bucket
    mats = [W.gaussian(n, 300 + n, 0.5 + n / 16) for n in (64, 8, 33, 17, 50, 64, 1, 40)]
    ins = [torch.from_numpy(A).cuda() for A in mats]
    outs = [torch.empty_like(x) for x in ins]
    b = api.Batch(ins, outs)
    h.expm_batched(b, flags=api.PREC_OZAKI)
    torch.cuda.synchronize()
    for A, out, inf in zip(mats, outs, b.infos()):
        want, oi = O.expm(A, "new")
        assert inf["status"] == 0 and (inf["m"], inf["s"]) == (oi.m, oi.s)
        assert rel_fro(out.cpu().numpy(), want) < 1e-6
    h.batch_set_tuning(0, 0)                         # FP64 products everywhere, reserved grid
    h.expm_batched(api.Batch(ins, outs), flags=api.PREC_OZAKI)
    torch.cuda.synchronize()
    for A, out in zip(mats, outs):
        want, _ = O.expm(A, "new")
        assert rel_fro(out.cpu().numpy(), want) < 1e-12
    h.close()


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_batch_single_precision_thresholds(api, prec):
    """Table 2's u = 2^-24 row through the batched call's tol: every matrix gets
    the oracle's (m, s) at u = 2^-24 and its result equals the oracle's exp(A) at
    that (m, s) within the batched workload's 1e-6 (binary32 storage)."""
    import torch
    hh = api.Handle(0)
    flags = api.PREC_OZAKI if prec == "split" else api.PREC_FP64
    hh.batch_reserve(256, flags)
    ns, norms = W.batch_spec(count=40, seed=9)
    ns[:5] = [1, 8, 65, 255, 256]
    mats = [W.batch_matrix(i, int(n), float(v), seed=9) for i, (n, v) in enumerate(zip(ns, norms))]
    ins = [torch.from_numpy(A.astype(np.float32)).cuda() for A in mats]
    outs = [torch.full_like(a, float("nan")) for a in ins]
    b = api.Batch(ins, outs)
    hh.expm_batched(b, tol=api.U_SINGLE, flags=flags)
    torch.cuda.synchronize()
    fewer = 0
    worst = 0.0
    for A, o, inf in zip(mats, outs, b.infos()):
        A = A.astype(np.float32).astype(np.float64)
        want, oi = O.expm(A, "new", u=2.0 ** -24)
        assert inf["status"] == 0, inf
        assert (inf["m"], inf["s"], inf["products"]) == (oi.m, oi.s, oi.products), (inf, oi)
        assert (oi.m, oi.s) == O.select(O.norm1(A), "new", 2.0 ** -24)
        _, od = O.expm(A, "new")                       # u = 2^-53, for the product count only
        fewer += od.products > oi.products
        worst = max(worst, rel_fro(o.cpu().numpy().astype(np.float64), want))
    assert worst < 1e-6, worst
    assert fewer >= 10        # the single-precision thresholds save products on many matrices
    hh.close()


def test_product_shapes_leave_results_bit_identical(api):
    """The autotuner's product shapes (FP64 output tiles of 64, 32 or 16; split warp
    tasks of 32 x 16 or 16 x 16) change only how the work is cut: every output sums
    the same terms in the same order, so results are bit-identical, and they match
    the oracle (1e-12 with FP64 products, 1e-6 with split products)."""
    import torch
    hh = api.Handle(0)
    hh.batch_reserve(256, api.PREC_OZAKI)
    sizes = [8, 13, 24, 33, 64, 100, 129, 200, 256]
    mats = [W.gaussian(n, 900 + n, 0.3 + n / 40) for n in sizes]
    ins = [torch.from_numpy(A).cuda() for A in mats]
    for flags, tol in ((api.PREC_FP64, 1e-12), (api.PREC_OZAKI, 1e-6)):
        results = []
        for shapes in (None, (0xFFFFFFFF, 0, 0xFFFFFFFF), (0, 0xFFFFFFFF, 0), (0x0000FFFF, 0xFFFF0000, 0x0F0F0F0F)):
            hh.batch_set_shapes(shapes)
            outs = [torch.empty_like(x) for x in ins]
            hh.expm_batched(api.Batch(ins, outs), flags=flags)
            torch.cuda.synchronize()
            results.append(outs)
        for outs in results[1:]:
            assert all(torch.equal(a, b) for a, b in zip(results[0], outs)), flags
        for A, o in zip(mats, results[0]):
            want, _ = O.expm(A, "new")
            assert rel_fro(o.cpu().numpy(), want) < tol, (A.shape, flags)
    assert hh.batch_get_shapes() == (0x0000FFFF, 0xFFFF0000, 0x0F0F0F0F)
    hh.batch_set_shapes(None)
    assert hh.batch_get_shapes() == (0, 0, 0)
    hh.close()
