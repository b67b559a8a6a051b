"""GPU parity, batched path with a thread-block cluster per matrix.

A batch of at most half as many matrices as SMs runs with up to 16 CTAs (on
distinct SMs) sharing each matrix: each CTA forms its share of the output tiles
of every product of the reduced-product scheme (Section 3) and of the squarings
(eq. eses), and the scalar work (||A||_1, the (m, s) choice by eq. theta) is
repeated in every CTA. Every output element still sums k in the same order, so
a matrix's exponential is bit for bit the one the one-CTA-per-matrix launch of
a large batch gives; the tests check that, and the oracle parity of the 64 x 64
single-matrix case at its 1e-13 tolerance.
"""
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
    hh.batch_reserve(256, api.PREC_OZAKI)
    yield hh
    hh.close()


def _sms():
    import torch
    return torch.cuda.get_device_properties(0).multi_processor_count


def _run(h, api, mats, dtype=np.float64, flags=0):
    import torch
    ins = [torch.from_numpy(np.ascontiguousarray(A, dtype=dtype)).cuda() for A in mats]
    outs = [torch.full_like(a, float("nan")) for a in ins]
    b = api.Batch(ins, outs)
    h.expm_batched(b, flags=flags)
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in outs], b.infos()


def test_launch_shape(h, api):
    c1, g1 = h.batch_launch_shape(1)
    assert c1 in (2, 4, 8, 16) and g1 % c1 == 0 and g1 >= c1, (c1, g1)
    c, g = h.batch_launch_shape(_sms() // 2 + 1)      # enough matrices for every SM: one CTA each
    assert c == 1 and g >= _sms(), (c, g)
    c, g = h.batch_launch_shape(20000)
    assert c == 1
    with pytest.raises(api.BBCError):
        h.batch_launch_shape(0)


def test_single_64_matches_oracle(h, api):
    """The 64 x 64 single-matrix case: N(0,1) entries from seed 0 rescaled to
    1-norm 1, (m, s) by the theta_m thresholds at u = 2^-53, 1e-13 relative
    Frobenius against the oracle."""
    assert h.batch_launch_shape(1)[0] > 1
    A = W.small_case()
    (E,), (inf,) = _run(h, api, [A])
    want, oi = O.expm(A, "new")
    assert inf["status"] == 0 and (inf["m"], inf["s"], inf["products"]) == (oi.m, oi.s, oi.products)
    assert rel_fro(E, want) < 1e-13, rel_fro(E, want)


@pytest.mark.parametrize("n,norm", [(1, 0.3), (5, 2.0), (17, 40.0), (64, 5.0), (100, 0.01), (255, 20.0),
                                    (256, 100.0)])
def test_single_matrix_sizes(h, api, n, norm):
    """Ragged sizes: fewer output tiles than CTAs (N <= 16), partial tiles, and
    the largest N with s > 0 squarings."""
    A = W.gaussian(n, 10 + n, norm)
    (E,), (inf,) = _run(h, api, [A])
    want, oi = O.expm(A, "new")
    assert inf["status"] == 0 and (inf["m"], inf["s"]) == (oi.m, oi.s)
    assert rel_fro(E, want) < 1e-12, (n, rel_fro(E, want))


@pytest.mark.parametrize("flags_name", ["fp64", "split"])
def test_cluster_equals_one_cta_per_matrix(h, api, flags_name):
    """The same matrices alone (cluster launch) and inside a batch large enough
    for one CTA per matrix give identical bits and identical (m, s)."""
    flags = 0 if flags_name == "fp64" else api.PREC_OZAKI
    probe = [W.gaussian(n, 50 + n, v) for n, v in ((64, 1.0), (200, 8.0), (33, 0.2), (256, 60.0), (9, 3.0))]
    filler = [W.gaussian(8, 900 + i, 1.0) for i in range(_sms())]
    assert h.batch_launch_shape(len(probe) + len(filler))[0] == 1
    big, big_inf = _run(h, api, probe + filler, flags=flags)
    for k, A in enumerate(probe):
        (E,), (inf,) = _run(h, api, [A], flags=flags)
        assert np.array_equal(E, big[k]), (A.shape, np.max(np.abs(E - big[k])))
        for key in ("m", "s", "products", "status"):
            assert inf[key] == big_inf[k][key], (key, inf, big_inf[k])
    trio, trio_inf = _run(h, api, probe[:3], flags=flags)  # three clusters at once
    for k in range(3):
        assert np.array_equal(trio[k], big[k])


def test_cluster_statuses(h, api):
    """Overflow found by any CTA of the cluster reaches the matrix's status: the
    binary32 result of e^900 I (N = 256) overflows in every CTA's share."""
    bad = np.eye(256)
    bad[200, 17] = np.inf
    for mats, want in (([np.eye(256) * 900.0], api.OVERFLOW), ([bad], api.NONFINITE_INPUT),
                       ([np.eye(256) * 0.5], api.OK)):
        outs, infos = _run(h, api, mats, dtype=np.float32)
        assert infos[0]["status"] == want, (infos[0], want)
    assert np.allclose(outs[0], np.eye(256) * np.exp(0.5), rtol=1e-6)


def test_cluster_learned_selector(api):
    """Learned (m, s) proposals in cluster mode: identical to the one-CTA launch."""
    from paper_1710_10989_gb300 import selector as SEL
    hh = api.Handle(0)
    hh.batch_reserve(256)
    SEL.install(hh)
    flags = api.SELECT_LEARNED
    probe = [W.batch_matrix(i, n, v, seed=8) for i, (n, v) in enumerate(((64, 3.0), (128, 0.05), (256, 30.0)))]
    filler = [W.gaussian(8, 700 + i, 1.0) for i in range(_sms())]
    big, big_inf = _run(hh, api, probe + filler, flags=flags)
    for k, A in enumerate(probe):
        (E,), (inf,) = _run(hh, api, [A], flags=flags)
        assert np.array_equal(E, big[k])
        assert (inf["m"], inf["s"], inf["selector"]) == (big_inf[k]["m"], big_inf[k]["s"], big_inf[k]["selector"])
        want, _ = O.expm(A, "new")
        assert rel_fro(E, want) < 1e-12
    hh.close()


def test_cluster_graph_capture_replay(h, api):
    """One matrix, captured once and replayed: the launch the small-matrix
    benchmark times."""
    import torch
    A = W.small_case()
    x = torch.from_numpy(A).cuda()
    y = torch.zeros_like(x)
    b = api.Batch([x], [y])
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        h.expm_batched(b, stream=s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            h.expm_batched(b, stream=s)
    for _ in range(3):
        y.zero_()
        g.replay()
    torch.cuda.synchronize()
    want, _ = O.expm(A, "new")
    assert rel_fro(y.cpu().numpy(), want) < 1e-13
