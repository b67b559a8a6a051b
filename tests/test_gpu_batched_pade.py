"""GPU parity, batched Pade comparators: r_10 or r_26 by products + squarings
(eq. pade10, eq. pade26; the solve, 4/3 of a product in the paper's count,
runs as Gaussian elimination with partial pivoting in one CTA per matrix),
and r_26 alone, against the oracle's same choice: 1e-12 relative Frobenius
with binary64 storage, in a cluster per matrix and one CTA per matrix."""
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


def _run(h, api, mats, flags, dtype=np.float64):
    import torch
    ins = [torch.from_numpy(np.ascontiguousarray(A, dtype=dtype)).cuda() for A in mats]
    outs = [torch.full_like(a, float("nan")) for a in ins]
    b = api.Batch(ins, outs)
    h.expm_batched(b, flags=flags)
    torch.cuda.synchronize()
    return [o.cpu().numpy().astype(np.float64) for o in outs], b.infos()


@pytest.mark.parametrize("count", [6, 100])  # a cluster per matrix / one CTA per matrix
def test_pade_matches_oracle(h, api, count):
    rng = np.random.default_rng(40 + count)
    ns = [1, 5, 64, 113, 200, 256] + [int(n) for n in rng.integers(8, 120, size=count - 6)]
    norms = [0.01, 0.2, 1.0, 2.0, 20.0, 100.0] + list(rng.uniform(0.001, 50.0, size=count - 6))
    mats = [W.gaussian(n, 1000 + i, float(v)) for i, (n, v) in enumerate(zip(ns, norms))]
    outs, infos = _run(h, api, mats, api.SCHEME_PADE)
    seen = set()
    for A, E, inf in zip(mats, outs, infos):
        want, oi = O.expm(A, "pade")
        assert inf["status"] == 0 and (inf["m"], inf["s"], inf["products"]) == (oi.m, oi.s, oi.products), (inf, oi)
        assert rel_fro(E, want) < 1e-12, (A.shape, inf, rel_fro(E, want))
        seen.add(inf["m"])
    assert seen == {10, 26}


def test_pade26_only(h, api):
    mats = [W.gaussian(n, 1100 + n, v) for n, v in ((40, 0.05), (150, 8.0), (256, 60.0))]
    outs, infos = _run(h, api, mats, api.SCHEME_PADE26)
    for A, E, inf in zip(mats, outs, infos):
        want, oi = O.expm(A, "pade26")
        assert inf["m"] == 26 and (inf["m"], inf["s"]) == (oi.m, oi.s)
        assert rel_fro(E, want) < 1e-12


def test_pade_binary32_storage_and_statuses(h, api):
    mats = [W.batch_matrix(i, n, v, seed=9) for i, (n, v) in enumerate(((32, 0.5), (96, 7.0), (200, 40.0)))]
    outs, infos = _run(h, api, mats, api.SCHEME_PADE, dtype=np.float32)
    for A, E, inf in zip(mats, outs, infos):
        A32 = A.astype(np.float32).astype(np.float64)
        want, _ = O.expm(A32, "pade")
        assert inf["status"] == 0 and rel_fro(E, want) < 1e-6
    bad = np.eye(20)
    bad[2, 3] = np.nan
    _, infos = _run(h, api, [bad, np.eye(30) * 900.0], api.SCHEME_PADE)
    assert [i["status"] for i in infos] == [api.NONFINITE_INPUT, api.OVERFLOW]


def test_pade_rejects_learned_selection(api):
    import torch
    hh = api.Handle(0)
    hh.batch_reserve(32)
    x = torch.eye(8, dtype=torch.float64, device="cuda")
    b = api.Batch([x], [torch.empty_like(x)])
    with pytest.raises(api.BBCError) as ei:
        hh.expm_batched(b, flags=api.SCHEME_PADE | api.SELECT_ALPHA)
    assert ei.value.code == api.UNSUPPORTED
    hh.close()
