"""GPU parity, exponential-integrator steps: Out_i = exp(A_i) B_i in one
persistent launch (bbc_expm_apply_batched), against the oracle's exp(A_i)
times B_i; then Lie-group integrators built on it: Lie-Euler with a constant
skew-symmetric generator (orthogonality kept, n steps = exp(n h A)), the
midpoint Magnus method for Y' = A(t) Y with skew A(t) (order 2 observed) and
the fourth-order Magnus method with its commutator from the library's products
(order 4 observed)."""
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


def _skew(n, seed, norm):
    G = np.random.default_rng(seed).standard_normal((n, n))
    S = G - G.T
    return S * (norm / np.max(np.sum(np.abs(S), axis=0)))


def _apply(h, api, As, Bs, dtype=np.float64, flags=0, in_place=False):
    import torch
    ins = [torch.from_numpy(np.ascontiguousarray(A, dtype=dtype)).cuda() for A in As]
    rhs = [torch.from_numpy(np.ascontiguousarray(B, dtype=dtype)).cuda() for B in Bs]
    outs = rhs if in_place else [torch.full_like(a, float("nan")) for a in ins]
    b = api.Batch(ins, outs, rhs=rhs)
    h.expm_apply_batched(b, flags=flags)
    torch.cuda.synchronize()
    return [o.cpu().numpy().astype(np.float64) for o in outs], b.infos()


@pytest.mark.parametrize("count", [5, 120])  # a cluster per matrix / one CTA per matrix
def test_apply_matches_oracle(h, api, count):
    rng = np.random.default_rng(count)
    ns = [1, 7, 64, 130, 256] + [int(n) for n in rng.integers(8, 100, size=count - 5)]
    As = [W.gaussian(n, 300 + i, float(v)) for i, (n, v) in enumerate(zip(ns, rng.uniform(0.01, 40, size=count)))]
    Bs = [rng.standard_normal((n, n)) for n in ns]
    outs, infos = _apply(h, api, As, Bs)
    for A, B, E, inf in zip(As, Bs, outs, infos):
        eA, oi = O.expm(A, "new")
        assert inf["status"] == 0 and (inf["m"], inf["s"]) == (oi.m, oi.s)
        assert inf["products"] == oi.products + 1
        assert rel_fro(E, eA @ B) < 1e-12, (A.shape, rel_fro(E, eA @ B))


def test_cluster_and_one_cta_agree_bitwise(h, api):
    rng = np.random.default_rng(4)
    As = [W.gaussian(n, 400 + n, 3.0) for n in (64, 200, 33)]
    Bs = [rng.standard_normal(A.shape) for A in As]
    filler_A = [W.gaussian(8, 500 + i, 1.0) for i in range(150)]
    filler_B = [np.eye(8)] * 150
    small, _ = _apply(h, api, As, Bs)
    big, _ = _apply(h, api, As + filler_A, Bs + filler_B)
    for k in range(3):
        assert np.array_equal(small[k], big[k])


def test_in_place_and_split_products(h, api):
    rng = np.random.default_rng(6)
    As = [W.gaussian(n, 600 + n, 5.0) for n in (16, 100, 256)]
    Bs = [rng.standard_normal(A.shape) for A in As]
    outs, _ = _apply(h, api, As, Bs, in_place=True)
    for A, B, E in zip(As, Bs, outs):
        assert rel_fro(E, O.expm(A, "new")[0] @ B) < 1e-12
    outs, _ = _apply(h, api, As, Bs, dtype=np.float32, flags=api.PREC_OZAKI)
    for A, B, E in zip(As, Bs, outs):
        A32, B32 = A.astype(np.float32).astype(np.float64), B.astype(np.float32).astype(np.float64)
        assert rel_fro(E, O.expm(A32, "new")[0] @ B32) < 1e-6


def test_lie_euler_keeps_orthogonality(h, api):
    """Y_{k+1} = exp(h A) Y_k with skew A: Y stays orthogonal and after n steps
    equals exp(n h A) Y_0 (the group property), for several systems at once."""
    import torch
    n_steps, hstep = 20, 0.25
    gens = [_skew(n, 700 + n, 4.0) for n in (8, 31, 64, 120)]
    Y0 = [np.linalg.qr(np.random.default_rng(n).standard_normal((n, n)))[0] for n in (8, 31, 64, 120)]
    ins = [torch.from_numpy(hstep * G).cuda() for G in gens]
    Y = [torch.from_numpy(y.copy()).cuda() for y in Y0]
    b = api.Batch(ins, Y, rhs=Y)                  # in place: Y <- exp(h A) Y
    for _ in range(n_steps):
        h.expm_apply_batched(b)
    torch.cuda.synchronize()
    for G, y0, y in zip(gens, Y0, Y):
        yn = y.cpu().numpy()
        n = yn.shape[0]
        assert np.linalg.norm(yn.T @ yn - np.eye(n)) < 1e-12 * n_steps * n
        want = O.expm(n_steps * hstep * G, "new")[0] @ y0
        assert rel_fro(yn, want) < 1e-11


def test_midpoint_magnus_is_second_order(h, api):
    """Y' = A(t) Y, A(t) = A0 + t A1 skew: Y_{k+1} = exp(h A(t_k + h/2)) Y_k. The
    error at t = 1 against a 256-step run falls about 4x per halving of h."""
    import torch
    ns = (6, 20, 48)
    A0 = [_skew(n, 800 + n, 3.0) for n in ns]
    A1 = [_skew(n, 900 + n, 6.0) for n in ns]

    def integrate(steps):
        hstep = 1.0 / steps
        Y = [torch.eye(n, dtype=torch.float64, device="cuda") for n in ns]
        gens = [torch.empty((n, n), dtype=torch.float64, device="cuda") for n in ns]
        b = api.Batch(gens, Y, rhs=Y)
        a0 = [torch.from_numpy(a).cuda() for a in A0]
        a1 = [torch.from_numpy(a).cuda() for a in A1]
        for k in range(steps):
            tm = (k + 0.5) * hstep
            for g, x0, x1 in zip(gens, a0, a1):
                torch.add(x0, x1, alpha=tm, out=g)
                g.mul_(hstep)
            h.expm_apply_batched(b)
        torch.cuda.synchronize()
        return [y.cpu().numpy() for y in Y]

    ref = integrate(256)
    errs = [[np.linalg.norm(y - r) for y, r in zip(integrate(s), ref)] for s in (8, 16, 32)]
    for i in range(len(ns)):
        r1, r2 = errs[0][i] / errs[1][i], errs[1][i] / errs[2][i]
        assert 3.0 < r1 < 5.0 and 3.0 < r2 < 5.0, (ns[i], r1, r2)


def test_fourth_order_magnus_with_library_commutators(h, api):
    """Fourth-order Magnus at the two Gauss points: Omega = h/2 (A1 + A2) +
    sqrt(3) h^2 / 12 [A2, A1], the commutator from the library's FP64 products
    (bbc_gemm), then Y <- exp(Omega) Y in the batched launch. The error against
    a 256-step run falls about 16x per halving of h."""
    import math
    import torch
    ns = (6, 20, 48)
    A0 = [torch.from_numpy(_skew(n, 800 + n, 3.0)).cuda() for n in ns]
    A1 = [torch.from_numpy(_skew(n, 900 + n, 6.0)).cuda() for n in ns]
    c1, c2 = 0.5 - math.sqrt(3) / 6, 0.5 + math.sqrt(3) / 6

    def integrate(steps):
        hstep = 1.0 / steps
        Y = [torch.eye(n, dtype=torch.float64, device="cuda") for n in ns]
        om = [torch.empty((n, n), dtype=torch.float64, device="cuda") for n in ns]
        b = api.Batch(om, Y, rhs=Y)
        for k in range(steps):
            t = k * hstep
            for o, a0, a1 in zip(om, A0, A1):
                X1 = a0 + (t + c1 * hstep) * a1
                X2 = a0 + (t + c2 * hstep) * a1
                P = torch.empty_like(X1)
                Q = torch.empty_like(X1)
                h.gemm(X2, X1, P)
                h.gemm(X1, X2, Q)
                torch.add(X1, X2, out=o)
                o.mul_(hstep / 2).add_(P - Q, alpha=math.sqrt(3) * hstep * hstep / 12)
            h.expm_apply_batched(b)
        torch.cuda.synchronize()
        return [y.cpu().numpy() for y in Y]

    ref = integrate(256)
    errs = [[np.linalg.norm(y - r) for y, r in zip(integrate(s), ref)] for s in (4, 8, 16)]
    for i in range(len(ns)):
        r1, r2 = errs[0][i] / errs[1][i], errs[1][i] / errs[2][i]
        assert 13.0 < r1 < 19.0 and 13.0 < r2 < 19.0, (ns[i], r1, r2)
