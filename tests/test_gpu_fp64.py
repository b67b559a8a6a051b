"""GPU parity, FP64 path: every step of the hot path through the C-ABI against
the CPU oracle on the same seeded inputs (relative Frobenius tolerances:
1e-13 for the 64 x 64 workload, 1e-12 for the 4096 x 4096 workload and the
mid-size cases)."""
import numpy as np
import pytest

from gpu_util import empty_like_dev, rel_fro, to_dev, to_host
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
    yield hh
    hh.close()


# ---- a1: 1-norm ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 7, 64, 255, 257, 1000])
def test_norm1(h, n):
    A = W.gaussian(n, 100 + n, None)
    got = h.norm1(to_dev(A))
    assert got == pytest.approx(O.norm1(A), rel=1e-14)


def test_norm1_nonfinite(h, api):
    A = np.eye(33)
    A[5, 7] = np.inf
    assert not np.isfinite(h.norm1(to_dev(A)))
    A[5, 7] = np.nan
    assert np.isnan(h.norm1(to_dev(A)))


# ---- product --------------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 7, 16, 64, 65, 200, 512, 513, 640])
def test_gemm_fp64(h, n):
    P = W.gaussian(n, 1 + n, None)
    Q = W.gaussian(n, 2 + n, None)
    C = empty_like_dev(n)
    h.gemm(to_dev(P), to_dev(Q), C)
    assert rel_fro(to_host(C), O.gemm(P, Q)) < 1e-15 * max(8, np.sqrt(n))


# ---- a3-a8: scaled Taylor polynomial by each program -----------------------------------------

@pytest.mark.parametrize("scheme,m", [("new", 1), ("new", 2), ("new", 4), ("new", 8), ("new", 12),
                                      ("new", 18), ("ps", 4), ("ps", 6), ("ps", 9), ("ps", 12),
                                      ("ps", 16)])
@pytest.mark.parametrize("n", [5, 130])
def test_taylor_programs(h, api, scheme, m, n):
    s = 3
    A = W.gaussian(n, 40 + m, 6.0)
    T = empty_like_dev(n)
    flags = api.SCHEME_NEW if scheme == "new" else api.SCHEME_PS
    prods = h.taylor(to_dev(A), m, s, T, flags)
    X = np.ldexp(A, -s)
    c0 = O.product_count()
    want = O.taylor_new(X, m) if scheme == "new" else O.taylor_ps(X, m)
    assert prods == O.product_count() - c0          # Table 3 counts, both sides
    assert rel_fro(to_host(T), want) < 1e-14


# ---- whole path, fixed (m, s) and selected -----------------------------------------------------

def test_small_workload_all_schemes(h, api):
    """64 x 64, N(0,1) from seed 0, ||A||_1 = 1: NEW (18, 0) and PS (16, 1)."""
    A = W.small_case()
    for flags, name in ((api.SCHEME_NEW, "new"), (api.SCHEME_PS, "ps")):
        out = empty_like_dev(64)
        info = h.expm(to_dev(A), out, 0.0, flags)
        want, oi = O.expm(A, name)
        assert (info.m, info.s, info.products) == (oi.m, oi.s, oi.products)
        assert rel_fro(to_host(out), want) < 1e-13
    assert (info.m, info.s) == (16, 1)


@pytest.mark.parametrize("idx", range(6))
@pytest.mark.parametrize("n,nonnormal", [(96, False), (257, False), (300, True)])
def test_expm_selected_matches_oracle(h, api, idx, n, nonnormal):
    A = W.dense_case(idx, n=n, nonnormal=nonnormal)
    out = empty_like_dev(n)
    info = h.expm(to_dev(A), out)
    # the non-normal family is upper triangular: the library finds that and takes
    # the triangular path, whose oracle is expm_upper
    want, oi = O.expm_upper(A, "new") if nonnormal else O.expm(A, "new")
    assert info.structure == (1 if nonnormal else 0)
    assert (info.m, info.s, info.products) == (oi.m, oi.s, oi.products)
    assert info.norm1 == pytest.approx(oi.norm1, rel=1e-14)
    assert rel_fro(to_host(out), want) < 1e-12


@pytest.mark.parametrize("m,s", [(1, 0), (2, 1), (4, 2), (8, 0), (12, 5), (18, 9)])
def test_expm_fixed_matches_oracle(h, api, m, s):
    A = W.gaussian(77, 5 + m, 2.0)
    out = empty_like_dev(77)
    info = h.expm_fixed(to_dev(A), out, m, s)
    want, oi = O.expm(A, "new", m=m, s=s)
    assert info.products == oi.products and info.selector == 1
    assert rel_fro(to_host(out), want) < 1e-13


def test_expm_host_buffers(h, api):
    A = W.gaussian(150, 9, 3.0)
    out = np.empty_like(A)
    info = h.expm_host(A, out)
    want, oi = O.expm(A, "new")
    assert (info.m, info.s) == (oi.m, oi.s)
    assert rel_fro(out, want) < 1e-12


def test_expm_host_many_pipelined(h, api):
    """Uneven sizes and both precisions through the pipelined host call: every
    result equals the single-matrix host call's bit for bit (same kernels, same
    order), and the oracle within the dense tolerance."""
    sizes = [150, 64, 257, 150, 33]
    As = [W.gaussian(n, 40 + i, 0.5 + i) for i, n in enumerate(sizes)]
    for flags in (api.PREC_FP64, api.PREC_OZAKI | api.ozaki_slices(7)):
        outs = [np.empty_like(A) for A in As]
        infos = h.expm_host_many(As, outs, 0.0, flags)
        for A, out, info in zip(As, outs, infos):
            ref = np.empty_like(A)
            one = h.expm_host(A, ref, 0.0, flags)
            assert (info.m, info.s, info.products) == (one.m, one.s, one.products)
            assert np.array_equal(out, ref)
            want, oi = O.expm(A, "new")
            assert (info.m, info.s) == (oi.m, oi.s)
            assert rel_fro(out, want) < 1e-12


def test_expm_host_many_reports_failure(h, api):
    As = [W.gaussian(40, 1, 1.0), np.full((40, 40), np.nan), W.gaussian(40, 2, 1.0)]
    outs = [np.zeros_like(A) for A in As]
    with pytest.raises(api.BBCError) as e:
        h.expm_host_many(As, outs)
    assert e.value.code == api.NONFINITE_INPUT
    want, _ = O.expm(As[0], "new")
    assert rel_fro(outs[0], want) < 1e-12   # the matrix before the failure is complete


# ---- status codes -------------------------------------------------------------------------------

def test_status_codes(h, api):
    A = np.eye(9)
    A[2, 3] = np.nan
    out = empty_like_dev(9)
    with pytest.raises(api.BBCError) as e:
        h.expm(to_dev(A), out)
    assert e.value.code == api.NONFINITE_INPUT
    with pytest.raises(api.BBCError) as e:
        h.expm(to_dev(np.eye(4) * 800.0), empty_like_dev(4))
    assert e.value.code == api.OVERFLOW
    Ad = to_dev(np.eye(4))
    with pytest.raises(api.BBCError) as e:
        h.expm(Ad, Ad)
    assert e.value.code == api.INVALID_ARG
    with pytest.raises(api.BBCError) as e:
        h.expm_fixed(Ad, empty_like_dev(4), 7, 0)
    assert e.value.code == api.INVALID_ARG
    z = empty_like_dev(6)
    info = h.expm(to_dev(np.zeros((6, 6))), z)
    assert (to_host(z) == np.eye(6)).all() and info.m == 1


# ---- upper triangular structure -----------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 5, 64, 130, 300, 1025])
@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_upper_products_match_oracle(h, api, n, prec):
    """Products of upper triangular operands that sum k over [i, j] only (K ranges
    per tile, tiles below the diagonal skipped) equal the oracle's full products."""
    rng = np.random.default_rng(n)
    P = np.triu(rng.standard_normal((n, n)))
    Q = np.triu(rng.standard_normal((n, n)))
    C = empty_like_dev(n)
    flags = api.UPPER | (api.PREC_FP64 if prec == "fp64" else api.PREC_OZAKI | api.ozaki_slices(7))
    h.gemm(to_dev(P), to_dev(Q), C, flags)
    got = to_host(C)
    want = O.gemm(P, Q)
    assert not np.tril(got, -1).any()
    assert rel_fro(got, want) < 4e-16 * max(4, np.sqrt(n))


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_upper_expm_matches_oracle(h, api, prec):
    flags = api.PREC_FP64 if prec == "fp64" else api.PREC_OZAKI | api.ozaki_slices(7)
    for n, norm, seed in ((200, 20.0, 3), (513, 100.0, 4), (64, 0.05, 5)):
        A = W.nonnormal_upper(n, seed, norm)
        out = empty_like_dev(n)
        info = h.expm(to_dev(A), out, 0.0, flags)
        want, oi = O.expm_upper(A, "new")
        assert info.structure == 1 and (info.m, info.s, info.products) == (oi.m, oi.s, oi.products)
        got = to_host(out)
        assert rel_fro(got, want) < 1e-12
        assert not np.tril(got, -1).any()
        # the exact diagonal is put back last: e^{a_ii} to the libraries' exp (CUDA's and
        # numpy's may differ in the last place)
        d, e = np.diag(got), np.exp(np.diag(A))
        assert np.all(np.abs(d - e) <= 2 * np.spacing(e))


def test_dense_flag_turns_structure_off(h, api):
    A = W.nonnormal_upper(150, 6, 5.0)
    out = empty_like_dev(150)
    info = h.expm(to_dev(A), out, 0.0, api.DENSE)
    want, oi = O.expm(A, "new")
    assert info.structure == 0 and (info.m, info.s) == (oi.m, oi.s)
    assert rel_fro(to_host(out), want) < 1e-12
    B = A.copy()
    B[100, 3] = 1e-30   # one entry below the diagonal: dense path
    info = h.expm(to_dev(B), out)
    assert info.structure == 0


def test_upper_flop_accounting(h, api):
    n = 300
    A = W.nonnormal_upper(n, 8, 1.0)
    out = empty_like_dev(n)
    h.profile_enable(True)
    info = h.expm(to_dev(A), out)
    f = h.profile_flops(api.KERNEL_PRODUCT)
    h.profile_enable(False)
    assert f == pytest.approx(info.products * n * (n + 1) * (n + 2) / 3.0, rel=1e-12)


# ---- the Pade r_26 comparator on the GPU --------------------------------------------------------

def test_small_workload_pade26(h, api):
    """64 x 64, ||A||_1 = 1: r_26 with s = 0 (the paper's reference method), GPU vs oracle."""
    A = W.small_case()
    out = empty_like_dev(64)
    info = h.expm(to_dev(A), out, 0.0, api.SCHEME_PADE26)
    want, oi = O.expm(A, "pade26")
    assert (info.m, info.s, info.products) == (oi.m, oi.s, oi.products) == (26, 0, 6)
    assert rel_fro(to_host(out), want) < 1e-13


# N <= 112: the shared-memory solve (one CTA per 4 right-hand sides, each factoring M);
# beyond: the blocked LU (cluster-factored panels, rank-32 updates)
@pytest.mark.parametrize("n,norm,nonnormal", [(1, 0.5, False), (7, 3.0, False), (96, 20.0, False),
                                              (112, 40.0, False), (113, 5.0, True), (300, 100.0, True),
                                              (257, 0.3, False), (1025, 2.0, False)])
def test_pade26_matches_oracle(h, api, n, norm, nonnormal):
    A = W.nonnormal_upper(n, 7, norm) if nonnormal else W.gaussian(n, 8, norm)
    out = empty_like_dev(n)
    info = h.expm(to_dev(A), out, 0.0, api.SCHEME_PADE26)
    want, oi = O.expm(A, "pade26")
    assert (info.m, info.s) == (oi.m, oi.s)
    assert rel_fro(to_host(out), want) < 1e-12


@pytest.mark.parametrize("norm,want", [(0.01, (10, 0)), (1.0, (10, 2)), (2.0, (26, 0)), (20.0, (26, 2))])
def test_pade_scheme_selects_r10_or_r26(h, api, norm, want):
    """BBC_SCHEME_PADE: r_10 (eq. pade10, 3 products) or r_26 (6 products), the
    cheaper in products + squarings, against the oracle's same choice."""
    A = W.gaussian(150, 12, norm)
    out = empty_like_dev(150)
    info = h.expm(to_dev(A), out, 0.0, api.SCHEME_PADE)
    ref, oi = O.expm(A, "pade")
    assert (info.m, info.s) == (oi.m, oi.s) == want
    assert info.products == oi.products
    assert rel_fro(to_host(out), ref) < 1e-12


@pytest.mark.parametrize("n,idx", [(1500, None), (4096, 4)])
def test_pade26_blocked_solve_large(h, api, n, idx):
    """The comparator at N = 1500 and at the dense workload's 4096 (norm 20: r_26
    with s = 2): products, the blocked LU solve and squarings against the oracle."""
    A = W.gaussian(1500, 11, 8.0) if idx is None else W.dense_case(idx)
    out = empty_like_dev(n)
    info = h.expm(to_dev(A), out, 0.0, api.SCHEME_PADE26)
    want, oi = O.expm(A, "pade26")
    assert (info.m, info.s, info.products) == (oi.m, oi.s, oi.products)
    assert rel_fro(to_host(out), want) < 1e-12


# ---- the comparator's solve on its own (bbc_solve): row interchanges exercised --------------------

@pytest.mark.parametrize("n", [1, 5, 64, 112, 113, 130, 500, 1025, 2000])
def test_solve_matches_oracle(h, api, n):
    """Gaussian matrices need row interchanges all the way down (the Pade denominators
    rarely do): the GPU solve against the oracle's elimination, same partial pivoting."""
    rng = np.random.default_rng(500 + n)
    M = rng.standard_normal((n, n))
    B = rng.standard_normal((n, n))
    dM, dB = to_dev(M), to_dev(B)
    h.solve(dM, dB)
    want = O.solve(M, B)
    cond = np.linalg.cond(M)
    assert rel_fro(to_host(dB), want) < 1e-15 * max(10.0, cond) * np.sqrt(n), (n, rel_fro(to_host(dB), want))


def test_solve_forced_pivots_and_singular(h, api):
    """A permuted, scaled identity plus noise: every pivot is forced and the result
    is known; a rank-deficient M reports BBC_OVERFLOW."""
    n = 300
    rng = np.random.default_rng(7)
    perm = rng.permutation(n)
    M = np.zeros((n, n))
    M[np.arange(n), perm] = rng.uniform(1.0, 2.0, n) * rng.choice([-1.0, 1.0], n)
    M += 1e-3 * rng.standard_normal((n, n))
    X = rng.standard_normal((n, n))
    B = M @ X
    dM, dB = to_dev(M), to_dev(B)
    h.solve(dM, dB)
    assert rel_fro(to_host(dB), X) < 1e-12
    assert rel_fro(to_host(dB), O.solve(M, B)) < 1e-13
    S = rng.standard_normal((n, n))
    S[:, 5] = 0.0                             # a zero column stays exactly zero under elimination
    with pytest.raises(api.BBCError) as e:
        h.solve(to_dev(S), to_dev(np.eye(n)))
    assert e.value.code == api.OVERFLOW


def test_pade26_split_products(h, api):
    A = W.gaussian(200, 9, 5.0)
    out = empty_like_dev(200)
    h.expm(to_dev(A), out, 0.0, api.SCHEME_PADE26 | api.PREC_OZAKI)
    want, _ = O.expm(A, "pade26")
    assert rel_fro(to_host(out), want) < 1e-12
