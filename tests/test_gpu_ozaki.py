"""GPU parity, split-precision path: products rebuilt exactly from BF16 slices on
the tcgen05 tensor cores, checked against the oracle's FP64 products and, for
small-integer operands, against the exact integer product."""
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


def oz(api, k=7):
    return api.PREC_OZAKI | api.ozaki_slices(k)


@pytest.mark.parametrize("n", [128, 1, 5, 64, 200, 256, 257, 1100, 2048])
def test_integer_operands_are_exact(h, api, n):
    # entries in [-127, 127] times a power of two per row / column: two slices hold
    # them exactly, so the product must be exact (it fits FP64 exactly as well)
    rng = np.random.default_rng(n)
    P = rng.integers(-127, 128, size=(n, n)).astype(np.float64) * np.ldexp(1.0, rng.integers(-5, 5, size=(n, 1)))
    Q = rng.integers(-127, 128, size=(n, n)).astype(np.float64) * np.ldexp(1.0, rng.integers(-5, 5, size=(1, n)))
    C = empty_like_dev(n)
    h.gemm(to_dev(P), to_dev(Q), C, oz(api, 2))
    exact = O.gemm(P, Q)  # every partial sum is an exact binary64 value here
    assert np.array_equal(to_host(C), exact)


@pytest.mark.parametrize("n", [1, 7, 64, 128, 255, 256, 300, 1025])
def test_gemm_matches_oracle(h, api, n):
    P = W.gaussian(n, 3 + n, None)
    Q = W.gaussian(n, 4 + n, None)
    C = empty_like_dev(n)
    h.gemm(to_dev(P), to_dev(Q), C, oz(api, 7))
    assert rel_fro(to_host(C), O.gemm(P, Q)) < 4e-16 * max(4, np.sqrt(n))


def test_error_falls_with_slices(h, api):
    n = 384
    P = W.gaussian(n, 31, None)
    Q = W.gaussian(n, 32, None)
    ref = O.gemm(P, Q)
    errs = []
    for k in (2, 3, 4, 5, 6, 7, 8):
        C = empty_like_dev(n)
        h.gemm(to_dev(P), to_dev(Q), C, oz(api, k))
        errs.append(rel_fro(to_host(C), ref))
    # about 8 bits per extra slice until FP64 rounding is reached
    for k, (a, b) in enumerate(zip(errs, errs[1:]), start=2):
        if a > 1e-13:
            assert b < a / 50, (k, errs)
    assert errs[-2] < 1e-15 and errs[-1] < 1e-15, errs


def test_wide_dynamic_range_rows(h, api):
    n = 200
    rng = np.random.default_rng(5)
    rs = rng.integers(-300, 300, size=(n, 1))
    cs = rng.integers(-300, 300, size=(1, n))
    P0 = rng.standard_normal((n, n))
    Q0 = rng.standard_normal((n, n))
    C = empty_like_dev(n)
    h.gemm(to_dev(np.ldexp(P0, rs)), to_dev(np.ldexp(Q0, cs)), C, oz(api, 7))
    # row i / column j scales are exact powers of two: remove them and compare
    got = np.ldexp(to_host(C), -(rs + cs))
    assert rel_fro(got, O.gemm(P0, Q0)) < 4e-15


def test_nonfinite_operand_reported(h, api):
    P = np.eye(130)
    P[3, 4] = np.inf
    C = empty_like_dev(130)
    with pytest.raises(api.BBCError) as e:
        h.gemm(to_dev(P), to_dev(np.eye(130)), C, oz(api, 7))
    assert e.value.code == api.OVERFLOW


@pytest.mark.parametrize("idx", range(6))
@pytest.mark.parametrize("n,nonnormal", [(192, False), (300, True)])
def test_expm_split_matches_oracle(h, api, idx, n, nonnormal):
    A = W.dense_case(idx, n=n, nonnormal=nonnormal)
    out = empty_like_dev(n)
    info = h.expm(to_dev(A), out, 0.0, api.SCHEME_NEW | oz(api, 7))
    want, oi = O.expm_upper(A, "new") if nonnormal else O.expm(A, "new")
    assert info.structure == (1 if nonnormal else 0)
    assert (info.m, info.s, info.products) == (oi.m, oi.s, oi.products)
    assert rel_fro(to_host(out), want) < 1e-12


def test_small_workload_split(h, api):
    A = W.small_case()
    out = empty_like_dev(64)
    h.expm(to_dev(A), out, 0.0, api.SCHEME_NEW | oz(api, 7))
    want, _ = O.expm(A, "new")
    assert rel_fro(to_host(out), want) < 1e-13


def test_identity_dominated_operands(h, api):
    # T = I + X + ... and the B_j of the scheme are dominated by their diagonal;
    # the diagonal is deflated before slicing, so 7 slices keep full accuracy
    n = 1024
    P = np.eye(n) * 1.5 + 0.05 * W.gaussian(n, 41, None)
    Q = np.eye(n) * -0.75 + 0.05 * W.gaussian(n, 42, None)
    C64 = empty_like_dev(n)
    h.gemm(to_dev(P), to_dev(Q), C64, api.PREC_FP64)
    for k in (7, 8):
        C = empty_like_dev(n)
        h.gemm(to_dev(P), to_dev(Q), C, oz(api, k))
        assert rel_fro(to_host(C), to_host(C64)) < 5e-15, k


def test_split_product_is_closer_to_exact_than_fp64(h, api):
    """Sampled entries of P Q computed exactly (rational arithmetic on the binary64
    inputs): the split product (exact slice sums) lands closer to them than the
    FP64 product, whose k-sum rounds at every step."""
    from fractions import Fraction
    n = 2048
    P = W.gaussian(n, 51, None)
    Q = W.gaussian(n, 52, None)
    Cs, Cf = empty_like_dev(n), empty_like_dev(n)
    h.gemm(to_dev(P), to_dev(Q), Cs, oz(api, 7))
    h.gemm(to_dev(P), to_dev(Q), Cf, api.PREC_FP64)
    Cs, Cf = to_host(Cs), to_host(Cf)
    rng = np.random.default_rng(0)
    es, ef = [], []
    for i, j in rng.integers(0, n, size=(24, 2)):
        exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(P[i], Q[:, j]))
        scale = float(np.abs(P[i]) @ np.abs(Q[:, j]))
        es.append(abs(float(Fraction(float(Cs[i, j])) - exact)) / scale)
        ef.append(abs(float(Fraction(float(Cf[i, j])) - exact)) / scale)
    assert max(es) < 1e-16                   # ~ the final rounding only
    assert max(es) < max(ef)


# ---- the literal split (BBC_PREC_SPLIT) and FP64 final squarings ----------------------------------

def test_literal_split_products(h, api):
    """Plain floating-point BF16 splitting with FP32 accumulation: about 8 bits per
    term until the FP32 sums limit it; far from the exact form at the same k."""
    n = 512
    P = W.gaussian(n, 71, None)
    Q = W.gaussian(n, 72, None)
    ref = O.gemm(P, Q)
    err = {}
    for k in (2, 3, 4):
        C = empty_like_dev(n)
        h.gemm(to_dev(P), to_dev(Q), C, api.PREC_SPLIT | api.ozaki_slices(k))
        err[k] = rel_fro(to_host(C), ref)
    assert 1e-9 < err[3] < 1e-5, err
    assert err[2] > err[3], err
    assert err[4] > 0.5 * err[3], err   # a fourth term buys nothing: the FP32 sums set the floor
    C = empty_like_dev(n)
    h.gemm(to_dev(P), to_dev(Q), C, oz(api, 7))
    assert rel_fro(to_host(C), ref) < 1e-15   # the exact form, for contrast


def test_literal_split_expm_and_fp64_last_squarings(h, api):
    A = W.gaussian(300, 73, 20.0)      # s = 5
    want, oi = O.expm(A, "new")
    out = empty_like_dev(300)
    info = h.expm(to_dev(A), out, 0.0, api.PREC_SPLIT)
    e_lit = rel_fro(to_host(out), want)
    info2 = h.expm(to_dev(A), out, 0.0, api.PREC_SPLIT | api.square_fp64_last(oi.s))
    e_last = rel_fro(to_host(out), want)
    info3 = h.expm(to_dev(A), out, 0.0, api.PREC_FP64 | api.square_fp64_last(2))
    e_fp64 = rel_fro(to_host(out), want)
    assert (info.m, info.s) == (info2.m, info2.s) == (info3.m, info3.s) == (oi.m, oi.s)
    assert 1e-10 < e_lit < 1e-4
    assert e_last < e_lit            # FP64 squarings stop the 2^s amplification
    assert e_fp64 < 1e-12            # an all-FP64 run is unchanged by the flag


# ---- the literal split in TF32 terms (BBC_PREC_SPLIT_TF32, BBC_PREC_FP32; kind::tf32 MMAs) ------------

@pytest.mark.parametrize("n", [1, 7, 64, 200, 256, 300])
@pytest.mark.parametrize("upper", [False, True])
def test_tf32_terms_exact_on_small_integers(h, api, n, upper):
    """Entries of at most 7 significant bits (integers up to 127 times a power of two
    per row / column) are one TF32 term each, and every partial sum of their products
    stays below 300 x 127^2 < 2^24, so the FP32 accumulation is exact: the TF32 path
    must give the exact product. Pins the kind::tf32 descriptor, the 32-bit TMA layout
    and the K steps of 32 elements, also on triangles (K ranges per tile)."""
    rng = np.random.default_rng(1000 + n)
    P = rng.integers(-127, 128, size=(n, n)).astype(np.float64) * np.ldexp(1.0, rng.integers(-6, 6, size=(n, 1)))
    Q = rng.integers(-127, 128, size=(n, n)).astype(np.float64) * np.ldexp(1.0, rng.integers(-6, 6, size=(1, n)))
    flags = api.PREC_SPLIT_TF32 | api.ozaki_slices(2)
    if upper:
        P, Q = np.triu(P), np.triu(Q)
        flags |= api.UPPER
    C = empty_like_dev(n)
    h.gemm(to_dev(P), to_dev(Q), C, flags)
    assert np.array_equal(to_host(C), O.gemm(P, Q))


def test_tf32_literal_split_products(h, api):
    """Two TF32 terms per operand (about 22 significant bits) with FP32 sums: the
    error sits at the FP32 accumulation floor (as the 3-term BF16 split's does), so
    a third term (BBC_PREC_FP32) is no worse and no better than that floor; all far
    from the exact form."""
    n = 512
    P = W.gaussian(n, 71, None)
    Q = W.gaussian(n, 72, None)
    ref = O.gemm(P, Q)
    err = {}
    for name, fl in (("tf32x2", api.PREC_SPLIT_TF32), ("tf32x3", api.PREC_SPLIT_TF32 | api.ozaki_slices(3)),
                     ("fp32", api.PREC_FP32), ("bf16x3", api.PREC_SPLIT)):
        C = empty_like_dev(n)
        h.gemm(to_dev(P), to_dev(Q), C, fl)
        err[name] = rel_fro(to_host(C), ref)
    print("literal split product errors (N = 512):", {k: f"{v:.2e}" for k, v in err.items()})
    assert 1e-8 < err["tf32x2"] < 1e-5, err
    assert err["tf32x3"] <= 1.5 * err["tf32x2"], err
    assert err["fp32"] == err["tf32x3"], err          # BBC_PREC_FP32 is the 3-term TF32 split
    assert 0.2 < err["tf32x2"] / err["bf16x3"] < 5, err


def test_tf32_flag_checks(h, api):
    P = to_dev(np.eye(8))
    with pytest.raises(api.BBCError) as e:
        h.gemm(P, P, empty_like_dev(8), api.PREC_SPLIT_TF32 | api.ozaki_slices(5))
    assert e.value.code == api.INVALID_ARG
    with pytest.raises(api.BBCError) as e:
        h.gemm(P, P, empty_like_dev(8), api.PREC_FP32 | api.ozaki_slices(2))
    assert e.value.code == api.INVALID_ARG


def test_tf32_literal_expm(h, api):
    A = W.gaussian(300, 73, 20.0)      # s = 5
    want, oi = O.expm(A, "new")
    out = empty_like_dev(300)
    errs = {}
    for name, fl in (("tf32x2", api.PREC_SPLIT_TF32), ("tf32x2+fp64 last", api.PREC_SPLIT_TF32 |
                                                        api.square_fp64_last(oi.s)), ("fp32", api.PREC_FP32)):
        info = h.expm(to_dev(A), out, 0.0, fl)
        assert (info.m, info.s, info.products) == (oi.m, oi.s, oi.products)
        errs[name] = rel_fro(to_host(out), want)
    assert 1e-9 < errs["tf32x2"] < 1e-3, errs
    assert errs["tf32x2+fp64 last"] < errs["tf32x2"], errs
    assert errs["fp32"] <= 1.5 * errs["tf32x2"], errs


def test_split_beyond_largest_n_is_unsupported(h, api):
    """N = 16385, one past the split path's largest N: every split precision is
    refused before any work (the buffers are full size all the same)."""
    import torch
    n = 16385
    A = torch.empty((n, n), dtype=torch.float64, device="cuda")
    C = torch.empty_like(A)
    for fl in (oz(api, 6), api.PREC_SPLIT, api.PREC_SPLIT_TF32, api.PREC_FP32):
        with pytest.raises(api.BBCError) as e:
            h.gemm(A, A, C, fl)
        assert e.value.code == api.UNSUPPORTED
    with pytest.raises(api.BBCError) as e:
        h.expm(A, C, 0.0, oz(api, 6))
    assert e.value.code == api.UNSUPPORTED
    del A, C
    torch.cuda.empty_cache()
