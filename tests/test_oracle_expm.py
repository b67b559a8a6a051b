"""Pins for the oracle's whole scaling-and-squaring path (eq. eses, Section 4)
against closed forms, invariants, independent libraries and hand-checked
selections."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1710_10989_gb300 import workloads as W

SCHEMES = ("new", "ps", "pade26", "pade")


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# ---- closed forms ------------------------------------------------------------------------

@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("t", [1e-3, 0.1, 1.0, 3.0, 10.0, 40.0])
def test_rotation_generator(scheme, t):
    A = np.array([[0.0, -t], [t, 0.0]])
    E, info = O.expm(A, scheme)
    want = np.array([[math.cos(t), -math.sin(t)], [math.sin(t), math.cos(t)]])
    assert info.status == 0
    assert np.abs(E - want).max() < 1e-15 * 2 ** (info.s + 2), (info, np.abs(E - want).max())


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("scale", [1e-2, 0.7, 4.0, 30.0])
def test_diagonal(scheme, scale):
    d = np.linspace(-1.0, 1.0, 7) * scale
    E, info = O.expm(np.diag(d), scheme)
    want = np.exp(d)
    # r_26's denominator p_13(-x) cancels ~55-fold at x = 4, hence 1e-14 rather than ~1e-15
    assert np.abs(np.diag(E) - want).max() / want.max() < 1e-14 * 2 ** info.s
    assert np.abs(E - np.diag(np.diag(E))).max() == 0.0


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("c", [0.01, 0.5, 3.0, 20.0])
def test_nilpotent_shift(scheme, c):
    # A = c J, J the 6x6 upper shift: J^6 = 0, so e^A has c^k/k! on the k-th superdiagonal.
    n = 6
    A = c * np.eye(n, k=1)
    E, info = O.expm(A, scheme)
    want = sum(np.linalg.matrix_power(A, k) / math.factorial(k) for k in range(n))
    assert rel(E, want) < 1e-15 * 2 ** (info.s + 3), (info, rel(E, want))


# ---- invariants --------------------------------------------------------------------------

@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("norm", [0.05, 1.0, 8.0])
def test_inverse_and_determinant(scheme, norm):
    A = W.gaussian(24, 11, norm)
    E, _ = O.expm(A, scheme)
    F, _ = O.expm(-A, scheme)
    assert np.abs(E @ F - np.eye(24)).max() < 1e-13 * max(1.0, np.linalg.norm(E) * np.linalg.norm(F))
    sign, logdet = np.linalg.slogdet(E)
    assert sign > 0 and logdet == pytest.approx(np.trace(A), abs=1e-12 * max(1, norm))


@pytest.mark.parametrize("scheme", SCHEMES)
def test_symmetric_gives_spd(scheme):
    B = W.gaussian(20, 12, None)
    A = (B + B.T) * 2.0
    E, _ = O.expm(A, scheme)
    assert np.abs(E - E.T).max() < 1e-14 * np.abs(E).max()
    assert np.linalg.eigvalsh((E + E.T) / 2).min() > 0


def test_doubling_identity():
    A = W.gaussian(16, 13, 3.0)
    E, _ = O.expm(A)
    E2, _ = O.expm(2 * A)
    assert rel(E @ E, E2) < 1e-13


# ---- independent libraries ----------------------------------------------------------------

@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("n,norm", [(30, 0.01), (30, 1.0), (64, 5.0), (100, 20.0), (257, 100.0)])
def test_against_scipy(scheme, n, norm):
    sl = pytest.importorskip("scipy.linalg")
    A = W.gaussian(n, n + 7, norm)
    E, info = O.expm(A, scheme)
    assert rel(E, sl.expm(A)) < 2e-14 * 2 ** info.s


@pytest.mark.parametrize("norm", [0.3, 2.0, 25.0])
def test_against_mpmath_50_digits(norm):
    mp = pytest.importorskip("mpmath")
    A = W.gaussian(8, 21, norm)
    mp.mp.dps = 50
    ref = np.array(mp.expm(mp.matrix(A.tolist())).tolist(), dtype=np.float64)
    for scheme in SCHEMES:
        E, info = O.expm(A, scheme)
        assert rel(E, ref) < 1e-15 * 2 ** (info.s + 2), (scheme, info, rel(E, ref))


def test_nonnormal_upper_against_scipy():
    sl = pytest.importorskip("scipy.linalg")
    A = W.nonnormal_upper(40, 101, 5.0)
    E, _ = O.expm(A)
    assert rel(E, sl.expm(A)) < 1e-12


# ---- 1-norm and selection ------------------------------------------------------------------

def test_norm1_hand_value():
    # column sums 1+3 = 4 and 2+4 = 6; row sums would give 7
    assert O.norm1(np.array([[1.0, -2.0], [3.0, 4.0]])) == 6.0


# (norm, expected (m, s)) worked by hand from the printed thetas (Table 2) and the
# product counts (Table 3): cost = pi_m + s with s the least integer such that
# norm/2^s <= theta_m; ties go to the smaller s.
#   0.01: theta_8 = 0.0499 >= 0.01 -> (8,0) cost 3; (4,5) cost 7; (12,0) cost 4.
#   0.1 : theta_8 < 0.1 <= theta_12 = 0.2996 -> (12,0) cost 4; (8,2) cost 5.
#   0.5 : (18,0) cost 5 ties (12,1) cost 5 (0.25 <= 0.2996): smaller s wins.
#   1   : (18,0) cost 5; (12,2) cost 6.
#   5   : (18,3) (5/8 <= 1.09, 5/4 > 1.09) cost 8; (12,5) cost 9.
#   20  : (18,5) (0.625) cost 10.    100: (18,7) (0.78) cost 12.
NEW_TABLE = [(0.01, (8, 0)), (0.1, (12, 0)), (0.5, (18, 0)), (1.0, (18, 0)), (5.0, (18, 3)),
             (20.0, (18, 5)), (50.0, (18, 6)), (100.0, (18, 7)), (1e-20, (1, 0)), (1e-9, (2, 0)),
             (1e-4, (4, 0)), (0.0, (1, 0))]
# Paterson-Stockmeyer, same rule with degrees {1,2,4,6,9,12,16} and 0..6 products:
#   0.01: theta_6 = 9.07e-3 < 0.01 <= theta_9 = 0.0896 -> (9,0) cost 4 ; (6,1) cost 4 -> s=0 wins.
#   1   : theta_16 = 0.78 < 1 -> (16,1) cost 7; (12,2) cost 7 -> (16,1).
PS_TABLE = [(0.01, (9, 0)), (0.1, (12, 0)), (1.0, (16, 1)), (5.0, (16, 3)), (100.0, (16, 8))]
# Pade r_26 with theta_26 = 5.37 (Table 1): s = ceil(log2(norm/5.37)).
PADE_TABLE = [(1.0, (26, 0)), (5.0, (26, 0)), (20.0, (26, 2)), (100.0, (26, 5))]
# Pade r_10 or r_26 (3 or 6 products; the solve is common to both) with theta_10 = 0.254, theta_26 = 5.37:
#   1: r_10 needs s = 2 (0.25 <= 0.254): cost 5 < r_26's 6 -> (10,2)
#   2: r_10 s = 3 cost 6 = r_26 s = 0 cost 6 -> the smaller s: (26,0)
#   20: r_10 s = 7 cost 10 ; r_26 s = 2 cost 8 -> (26,2)
PADE_BOTH_TABLE = [(0.01, (10, 0)), (0.2, (10, 0)), (1.0, (10, 2)), (2.0, (26, 0)), (5.0, (26, 0)),
                   (20.0, (26, 2)), (100.0, (26, 5))]


def test_selection_tables():
    for norm, want in NEW_TABLE:
        assert O.select(norm, "new") == want, norm
    for norm, want in PS_TABLE:
        assert O.select(norm, "ps") == want, norm
    for norm, want in PADE_TABLE:
        assert O.select(norm, "pade26") == want, norm
    for norm, want in PADE_BOTH_TABLE:
        assert O.select(norm, "pade") == want, norm


def test_selection_boundary_is_inclusive():
    th18 = O.theta_array("new")[18]
    assert O.select(th18, "new") == (18, 0)
    assert O.select(np.nextafter(th18, 10.0), "new")[1] == 1


def test_selection_single_precision_row():
    # u = 2^-24 (Table 2, first row): theta_18 = 3.01 -> norm 3 fits with s = 0
    assert O.select(3.0, "new", 2.0 ** -24) == (18, 0)
    assert O.select(0.5, "new", 2.0 ** -24) == (8, 0)  # theta_8 = 0.580


def test_status_codes():
    A = np.eye(3)
    A[1, 2] = np.nan
    _, info = O.expm(A)
    assert info.status == 2
    _, info = O.expm(np.eye(2) * 800.0)  # e^800 overflows double
    assert info.status == 3
    E, info = O.expm(np.zeros((5, 5)))
    assert info.status == 0 and (E == np.eye(5)).all()


def test_forced_parameters_are_used():
    A = W.gaussian(10, 3, 2.0)
    E1, i1 = O.expm(A, m=18, s=4)
    assert (i1.m, i1.s, i1.products) == (18, 4, 9)
    E2, i2 = O.expm(A)
    assert rel(E1, E2) < 1e-14


@pytest.mark.parametrize("scheme", SCHEMES)
def test_one_by_one_is_the_scalar_exponential(scheme):
    """N = 1, the degenerate size: T_m(a / 2^s)^(2^s) is the scalar exponential, to
    rounding: each squaring doubles a relative error, and alternating sums at
    x = a / 2^s (Taylor's for a < 0, a Pade denominator's for a > 0) cancel by up to e^(2|x|)."""
    for a in (-30.0, -1.0, -1e-9, 0.0, 1e-300, 0.5, 2.0, 40.0, 700.0):
        E, info = O.expm(np.array([[a]]), scheme)
        assert info.status == 0
        cancel = math.exp(2.0 * abs(a) / 2 ** info.s)
        assert abs(E[0, 0] - math.exp(a)) <= 4e-16 * 2 ** info.s * cancel * math.exp(a), (a, info, E[0, 0])


def test_extreme_norms_keep_their_closed_forms():
    """At 1-norms far past where A A overflows (the oracle forms X = 2^-s A before any
    product): exp of a huge nilpotent shift is I + A, of -1e200 I it is 0."""
    E, info = O.expm(np.array([[0.0, 1e200], [0.0, 0.0]]))
    assert info.status == 0 and info.s == 665
    assert E[0, 0] == 1.0 and E[1, 1] == 1.0 and E[1, 0] == 0.0
    assert abs(E[0, 1] - 1e200) <= 1e-14 * 1e200   # T's X coefficient, then exact doublings
    E, info = O.expm(-1e200 * np.eye(3))
    assert info.status == 0 and (E == 0.0).all()
