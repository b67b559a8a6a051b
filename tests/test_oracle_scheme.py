"""Pins for the oracle's polynomial evaluation (Section 3 schemes, eq. poli9,
eq. pade10/pade26) and its product counts (Table 3)."""
import json
import os
from fractions import Fraction
from math import factorial

import numpy as np
import pytest

import ratmat as R
from oracle import oracle as O
from oracle import theta as TH

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


# spectral radius ~3.5: every Taylor degree up to 19 is visible far above rounding
WIDE = np.array([[3.0, 1.0, 0.5], [-1.0, 2.5, 0.25], [0.5, -0.75, 3.5]])


def dyadic_matrix(n, seed, target):
    """Tiny matrix with dyadic-rational entries (exact in binary) and 1-norm near target."""
    rng = np.random.default_rng(seed)
    A = rng.integers(-8, 9, size=(n, n)).astype(np.float64)
    A *= 2.0 ** np.round(np.log2(target / np.abs(A).sum(0).max()))
    return A


# ---- coefficient tables ---------------------------------------------------------------

def test_t8_closed_forms_exact():
    sp = pytest.importorskip("sympy")
    r = sp.sqrt(177)
    x3 = sp.Rational(2, 3)
    x1 = x3 * (1 + r) / 88
    x2 = (1 + r) / 352 * x3
    x4 = (-271 + 29 * r) / (315 * x3)
    x5 = 11 * (-1 + r) / (1260 * x3)
    x6 = 11 * (-9 + r) / (5040 * x3)
    x7 = (89 - r) / (5040 * x3 ** 2)
    y2 = (857 - 58 * r) / 630
    x = sp.symbols("x")
    A2 = x ** 2
    A4 = A2 * (x1 * x + x2 * A2)
    A8 = (x3 * A2 + A4) * (x4 + x5 * x + x6 * A2 + x7 * A4)
    T8 = sp.expand(1 + x + y2 * A2 + A8)
    poly = sp.Poly(T8, x)
    assert poly.degree() == 8
    for k in range(9):
        assert sp.simplify(poly.coeff_monomial(x ** k) - sp.Rational(1, factorial(k))) == 0
    # the oracle's doubles evaluate those closed forms in double precision; y2 has
    # cancellation (857 - 771.6), so a few ulps are expected there
    got = O.coeffs(1)
    want = [x1, x2, x3, x4, x5, x6, x7, 1, 1, y2]
    for g, w in zip(got, want):
        assert g == pytest.approx(float(sp.N(w, 30)), rel=4e-15, abs=0)


def _t12_poly(a):
    """Coefficients of T12 built from a_{i,j} (exact rationals of the given doubles)."""
    x = [Fraction(0), Fraction(1)]

    def P(c):  # list-of-coeffs polynomial helpers
        return [Fraction(v) for v in c]

    def mulp(p, q):
        out = [Fraction(0)] * (len(p) + len(q) - 1)
        for i, pi in enumerate(p):
            for j, qj in enumerate(q):
                out[i + j] += pi * qj
        return out

    def addp(p, q):
        n = max(len(p), len(q))
        return [(p[i] if i < len(p) else 0) + (q[i] if i < len(q) else 0) for i in range(n)]

    B = [P([a[i][j] for i in range(4)]) for j in range(4)]
    A6 = addp(B[2], mulp(B[3], B[3]))
    return addp(B[0], mulp(addp(B[1], A6), A6)), mulp, addp


def test_t12_coefficients_reproduce_taylor():
    c = O.coeffs(2).reshape(4, 4)  # c[i][j-1] = a_{i,j}
    p, _, _ = _t12_poly(c.tolist())
    assert len(p) == 13 and p[12] != 0
    dev = [abs(float(p[k] * factorial(k)) - 1.0) for k in range(13)]
    assert max(dev) < 1e-14, dev


def test_t18_coefficients_reproduce_taylor():
    c = O.coeffs(3)
    a1 = [Fraction(v) for v in c[:4]]
    b = [[Fraction(v) for v in c[4 + 4 * i: 8 + 4 * i]] for i in range(5)]  # rows i = 0,1,2,3,6
    _, mulp, addp = _t12_poly(np.zeros((4, 4)).tolist())

    def Bj(j):  # polynomial in x of b_{i,j}, i in {0,1,2,3,6}
        p = [Fraction(0)] * 7
        for r, deg in enumerate((0, 1, 2, 3, 6)):
            p[deg] += b[r][j]
        return p

    B1 = a1
    B2, B3, B4, B5 = Bj(0), Bj(1), Bj(2), Bj(3)
    A9 = addp(mulp(B1, B5), B4)
    T = addp(B2, mulp(addp(B3, A9), A9))
    assert len(T) == 19 and T[18] != 0
    dev = [abs(float(T[k] * factorial(k)) - 1.0) for k in range(19)]
    # printed to 18-20 digits; relative coefficient error of the top terms ~2e-15
    assert max(dev[:16]) < 4e-15, dev
    assert max(dev) < 1e-14, dev


def test_pade_coefficients_match_formula():
    for which, m in ((4, 13), (5, 5)):
        got = O.coeffs(which)
        want = TH.pade_p(m)
        assert len(got) == m + 1
        for g, w in zip(got, want):
            assert g == pytest.approx(float(w), rel=2e-15)


# ---- matrix evaluation against exact rational sums -------------------------------------

@pytest.mark.parametrize("m", [1, 2, 4, 8, 12, 18])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_new_scheme_equals_exact_taylor(m, seed):
    X = WIDE if seed == 0 else dyadic_matrix(3, seed, 4.0)
    got = O.taylor_new(X, m)
    Xf = R.to_frac(X)
    exact = R.to_float(R.taylor(Xf, m))
    nxt = R.to_float(R.taylor(Xf, m + 1))
    err = np.abs(got - exact).max() / np.abs(exact).max()
    assert err < 1e-12, err
    if seed == 0:  # and it is degree m, not m+1
        assert np.abs(nxt - exact).max() / np.abs(exact).max() > 1e3 * max(err, 1e-16)


@pytest.mark.parametrize("m", [1, 2, 4, 6, 9, 12, 16])
def test_ps_equals_exact_taylor(m):
    X = WIDE
    got = O.taylor_ps(X, m)
    Xf = R.to_frac(X)
    exact = R.to_float(R.taylor(Xf, m))
    nxt = R.to_float(R.taylor(Xf, m + 1))
    err = np.abs(got - exact).max() / np.abs(exact).max()
    assert err < 1e-12, err
    assert np.abs(nxt - exact).max() / np.abs(exact).max() > 1e3 * max(err, 1e-16)


@pytest.mark.parametrize("two_m", [10, 26])
def test_pade_equals_exact_quotient(two_m):
    X = dyadic_matrix(3, 4, 2.0)
    got = O.pade(X, two_m)
    p = TH.pade_p(two_m // 2)
    Xf = R.to_frac(X)
    num = R.poly(Xf, p)
    den = R.poly(Xf, [c * (-1) ** j for j, c in enumerate(p)])
    exact = R.to_float(R.mul(R.inv(den), num))
    err = np.abs(got - exact).max() / np.abs(exact).max()
    assert err < 1e-13, err


# ---- Table 3 -----------------------------------------------------------------------------

def _count(f, X, m):
    c0 = O.product_count()
    f(X, m)
    return O.product_count() - c0


def test_product_counts_table3():
    X = dyadic_matrix(4, 5, 1.0)
    t3 = GOLD["table3_products"]
    new = dict(zip(t3["new_decomposition"]["degree"], t3["new_decomposition"]["products"]))
    ps = dict(zip(t3["paterson_stockmeyer"]["degree"], t3["paterson_stockmeyer"]["products"]))
    for m in (2, 4, 8, 12, 18):
        assert _count(O.taylor_new, X, m) == new[m]
    assert _count(O.taylor_new, X, 1) == 0
    for m in (2, 4, 6, 9, 12, 16):
        assert _count(O.taylor_ps, X, m) == ps[m]
    pp = GOLD["pade_products"]
    assert _count(O.pade, X, 10) == pp["r10"]
    assert _count(O.pade, X, 26) == pp["r26"]
