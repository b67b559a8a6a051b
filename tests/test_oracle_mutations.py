"""Negative controls: plant one plausible mistake at a time in the oracle (on
the CPU, through its mutation switch) and check that the pins catch it."""
import math

import numpy as np
import pytest

import ratmat as R
from oracle import oracle as O
from oracle import theta as TH

WIDE = np.array([[3.0, 1.0, 0.5], [-1.0, 2.5, 0.25], [0.5, -0.75, 3.5]])


def _taylor_pins() -> bool:
    Xf = R.to_frac(WIDE)
    for m in (8, 12, 18):
        exact = R.to_float(R.taylor(Xf, m))
        if np.abs(O.taylor_new(WIDE, m) - exact).max() / np.abs(exact).max() > 1e-12:
            return False
    for m in (4, 6, 9, 12, 16):
        exact = R.to_float(R.taylor(Xf, m))
        if np.abs(O.taylor_ps(WIDE, m) - exact).max() / np.abs(exact).max() > 1e-12:
            return False
    return True


def _closed_form_pins() -> bool:
    for scheme in ("new", "ps", "pade26"):
        for t in (1.0, 10.0):
            A = np.array([[0.0, -t], [t, 0.0]])
            E, info = O.expm(A, scheme)
            want = np.array([[math.cos(t), -math.sin(t)], [math.sin(t), math.cos(t)]])
            if np.abs(E - want).max() > 1e-15 * 2 ** (info.s + 2):
                return False
    return True


def _norm_and_selection_pins() -> bool:
    if O.norm1(np.array([[1.0, -2.0], [3.0, 4.0]])) != 6.0:
        return False
    table = [(0.01, (8, 0)), (0.1, (12, 0)), (5.0, (18, 3)), (100.0, (18, 7))]
    pade = [(0.2, (10, 0)), (1.0, (10, 2)), (2.0, (26, 0)), (20.0, (26, 2))]
    return (all(O.select(n, "new") == w for n, w in table)
            and all(O.select(n, "pade") == w for n, w in pade))


def _coefficient_pins() -> bool:
    c = O.coeffs(2).reshape(4, 4)
    from test_oracle_scheme import _t12_poly  # noqa: E402
    p, _, _ = _t12_poly(c.tolist())
    return max(abs(float(p[k] * math.factorial(k)) - 1.0) for k in range(13)) < 1e-14


def _triangular_pins() -> bool:
    """exp([[a, b], [0, c]]) in closed form (divided difference of exp, evaluated
    as e^a (e^(c-a) - 1)/(c - a) with expm1: no cancellation), and the diagonal
    of exp of an upper triangular matrix, e^{a_ii}."""
    for a, b, c in ((1.0, 1e4, 1.0 + 1e-7), (-3.0, 250.0, 2.5)):
        E, _ = O.expm_upper(np.array([[a, b], [0.0, c]]))
        sup = b * math.exp(a) * math.expm1(c - a) / (c - a)
        if abs(E[0, 1] - sup) > 1e-14 * abs(sup) or E[0, 0] != math.exp(a) or E[1, 1] != math.exp(c):
            return False
    rng = np.random.default_rng(3)
    A = np.triu(rng.standard_normal((12, 12))) * 4.0
    E, _ = O.expm_upper(A)
    return all(E[i, i] == math.exp(A[i, i]) for i in range(12))


def _solve_pins() -> bool:
    from test_oracle_solve import exact_solve
    P = np.array([[0.0, 2.0, 1.0, 0.0], [1.0, 0.0, 0.0, 3.0], [0.0, 1.0, 0.0, 0.0], [2.0, 0.0, 1.0, 1.0]])
    Q = np.arange(16.0).reshape(4, 4) - 5.0
    try:
        got = O.solve(P, Q)
    except ValueError:
        return False
    want = exact_solve(P, Q)
    return bool(np.all(np.isfinite(got))) and np.abs(got - want).max() <= 1e-14 * np.abs(want).max()


def all_pins_pass() -> bool:
    return (_taylor_pins() and _closed_form_pins() and _norm_and_selection_pins()
            and _coefficient_pins() and _triangular_pins() and _solve_pins())


MUTATIONS = {
    1: "T12 a_{0,4} dropped (looks like noise, is not)",
    2: "T18 b_{6,3} sign flipped",
    3: "T8 x5 and x6 swapped",
    4: "T18 A9 = B1 B5 without + B4",
    5: "product computes A B^T (transposed operand)",
    6: "Paterson-Stockmeyer top coefficient dropped",
    7: "Pade numerator and denominator swapped",
    8: "one squaring too few",
    9: "infinity-norm instead of 1-norm",
    10: "triangular path: superdiagonal without the divided difference of exp",
    11: "triangular path: exact diagonals not put back after the last squaring",
    12: "Pade scheme: r_10 charged 6 products, as r_26",
    13: "comparator's solve without row interchanges",
}


def test_clean_oracle_passes_pins():
    O.set_mutation(0)
    assert all_pins_pass()


@pytest.mark.parametrize("code", sorted(MUTATIONS))
def test_planted_mistake_is_caught(code):
    try:
        O.set_mutation(code)
        assert not all_pins_pass(), MUTATIONS[code]
    finally:
        O.set_mutation(0)
