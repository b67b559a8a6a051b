"""Pins of the oracle's linear solve (the Pade comparator's step (v - u) R = u + v,
eq. pade26; Gaussian elimination with partial pivoting on all right-hand sides):
exact rational solutions of small systems, LAPACK (numpy) on larger ones, a
system that cannot be solved without row interchanges, and a singular one."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O


def exact_solve(P, Q):
    """P^-1 Q in exact rational arithmetic (Gauss-Jordan, any non-zero pivot)."""
    n = len(P)
    M = [[Fraction(float(x)) for x in P[i]] + [Fraction(float(x)) for x in Q[i]] for i in range(n)]
    for k in range(n):
        r = next(i for i in range(k, n) if M[i][k] != 0)
        M[k], M[r] = M[r], M[k]
        d = M[k][k]
        M[k] = [x / d for x in M[k]]
        for i in range(n):
            if i != k and M[i][k] != 0:
                f = M[i][k]
                M[i] = [a - f * b for a, b in zip(M[i], M[k])]
    return np.array([[float(x) for x in row[n:]] for row in M])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_solve_matches_exact_rational(seed):
    rng = np.random.default_rng(seed)
    n = 6
    P = rng.integers(-9, 10, size=(n, n)).astype(np.float64)
    P += np.diag(rng.integers(1, 3, size=n))          # keep it comfortably non-singular
    Q = rng.integers(-9, 10, size=(n, n)).astype(np.float64)
    got = O.solve(P, Q)
    want = exact_solve(P, Q)
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()


def test_solve_needs_row_interchanges():
    """A zero leading entry (and zero pivots further down without interchanges):
    only partial pivoting solves it."""
    P = np.array([[0.0, 2.0, 1.0, 0.0], [1.0, 0.0, 0.0, 3.0], [0.0, 1.0, 0.0, 0.0], [2.0, 0.0, 1.0, 1.0]])
    Q = np.arange(16.0).reshape(4, 4) - 5.0
    got = O.solve(P, Q)
    want = exact_solve(P, Q)
    assert np.abs(got - want).max() <= 1e-14 * np.abs(want).max()


@pytest.mark.parametrize("n", [1, 37, 120])
def test_solve_matches_lapack(n):
    rng = np.random.default_rng(n)
    P = rng.standard_normal((n, n))
    Q = rng.standard_normal((n, n))
    got = O.solve(P, Q)
    want = np.linalg.solve(P, Q)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-11 * np.linalg.cond(P) / n


def test_singular_is_reported():
    P = np.array([[1.0, 2.0], [2.0, 4.0]])
    with pytest.raises(ValueError):
        O.solve(P, np.eye(2))
