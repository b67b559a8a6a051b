"""Exact rational matrix arithmetic for pins (pure Python Fractions).

Independent of both implementations: used only to build exact Taylor sums
and exact Pade quotients on tiny matrices.
"""
from __future__ import annotations

from fractions import Fraction
from math import factorial

import numpy as np


def to_frac(A) -> list[list[Fraction]]:
    return [[Fraction(float(x)) for x in row] for row in np.asarray(A, dtype=np.float64)]


def eye(n):
    return [[Fraction(int(i == j)) for j in range(n)] for i in range(n)]


def mul(A, B):
    n = len(A)
    return [[sum(A[i][k] * B[k][j] for k in range(n)) for j in range(n)] for i in range(n)]


def add(A, B, b=Fraction(1)):
    return [[a + b * c for a, c in zip(ra, rb)] for ra, rb in zip(A, B)]


def scale(A, c):
    return [[c * a for a in r] for r in A]


def taylor(X, m: int):
    """sum_{k=0}^m X^k / k!, exactly."""
    n = len(X)
    T, P = eye(n), eye(n)
    for k in range(1, m + 1):
        P = mul(P, X)
        T = add(T, P, Fraction(1, factorial(k)))
    return T


def poly(X, coeffs):
    """sum_k coeffs[k] X^k for exact rational coefficients."""
    n = len(X)
    T = [[Fraction(0)] * n for _ in range(n)]
    P = eye(n)
    for c in coeffs:
        T = add(T, P, Fraction(c))
        P = mul(P, X)
    return T


def inv(A):
    """Gauss-Jordan inverse in exact arithmetic."""
    n = len(A)
    M = [list(r) + [Fraction(int(i == j)) for j in range(n)] for i, r in enumerate(A)]
    for c in range(n):
        p = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        piv = M[c][c]
        M[c] = [x / piv for x in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [x - f * y for x, y in zip(M[r], M[c])]
    return [r[n:] for r in M]


def to_float(A) -> np.ndarray:
    return np.array([[float(x) for x in r] for r in A])
