"""exp(A) for complex A by the paper's method, in plain numpy complex128.

TEST INFRASTRUCTURE: only the tests, smoke() and the benchmark's CPU legs use
it; the library never does.

The paper states the problem for A in C^{N x N} (Section 2): the backward-error
thresholds theta_m(u) (eq. theta) bound ||2^-s A||_1, with ||.||_1 the largest
column sum of moduli, whatever the field. This module follows the same steps as
the real oracle, in complex arithmetic and in the paper's order:

  ||A||_1 (moduli)  ->  (m, s) by the theta rule (the real oracle's selection,
  pinned by its own tests)  ->  X = 2^-s A  ->  T_m(X) by the reduced-product
  scheme of Section 3 (T1, T2, T4, and T8 / T12 / T18 of eq. Algorithm83eA,
  eq. poly12, eq. poly.18, coefficients from the real oracle's tables)  ->  s
  squarings (eq. eses).

Products are numpy matmuls (a library primitive used as one step); linear
combinations are written out term by term. No real embedding is used, so the
GPU path, which does use one, is checked against independent complex
arithmetic.

_MUTATION plants one mistake for the negative-control tests (0 = none):
  1  the norm sums |Re a| only          2  X conjugated in the first product
  3  T18 takes B4 where B3 belongs      4  X transposed in X3 = X2 X
"""
from __future__ import annotations

import numpy as np

from . import oracle as _real

_MUTATION = 0


def set_mutation(code: int) -> None:
    global _MUTATION
    _MUTATION = int(code)


def norm1(A: np.ndarray) -> float:
    """max_j sum_i |a_ij| with |.| the complex modulus."""
    A = np.asarray(A, dtype=np.complex128)
    if _MUTATION == 1:
        return float(np.max(np.sum(np.abs(A.real), axis=0))) if A.size else 0.0
    return float(np.max(np.sum(np.abs(A), axis=0))) if A.size else 0.0


def _mm(P: np.ndarray, Q: np.ndarray) -> np.ndarray:
    return P @ Q


def _lin(n: int, c0: complex, terms) -> np.ndarray:
    """c0 I + sum_k c_k M_k, one term at a time."""
    out = np.zeros((n, n), dtype=np.complex128)
    out[np.diag_indices(n)] = c0
    for c, M in terms:
        out = out + c * M
    return out


def taylor_new(X: np.ndarray, m: int) -> np.ndarray:
    """T_m(X) by the reduced-product scheme (Section 3) for m in {1, 2, 4, 8, 12, 18}."""
    X = np.asarray(X, dtype=np.complex128)
    n = X.shape[0]
    X2 = _mm(np.conj(X) if _MUTATION == 2 else X, X) if m >= 2 else None
    if m == 1:
        return _lin(n, 1.0, [(1.0, X)])
    if m == 2:
        return _lin(n, 1.0, [(1.0, X), (0.5, X2)])
    if m == 4:  # I + X + X2 (I/2 + X/6 + X2/24)
        P = _lin(n, 0.5, [(1.0 / 6.0, X), (1.0 / 24.0, X2)])
        return _lin(n, 1.0, [(1.0, X)]) + _mm(X2, P)
    if m == 8:  # eq. Algorithm83eA
        x1, x2, x3, x4, x5, x6, x7, y0, y1, y2 = _real.coeffs(1)
        X4 = _mm(X2, _lin(n, 0.0, [(x1, X), (x2, X2)]))
        X8 = _mm(_lin(n, 0.0, [(x3, X2), (1.0, X4)]), _lin(n, x4, [(x5, X), (x6, X2), (x7, X4)]))
        return _lin(n, y0, [(y1, X), (y2, X2)]) + X8
    if m == 12:  # eq. poly12
        a = _real.coeffs(2).reshape(4, 4)  # a[i][j]: coefficient of X^i in B_{j+1}
        X3 = _mm(X2, X.T if _MUTATION == 4 else X)
        B = [_lin(n, a[0][j], [(a[1][j], X), (a[2][j], X2), (a[3][j], X3)]) for j in range(4)]
        X6 = _mm(B[3], B[3]) + B[2]                                   # B3 + B4^2
        return B[0] + _mm(B[1] + X6, X6)                              # B1 + (B2 + X6) X6
    if m == 18:  # eq. poly.18
        c = _real.coeffs(3)
        a1, b = c[:4], c[4:].reshape(5, 4)  # b[i][j]: coefficient of X^{0,1,2,3,6}[i] in B_{j+2}
        X3 = _mm(X2, X.T if _MUTATION == 4 else X)
        X6 = _mm(X3, X3)
        B1 = _lin(n, a1[0], [(a1[1], X), (a1[2], X2), (a1[3], X3)])
        Bj = [_lin(n, b[0][j], [(b[1][j], X), (b[2][j], X2), (b[3][j], X3), (b[4][j], X6)]) for j in range(4)]
        X9 = _mm(B1, Bj[3]) + Bj[2]                                   # B1 B5 + B4
        B3 = Bj[2] if _MUTATION == 3 else Bj[1]
        return Bj[0] + _mm(B3 + X9, X9)                               # B2 + (B3 + X9) X9
    raise ValueError(f"unsupported degree {m}")


def expm(A, u: float = 2.0 ** -53, m: int | None = None, s: int | None = None):
    """exp(A) for complex A; (m, s) by the theta rule on the complex 1-norm unless
    both are given. Returns (exp(A), (m, s, products, norm1))."""
    A = np.ascontiguousarray(A, dtype=np.complex128)
    nrm = norm1(A)
    if m is None or s is None:
        m, s = _real.select(nrm, "new", u)
    X = A * (2.0 ** -s)
    T = taylor_new(X, m)
    for _ in range(s):
        T = _mm(T, T)
    products = {1: 0, 2: 1, 4: 2, 8: 3, 12: 4, 18: 5}[m] + s
    return T, (m, s, products, nrm)
