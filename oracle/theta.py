"""Backward-error thresholds theta_m(u) -- oracle side.

TEST INFRASTRUCTURE: only the test suite, the smoke entry point and the
benchmark's CPU-baseline leg import this module. The CUDA library computes its
own thresholds with its own code.

Definition (Section 1, eq. theta and the paragraph after it): for an
approximant R of e^x (Taylor T_m or diagonal Pade r_2m), write

    rho(x) = log(e^{-x} R(x)) = sum_i c_i x^i,

take the majorant f(theta) = sum_i |c_i| theta^i, truncate it after 150
terms, and let theta(u) be the root of f(theta)/theta = u.  Reading of the
truncation: the 150 terms are the first 150 possibly non-zero ones, i.e.
i = m+1 .. m+150 for Taylor T_m and i = 2m+1 .. 2m+150 for Pade r_2m (all
lower c_i vanish exactly; the tests check that).

The series coefficients are exact rationals (fractions.Fraction); the root is
found by bisection in 60-digit decimal arithmetic. Pure standard library, so it
runs wherever Python runs.
"""
from __future__ import annotations

import functools
from decimal import Decimal, getcontext
from fractions import Fraction
from math import factorial

NTERMS = 150


def _mul(a: list[Fraction], b: list[Fraction], n: int) -> list[Fraction]:
    """Truncated product of two power series (coefficient lists), length n."""
    out = [Fraction(0)] * n
    for i, ai in enumerate(a[:n]):
        if ai == 0:
            continue
        for j, bj in enumerate(b[: n - i]):
            if bj:
                out[i + j] += ai * bj
    return out


def _log_series(h: list[Fraction], n: int) -> list[Fraction]:
    """log h(x) for a series with h[0] = 1, via g' = h'/h:
    n g_n = n h_n - sum_{k=1}^{n-1} k g_k h_{n-k}."""
    assert h[0] == 1
    g = [Fraction(0)] * n
    for k in range(1, n):
        acc = k * h[k]
        for j in range(1, k):
            if g[j] and h[k - j]:
                acc -= j * g[j] * h[k - j]
        g[k] = acc / k
    return g


def _exp_neg(n: int) -> list[Fraction]:
    return [Fraction((-1) ** k, factorial(k)) for k in range(n)]


@functools.lru_cache(maxsize=None)
def taylor_rho(m: int) -> tuple[Fraction, ...]:
    """Exact coefficients c_0..c_{m+NTERMS} of log(e^{-x} T_m(x))."""
    n = m + NTERMS + 1
    tm = [Fraction(1, factorial(k)) if k <= m else Fraction(0) for k in range(n)]
    h = _mul(_exp_neg(n), tm, n)
    return tuple(_log_series(h, n))


def pade_p(m: int) -> list[Fraction]:
    """p_m(x) coefficients of eq. (24): (2m-j)! m! / ((2m)! (m-j)! j!)."""
    return [Fraction(factorial(2 * m - j) * factorial(m),
                     factorial(2 * m) * factorial(m - j) * factorial(j)) for j in range(m + 1)]


@functools.lru_cache(maxsize=None)
def pade_rho(two_m: int) -> tuple[Fraction, ...]:
    """Exact coefficients c_0..c_{2m+NTERMS} of log(e^{-x} r_2m(x)),
    r_2m = p_m(x) / p_m(-x):  rho = -x + log p_m(x) - log p_m(-x)."""
    m = two_m // 2
    n = two_m + NTERMS + 1
    p = pade_p(m) + [Fraction(0)] * (n - m - 1)
    pm = [c * (-1) ** j for j, c in enumerate(p)]
    lp = _log_series(p, n)
    lm = _log_series(pm, n)
    rho = [a - b for a, b in zip(lp, lm)]
    rho[1] -= 1
    return tuple(rho)


def _solve(coeffs: tuple[Fraction, ...], first: int, u: float) -> float:
    """Root of f(theta)/theta = u with f = sum_{i=first}^{first+NTERMS-1} |c_i| theta^i."""
    getcontext().prec = 60
    ca = [Decimal(abs(c.numerator)) / Decimal(c.denominator) for c in coeffs[first:first + NTERMS]]
    target = Decimal(Fraction(u).numerator) / Decimal(Fraction(u).denominator)

    def g(t: Decimal) -> Decimal:  # f(t)/t, increasing in t > 0
        acc = Decimal(0)
        tp = t ** (first - 1)
        for c in ca:
            acc += c * tp
            tp *= t
        return acc

    lo, hi = Decimal(0), Decimal(1)
    while g(hi) < target:
        hi *= 2
    for _ in range(220):
        mid = (lo + hi) / 2
        if g(mid) < target:
            lo = mid
        else:
            hi = mid
    return float(lo)


@functools.lru_cache(maxsize=None)
def theta_taylor(m: int, u: float = 2.0 ** -53) -> float:
    """theta_m(u) for the Taylor polynomial T_m (Table 2)."""
    return _solve(taylor_rho(m), m + 1, u)


@functools.lru_cache(maxsize=None)
def theta_pade(two_m: int, u: float = 2.0 ** -53) -> float:
    """theta_2m(u) for the diagonal Pade approximant r_2m (Table 1)."""
    return _solve(pade_rho(two_m), two_m + 1, u)


def theta_array(scheme: str, u: float = 2.0 ** -53) -> list[float]:
    """Length-27 array indexed by degree, as the C oracle's selection reads it.
    scheme 'new' / 'ps' fill Taylor degrees; 'pade26' fills index 26 with the
    Pade threshold; 'pade' fills indices 10 and 26."""
    out = [0.0] * 27
    if scheme in ("new", "ps"):
        for d in (1, 2, 4, 6, 8, 9, 12, 16, 18):
            out[d] = theta_taylor(d, u)
    elif scheme == "pade26":
        out[26] = theta_pade(26, u)
    elif scheme == "pade":
        out[10] = theta_pade(10, u)
        out[26] = theta_pade(26, u)
    else:
        raise ValueError(scheme)
    return out
