"""Pins for the oracle's backward-error thresholds (eq. theta, Tables 1 and 2).

The oracle's theta values are checked against numbers the paper prints and
against closed forms, never against themselves.
"""
import json
import math
import os
from fractions import Fraction
from math import factorial

import pytest

from oracle import theta as TH

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))
U53, U24 = 2.0 ** -53, 2.0 ** -24


def agrees_with_print(x: float, s: str) -> bool:
    """True when x agrees with the printed 3-digit value to within one unit of
    its last printed digit. The tables round some entries (theta_4 = 3.397e-4
    printed 3.40e-4) and truncate others (theta_12 = 0.29962 printed 2.99e-1),
    so both directions are allowed, but nothing further."""
    p = float(s)
    unit = 10.0 ** (math.floor(math.log10(abs(p))) - 2)
    return abs(x - p) < unit


@pytest.mark.parametrize("key,u", [("u_2^-53", U53), ("u_2^-24", U24)])
def test_taylor_theta_matches_table2(key, u):
    t = GOLD["table2_taylor_theta"]
    for m, val in zip(t["m"], t[key]):
        assert agrees_with_print(TH.theta_taylor(m, u), val), (m, TH.theta_taylor(m, u), val)


@pytest.mark.parametrize("key,u", [("u_2^-53", U53), ("u_2^-24", U24)])
def test_pade_theta_matches_table1(key, u):
    t = GOLD["table1_pade_theta"]
    for two_m, val in zip(t["two_m"], t[key]):
        assert agrees_with_print(TH.theta_pade(two_m, u), val), (two_m, TH.theta_pade(two_m, u), val)


@pytest.mark.parametrize("u", [U53, U24, 2.0 ** -40])
def test_closed_forms_low_degree(u):
    # T1: e^{-x}(1+x) = 1 - x^2/2 + ..., so f(t)/t = t/2 (1 + O(t)) and theta_1 = 2u (1 + O(u)).
    assert TH.theta_taylor(1, u) == pytest.approx(2 * u, rel=10 * u)
    # T2: e^{-x}(1+x+x^2/2) = 1 - x^3/6 + ..., so theta_2 = sqrt(6u) (1 + O(sqrt(u))).
    assert TH.theta_taylor(2, u) == pytest.approx(math.sqrt(6 * u), rel=10 * math.sqrt(u))
    # and the first-order correction has the sign the next term forces (f grows faster).
    assert TH.theta_taylor(2, u) < math.sqrt(6 * u)


def test_rho_vanishes_below_order():
    # log(e^{-x} T_m) = O(x^{m+1}); log(e^{-x} r_2m) = O(x^{2m+1}).
    for m in (1, 2, 4, 8, 12, 18):
        c = TH.taylor_rho(m)
        assert all(ci == 0 for ci in c[: m + 1])
        assert c[m + 1] == Fraction(-1, factorial(m + 1))  # leading term -x^{m+1}/(m+1)!
    for two_m in (2, 6, 10, 26):
        c = TH.pade_rho(two_m)
        assert all(ci == 0 for ci in c[: two_m + 1])
        assert c[two_m + 1] != 0


def test_pade_coefficients_are_pade():
    # p_m(x) - e^x p_m(-x) = O(x^{2m+1}) exactly (eq. 24), for the formula as printed.
    for m in (3, 5, 13):
        p = TH.pade_p(m)
        n = 2 * m + 2
        e = [Fraction(1, factorial(k)) for k in range(n)]
        pm = [c * (-1) ** j for j, c in enumerate(p)]
        prod = [sum(e[i] * pm[k - i] for i in range(k + 1) if k - i < len(pm)) for k in range(n)]
        diff = [(p[k] if k < len(p) else 0) - prod[k] for k in range(n)]
        assert all(d == 0 for d in diff[: 2 * m + 1])
        assert diff[2 * m + 1] != 0


def test_theta_monotone_in_u_and_degree():
    for m in (2, 4, 8, 12, 18):
        assert TH.theta_taylor(m, U53) < TH.theta_taylor(m, U24)
    seq = [TH.theta_taylor(m) for m in (1, 2, 4, 8, 12, 18)]
    assert seq == sorted(seq)
