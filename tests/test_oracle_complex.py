"""Pins of the complex oracle (oracle/complex_oracle.py) against what the
mathematics fixes: the complex 1-norm and the (m, s) it selects (eq. theta with
moduli), exp of diagonal and 2 x 2 triangular matrices in closed form, the
Taylor sum on 1 x 1 matrices (Section 3: T_m reproduces 1/k! up to degree m),
unitarity of exp(iH) for Hermitian H, exp(A) exp(-A) = I, agreement with the
real oracle on real input and with an independent Pade library. Each planted
mistake of the oracle must fail at least one pin."""
import cmath
import math

import numpy as np
import pytest

from oracle import complex_oracle as C
from oracle import oracle as O


def _rand_complex(n, seed, norm):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return A * (norm / C.norm1(A))


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# --- pins, each returning True when the oracle passes it -------------------------

def pin_norm_and_selection():
    A = np.array([[3 + 4j, 1.0], [0.0, 1j]])
    E, (m, s, _, nrm) = C.expm(A)
    return nrm == 5.0 and (m, s) == O.select(5.0, "new")


def pin_diagonal():
    z = np.array([0.3 + 2j, -4 + 0.5j, 12j, -20 - 7j, 1e-3 + 1e-3j, 9.0])
    E, _ = C.expm(np.diag(z))
    want = np.exp(z)
    return (np.max(np.abs(np.diag(E) - want) / np.abs(want)) < 1e-13
            and np.all(E[~np.eye(len(z), dtype=bool)] == 0))


def pin_triangular_2x2():
    ok = True
    for a, b, c in ((0.5 + 1j, 3 - 2j, -1 + 0.25j), (2j, 10.0, -3j), (-6 + 1j, 1j, 4 - 2j)):
        E, _ = C.expm(np.array([[a, b], [0, c]]))
        want = np.array([[cmath.exp(a), b * (cmath.exp(a) - cmath.exp(c)) / (a - c)], [0, cmath.exp(c)]])
        ok &= _rel(E, want) < 1e-13
    return bool(ok)


def pin_scalar_taylor():
    ok = True
    for m in (1, 2, 4, 8, 12, 18):
        for x in (0.01 + 0.02j, -0.3j, 0.7 - 0.6j):
            T = C.taylor_new(np.array([[x]]), m)[0, 0]
            want = sum(x ** k / math.factorial(k) for k in range(m + 1))
            ok &= abs(T - want) <= 1e-14 * abs(want)
    return bool(ok)


def pin_unitary():
    ok = True
    rng = np.random.default_rng(5)
    for n, norm in ((6, 0.5), (20, 5.0), (33, 50.0)):
        G = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        H = (G + G.conj().T) / 2
        A = 1j * H * (norm / C.norm1(1j * H))
        E, _ = C.expm(A)
        ok &= np.linalg.norm(E.conj().T @ E - np.eye(n)) < 1e-12 * n
    return bool(ok)


def pin_inverse():
    ok = True
    for n, norm, seed in ((10, 0.2, 1), (25, 8.0, 2)):
        A = _rand_complex(n, seed, norm)
        E, _ = C.expm(A)
        F, _ = C.expm(-A)
        ok &= np.linalg.norm(E @ F - np.eye(n)) < 1e-11 * n * max(1.0, np.exp(norm) ** 0.5)
    return bool(ok)


def pin_real_input():
    A = np.random.default_rng(9).standard_normal((30, 30))
    A *= 7.0 / np.max(np.sum(np.abs(A), axis=0))
    E, (m, s, _, _) = C.expm(A.astype(np.complex128))
    R, oi = O.expm(A, "new")
    return (m, s) == (oi.m, oi.s) and _rel(E.real, R) < 1e-14 and np.max(np.abs(E.imag)) == 0.0


def pin_scipy():
    sl = pytest.importorskip("scipy.linalg")
    ok = True
    for n, norm, seed in ((5, 0.01, 3), (17, 0.3, 4), (40, 3.0, 5), (24, 30.0, 6)):
        A = _rand_complex(n, seed, norm)
        E, _ = C.expm(A)
        ok &= _rel(E, sl.expm(A)) < 1e-12
    return bool(ok)


PINS = [pin_norm_and_selection, pin_diagonal, pin_triangular_2x2, pin_scalar_taylor, pin_unitary,
        pin_inverse, pin_real_input, pin_scipy]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    assert pin()


@pytest.mark.parametrize("code", [1, 2, 3, 4])
def test_planted_mistake_is_caught(code):
    C.set_mutation(code)
    try:
        failed = [p.__name__ for p in PINS if not p()]
    finally:
        C.set_mutation(0)
    assert failed, f"mutation {code} passed every pin"
