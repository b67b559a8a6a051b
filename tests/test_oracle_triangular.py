"""Pins of the oracle's upper-triangular path (exact diagonal and first
superdiagonal of exp(2^-q A) put in before every squaring; Section 5, concluding
remarks): closed forms of the 2 x 2 exponential, the diagonal e^{a_ii}, zero
lower triangle, 50-digit references, and agreement with the plain method."""
import math

import numpy as np
import pytest

from oracle import oracle as O


def exp2x2_exact(a, b, c, mp):
    """exp([[a, b], [0, c]]) to 50 digits: [[e^a, b (e^c - e^a)/(c - a)], [0, e^c]]."""
    mp.mp.dps = 50
    a, b, c = mp.mpf(a), mp.mpf(b), mp.mpf(c)
    ea, ec = mp.e ** a, mp.e ** c
    sup = b * ea if a == c else b * (ec - ea) / (c - a)
    return float(ea), float(sup), float(ec)


@pytest.mark.parametrize("a,b,c", [(1.0, 1e4, 1.0 + 1e-7), (-3.0, 250.0, 2.5), (0.5, -40.0, 0.5),
                                   (-20.0, 1e3, -19.999)])
def test_two_by_two_closed_form(a, b, c):
    mp = pytest.importorskip("mpmath")
    E, info = O.expm_upper(np.array([[a, b], [0.0, c]]))
    ea, sup, ec = exp2x2_exact(a, b, c, mp)
    assert E[1, 0] == 0.0
    assert abs(E[0, 0] - ea) <= 4e-16 * abs(ea)
    assert abs(E[1, 1] - ec) <= 4e-16 * abs(ec)
    # exp((l1 + l2)/2): the rounded argument carries an absolute error ~|l|u into the result
    assert abs(E[0, 1] - sup) <= 4e-16 * (3 + (abs(a) + abs(c)) / 2) * abs(sup)
    assert info.s > 0 or abs(b) < 1  # these cases do scale: the replacement runs after squarings


def test_diagonal_is_exp_of_diagonal_and_lower_is_zero():
    rng = np.random.default_rng(3)
    A = np.triu(rng.standard_normal((12, 12))) * 4.0
    E, info = O.expm_upper(A)
    assert info.s > 0
    assert all(E[i, i] == math.exp(A[i, i]) for i in range(12))
    assert not np.tril(E, -1).any()


@pytest.mark.parametrize("seed", [1, 2])
def test_upper_against_mpmath(seed):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    rng = np.random.default_rng(seed)
    n = 10
    A = np.triu(rng.standard_normal((n, n)) * 10.0, 1) + np.diag(rng.standard_normal(n))
    E, info = O.expm_upper(A)
    ref = mp.expm(mp.matrix(A.tolist()))
    R = np.array([[float(ref[i, j]) for j in range(n)] for i in range(n)])
    assert np.linalg.norm(E - R) / np.linalg.norm(R) < 1e-13


def test_agrees_with_plain_method_and_rejects_non_triangular():
    rng = np.random.default_rng(4)
    A = np.triu(rng.standard_normal((20, 20)))
    E, i1 = O.expm_upper(A)
    F, i2 = O.expm(A)
    assert (i1.m, i1.s, i1.products) == (i2.m, i2.s, i2.products)
    assert np.linalg.norm(E - F) / np.linalg.norm(F) < 1e-13
    A[5, 2] = 1e-300
    with pytest.raises(ValueError):
        O.expm_upper(A)


def test_replacement_beats_plain_on_near_equal_eigenvalues():
    """The case the paper's remark is about: a large superdiagonal over nearly
    equal diagonal entries; the plain squarings lose digits the closed form keeps."""
    mp = pytest.importorskip("mpmath")
    a, b, c = 1.0, 1e6, 1.0 + 1e-9
    A = np.array([[a, b], [0.0, c]])
    E, _ = O.expm_upper(A)
    F, _ = O.expm(A)
    _, sup, _ = exp2x2_exact(a, b, c, mp)
    assert abs(E[0, 1] - sup) <= abs(F[0, 1] - sup)
