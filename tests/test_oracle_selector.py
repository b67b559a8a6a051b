"""Pins for the oracle's certified selection (power norms, the alpha_2 bound)
and for its numpy MLP (finite differences)."""
import numpy as np
import pytest

from oracle import mlp as M
from oracle import oracle as O
from paper_1710_10989_gb300 import workloads as W


@pytest.mark.parametrize("a,c", [(0.5, 40.0), (-1.25, 3.0), (0.0, 7.0)])
def test_power_norms_of_jordan_block(a, c):
    # [[a, c], [0, a]]^k = [[a^k, k a^(k-1) c], [0, a^k]]: the second column dominates
    J = np.array([[a, c], [0.0, a]])
    want = [abs(a) ** k + k * abs(a) ** (k - 1) * abs(c) if k > 1 or a != 0 else abs(c) for k in (1, 2, 3, 4)]
    want[0] = abs(a) + abs(c)
    assert np.allclose(O.power_norms(J), want, rtol=1e-15, atol=0)


def test_certified_selection_hand_case():
    # a = 0.5, c = 40: ||A|| = 40.5 -> paper's bound needs (18, 6) (40.5/64 <= 1.09 < 40.5/32).
    # ||A^2|| = 40.25, ||A^3|| = 30.125: alpha_2 = max(6.344, 3.112) = 6.344 -> (18, 3)
    # (6.344/8 = 0.79 <= 1.09 < 6.344/4); (12, 5) would cost 9.
    J = np.array([[0.5, 40.0], [0.0, 0.5]])
    nrm = O.power_norms(J)
    assert O.select(nrm[0]) == (18, 6)
    assert O.select_certified(nrm) == (18, 3)


def test_nilpotent_certifies_degree_one():
    J = np.array([[0.0, 5.0], [0.0, 0.0]])
    assert O.select_certified(O.power_norms(J)) == (1, 0)
    E, _ = O.expm(J, m=1, s=0)
    assert np.array_equal(E, np.array([[1.0, 5.0], [0.0, 1.0]]))


def test_certified_never_costs_more_and_stays_accurate():
    sl = pytest.importorskip("scipy.linalg")
    pi = {1: 0, 2: 1, 4: 2, 8: 3, 12: 4, 18: 5}
    for i in range(12):
        n = 24 + 8 * i
        A = (W.diagonalisable(n, 500 + i, 30.0) if i % 2 else W.nonnormal_upper(n, 500 + i, 30.0))
        nrm = O.power_norms(A)
        m0, s0 = O.select(nrm[0])
        m1, s1 = O.select_certified(nrm)
        assert pi[m1] + s1 <= pi[m0] + s0
        E, _ = O.expm(A, m=m1, s=s1)
        R = sl.expm(A)
        assert np.linalg.norm(E - R) / np.linalg.norm(R) < 1e-11


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    n_in, hid, n_out, B = 5, 7, 4, 6
    nparam = sum(int(np.prod(s)) for s in M.shapes(n_in, hid, n_out))
    theta = rng.standard_normal(nparam) * 0.5
    X = rng.standard_normal((B, n_in))
    y = rng.integers(0, n_out, size=B)
    _, g = M.loss_and_grad(theta, X, y, n_in, hid, n_out)
    eps = 1e-6
    for k in rng.choice(nparam, 25, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += eps
        tm[k] -= eps
        fd = (M.loss_and_grad(tp, X, y, n_in, hid, n_out)[0] - M.loss_and_grad(tm, X, y, n_in, hid, n_out)[0]) / (2 * eps)
        assert fd == pytest.approx(g[k], abs=1e-7, rel=1e-5)


def test_mlp_adam_learns_a_separable_rule():
    rng = np.random.default_rng(4)
    n_in, hid, n_out = 2, 16, 2
    nparam = sum(int(np.prod(s)) for s in M.shapes(n_in, hid, n_out))
    theta = rng.standard_normal(nparam) * 0.3
    X = rng.standard_normal((256, n_in))
    y = (X[:, 0] + X[:, 1] > 0).astype(int)
    m = np.zeros(nparam)
    v = np.zeros(nparam)
    l0 = M.loss_and_grad(theta, X, y, n_in, hid, n_out)[0]
    for step in range(1, 301):
        _, g = M.loss_and_grad(theta, X, y, n_in, hid, n_out)
        theta, m, v = M.adam(theta, g, m, v, step, lr=1e-2)
    l1 = M.loss_and_grad(theta, X, y, n_in, hid, n_out)[0]
    acc = (M.forward(theta, X, n_in, hid, n_out)[0].argmax(1) == y).mean()
    assert l1 < 0.3 * l0 and acc > 0.95
