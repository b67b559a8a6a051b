"""GPU parity of the (m, s)-proposing network's kernels against the numpy
oracle (forward, cross-entropy gradient, Adam), and of the learned/certified
selection path against the oracle's certified selection."""
import numpy as np
import pytest

from oracle import mlp as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_10989_gb300 import api as A
    return A


def _setup(api, n_in=5, hid=64, n_out=60, B=96, seed=0):
    import torch
    rng = np.random.default_rng(seed)
    net = api.MLP(n_in, hid, n_out, seed=seed)
    theta = net.params.cpu().numpy().astype(np.float64)
    theta += rng.standard_normal(theta.size) * 0.05          # non-zero biases too
    net.params.copy_(torch.from_numpy(theta.astype(np.float32)))
    theta = net.params.cpu().numpy().astype(np.float64)
    X = rng.standard_normal((B, n_in)).astype(np.float32)
    y = rng.integers(0, n_out, size=B)
    return net, theta, X, y


def test_forward_matches_oracle(api):
    import torch
    net, theta, X, _ = _setup(api)
    got = net.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    want, _ = M.forward(theta, X.astype(np.float64), 5, 64, 60)
    assert np.abs(got - want).max() < 1e-5 * max(1.0, np.abs(want).max())


def test_gradient_matches_oracle(api):
    import torch
    net, theta, X, y = _setup(api, seed=1)
    g, loss = net.grad(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda())
    wl, wg = M.loss_and_grad(theta, X.astype(np.float64), y, 5, 64, 60)
    g = g.cpu().numpy()
    assert float(loss.mean()) == pytest.approx(wl, rel=1e-5)
    assert np.linalg.norm(g - wg) / np.linalg.norm(wg) < 1e-5
    assert np.abs(g - wg).max() < 1e-4 * np.abs(wg).max()


def test_adam_step_matches_oracle(api):
    import torch
    net, theta, X, y = _setup(api, seed=2)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    for step in (1, 2, 3):
        _, wg = M.loss_and_grad(theta, X.astype(np.float64), y, 5, 64, 60)
        theta, m, v = M.adam(theta, wg, m, v, step, lr=1e-3)
        net.train_step(Xd, yd, lr=1e-3)
    got = net.params.cpu().numpy()
    assert np.abs(got - theta).max() < 1e-5


def test_training_learns(api):
    import torch
    rng = np.random.default_rng(5)
    X = rng.standard_normal((2048, 5)).astype(np.float32)
    y = (np.clip(np.floor((X[:, 0] + 2.5) * 2), 0, 9)).astype(np.int64)   # 10 ordered classes
    net = api.MLP(5, 64, 10, seed=3)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    l0 = float(net.grad(Xd, yd)[1].mean())
    for _ in range(400):
        net.train_step(Xd, yd, lr=3e-3)
    l1 = float(net.grad(Xd, yd)[1].mean())
    acc = float((net.forward(Xd).argmax(1) == yd).float().mean())
    assert l1 < 0.25 * l0 and acc > 0.9
