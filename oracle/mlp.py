"""Plain numpy FP64 reference of the (m, s)-proposing MLP: forward pass,
softmax cross-entropy and its gradients, one Adam step.

TEST INFRASTRUCTURE (see the package docstring). The network: in -> hidden
(ReLU) -> hidden (ReLU) -> out logits. Parameters flattened in the order
W1[hidden][in], b1[hidden], W2[hidden][hidden], b2[hidden], W3[out][hidden],
b3[out] (row-major), the layout the CUDA kernels use too.
"""
from __future__ import annotations

import numpy as np


def shapes(n_in: int, hidden: int, n_out: int):
    return [(hidden, n_in), (hidden,), (hidden, hidden), (hidden,), (n_out, hidden), (n_out,)]


def unpack(theta, n_in, hidden, n_out):
    out, off = [], 0
    for shp in shapes(n_in, hidden, n_out):
        k = int(np.prod(shp))
        out.append(np.asarray(theta[off:off + k], dtype=np.float64).reshape(shp))
        off += k
    return out


def forward(theta, X, n_in, hidden, n_out):
    W1, b1, W2, b2, W3, b3 = unpack(theta, n_in, hidden, n_out)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    logits = h2 @ W3.T + b3
    return logits, (X, z1, h1, z2, h2)


def loss_and_grad(theta, X, y, n_in, hidden, n_out):
    """Mean softmax cross-entropy over the batch and its gradient (flattened)."""
    W1, b1, W2, b2, W3, b3 = unpack(theta, n_in, hidden, n_out)
    logits, (X, z1, h1, z2, h2) = forward(theta, X, n_in, hidden, n_out)
    B = X.shape[0]
    zmax = logits.max(axis=1, keepdims=True)
    ez = np.exp(logits - zmax)
    p = ez / ez.sum(axis=1, keepdims=True)
    loss = float(np.mean(-np.log(p[np.arange(B), y])))
    g = p.copy()
    g[np.arange(B), y] -= 1.0
    g /= B
    gW3 = g.T @ h2
    gb3 = g.sum(axis=0)
    d2 = (g @ W3) * (z2 > 0)
    gW2 = d2.T @ h1
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * (z1 > 0)
    gW1 = d1.T @ X
    gb1 = d1.sum(axis=0)
    grad = np.concatenate([a.ravel() for a in (gW1, gb1, gW2, gb2, gW3, gb3)])
    return loss, grad


def adam(theta, grad, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
