"""Reference for the learned per-bond rank predictor (FP64 numpy).

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this module.

The predictor is not part of the paper: it is the build's learned rank
choice for TT rounding. Network: 10 features -> 64 -> 64 -> 64 -> 1 with tanh
hidden activations and a sigmoid output, trained on the mean squared error
against the rank the adaptive SVD chose, divided by the rank cap.

Parameters are one flat vector in the order W1 (64 x 10, row-major), b1 (64),
W2 (64 x 64), b2 (64), W3 (64 x 64), b3 (64), w4 (64), b4 (1).
"""
from __future__ import annotations

import numpy as np

NIN, NH = 10, 64
SIZES = [(NH, NIN), (NH,), (NH, NH), (NH,), (NH, NH), (NH,), (NH,), (1,)]
NPARAM = int(sum(np.prod(s) for s in SIZES))


def unpack(theta: np.ndarray):
    out, off = [], 0
    for s in SIZES:
        n = int(np.prod(s))
        out.append(theta[off:off + n].reshape(s))
        off += n
    return out


def forward(theta: np.ndarray, X: np.ndarray):
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(np.asarray(theta, dtype=np.float64))
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    h3 = np.tanh(h2 @ W3.T + b3)
    z = h3 @ w4 + b4[0]
    y = 1.0 / (1.0 + np.exp(-z))
    return y, (h1, h2, h3, y)


def loss_and_grad(theta: np.ndarray, X: np.ndarray, t: np.ndarray):
    """Mean squared error and its gradient by backpropagation (chain rule, layer by layer)."""
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(np.asarray(theta, dtype=np.float64))
    B = X.shape[0]
    y, (h1, h2, h3, _) = forward(theta, X)
    loss = float(np.mean((y - t) ** 2))
    dy = 2.0 * (y - t) / B                  # d loss / d y
    dz = dy * y * (1.0 - y)                 # sigmoid'
    gw4 = h3.T @ dz
    gb4 = np.array([dz.sum()])
    d3 = np.outer(dz, w4) * (1.0 - h3 ** 2)
    gW3 = d3.T @ h2
    gb3 = d3.sum(0)
    d2 = (d3 @ W3) * (1.0 - h2 ** 2)
    gW2 = d2.T @ h1
    gb2 = d2.sum(0)
    d1 = (d2 @ W2) * (1.0 - h1 ** 2)
    gW1 = d1.T @ X
    gb1 = d1.sum(0)
    g = np.concatenate([a.reshape(-1) for a in (gW1, gb1, gW2, gb2, gW3, gb3, gw4, gb4)])
    return loss, g
