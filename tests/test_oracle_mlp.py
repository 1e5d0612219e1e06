"""Pins for the reference rank-predictor MLP: backpropagation against central finite differences."""
import numpy as np

from oracle import mlp
from paper_2509_11890_gb300 import inputs


def test_backprop_matches_central_differences():
    g = inputs.rng(3, 40)
    theta = g.normal(0, 0.3, mlp.NPARAM)
    X = g.uniform(-1, 1, (17, mlp.NIN))
    t = g.uniform(0, 1, 17)
    loss, grad = mlp.loss_and_grad(theta, X, t)
    idx = g.choice(mlp.NPARAM, 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.NPARAM)
        e[i] = h
        fd = (mlp.loss_and_grad(theta + e, X, t)[0] - mlp.loss_and_grad(theta - e, X, t)[0]) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-7 * (1 + abs(fd)), (i, fd, grad[i])
    # every parameter block is reached (the last layer's bias, the first layer's weights)
    assert np.any(grad[: 64 * 9] != 0) and grad[-1] != 0


def test_forward_limits():
    theta = np.zeros(mlp.NPARAM)
    y, _ = mlp.forward(theta, np.ones((3, mlp.NIN)))
    np.testing.assert_allclose(y, 0.5)   # sigmoid(0)
