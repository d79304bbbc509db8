"""Pins of the FP64 reference MLP (oracle/mlp.py): central finite differences
and a closed form."""
import numpy as np

from oracle import mlp


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    nin, nh, nout, B = 4, 7, 5, 6
    theta = rng.standard_normal(mlp.size(nin, nh, nout)) * 0.5
    X = rng.uniform(-1, 1, (B, nin))
    T = rng.standard_normal((B, nout))
    L, g = mlp.loss_grad(theta, X, T, nin, nh, nout)
    assert abs(L - mlp.loss(theta, X, T, nin, nh, nout)) < 1e-15
    h = 1e-6
    for k in rng.choice(theta.size, 40, replace=False):
        e = np.zeros_like(theta)
        e[k] = h
        fd = (mlp.loss(theta + e, X, T, nin, nh, nout) - mlp.loss(theta - e, X, T, nin, nh, nout)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(fd))


def test_zero_weights_closed_form():
    # W = 0: Y = b3 for every sample, loss = mean((b3 - T)^2), db3 = 2 mean over
    # samples of (b3 - T) / nout, every weight gradient vanishes except dW3 = 0
    nin, nh, nout, B = 3, 4, 2, 5
    theta = np.zeros(mlp.size(nin, nh, nout))
    b3 = np.array([0.5, -1.0])
    theta[-nout:] = b3
    rng = np.random.default_rng(1)
    T = rng.standard_normal((B, nout))
    L, g = mlp.loss_grad(theta, rng.standard_normal((B, nin)), T, nin, nh, nout)
    assert np.isclose(L, np.mean((b3 - T) ** 2))
    assert np.allclose(g[-nout:], 2 * (b3 - T).sum(axis=0) / (B * nout))
    assert np.allclose(g[:-nout], 0.0)
