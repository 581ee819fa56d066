"""Pins of the MLP oracle: backpropagation against central finite differences, and closed forms."""

import numpy as np

from oracle.mlp import N_PARAMS, forward, init_params, loss_and_grad, pack, unpack


def test_parameter_count():
    assert N_PARAMS == 64 * 8 + 64 + 64 * 64 + 64 + 64 + 1 == 4801


def test_gradient_against_central_differences():
    rng = np.random.default_rng(0)
    theta = init_params(3) + rng.normal(scale=0.05, size=N_PARAMS)
    X = rng.normal(size=(16, 8))
    t = rng.normal(size=16)
    L, g = loss_and_grad(theta, X, t)
    idx = rng.choice(N_PARAMS, size=60, replace=False)
    idx = np.concatenate([idx, [N_PARAMS - 1, 0, 512, 576, 4672]])  # b3, W1[0,0], b1[0], W2[0,0], W3[0]
    h = 1e-6
    for i in idx:
        e = np.zeros(N_PARAMS)
        e[i] = h
        fd = (loss_and_grad(theta + e, X, t)[0] - loss_and_grad(theta - e, X, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd)), (i, fd, g[i])


def test_closed_forms():
    theta = np.zeros(N_PARAMS)
    parts = unpack(theta)
    parts["b3"] = np.array([0.25])
    X = np.random.default_rng(1).normal(size=(5, 8))
    y, _ = forward(pack(parts), X)
    assert np.allclose(y, 0.25)           # zero weights: the output bias alone
    L, g = loss_and_grad(pack(parts), X, np.zeros(5))
    assert abs(L - 0.0625) < 1e-15
    gp = unpack(g)
    assert abs(gp["b3"][0] - 0.5) < 1e-15  # d/db3 mean((b3 - 0)^2) = 2 b3
    assert np.all(gp["W1"] == 0) and np.all(gp["W2"] == 0) and np.all(gp["W3"] == 0)
    # a single active path: y = w3 tanh(w2 tanh(w1 x0))
    parts = unpack(np.zeros(N_PARAMS))
    parts["W1"][0, 0], parts["W2"][0, 0], parts["W3"][0] = 0.7, -1.3, 2.0
    x = np.zeros((1, 8))
    x[0, 0] = 0.4
    y, _ = forward(pack(parts), x)
    assert abs(y[0] - 2.0 * np.tanh(-1.3 * np.tanh(0.7 * 0.4))) < 1e-15
