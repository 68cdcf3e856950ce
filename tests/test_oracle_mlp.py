"""Pins for the selector-network oracle: finite differences and closed forms."""
import math

import numpy as np

from oracle import mlp


def _params(seed, scale=0.3):
    return np.random.default_rng(seed).standard_normal(mlp.N_PARAMS) * scale


def test_param_count():
    assert mlp.N_PARAMS == 16 * 64 + 64 + 64 * 64 + 64 + 64 * 3 + 3 == 5443


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    p = _params(2)
    X = rng.standard_normal((7, 16))
    y = rng.integers(0, 3, 7)
    _, g = mlp.loss_and_grad(p, X, y)
    h = 1e-6
    idx = np.concatenate([np.arange(0, 1024, 37), np.arange(1024, 1088, 5), np.arange(1088, 5184, 211),
                          np.arange(5184, 5248, 7), np.arange(5248, 5443)])
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (mlp.loss(p + e, X, y) - mlp.loss(p - e, X, y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_standardisation_enters_the_gradient():
    rng = np.random.default_rng(3)
    p = _params(4)
    X = rng.standard_normal((5, 16)) * 10 + 3
    mean, std = X.mean(axis=0), X.std(axis=0) + 0.5
    y = rng.integers(0, 3, 5)
    L1, g1 = mlp.loss_and_grad(p, X, y, mean, std)
    L2, g2 = mlp.loss_and_grad(p, (X - mean) / std, y)
    assert abs(L1 - L2) < 1e-12 and np.allclose(g1, g2, rtol=1e-12, atol=1e-14)


def test_zero_network_is_uniform():
    p = np.zeros(mlp.N_PARAMS)
    X = np.random.default_rng(5).standard_normal((10, 16))
    y = np.array([0, 1, 2, 0, 0, 1, 2, 2, 2, 1])
    probs, _ = mlp.forward(p, X)
    assert np.allclose(probs, 1 / 3)
    L, g = mlp.loss_and_grad(p, X, y)
    assert abs(L - math.log(3)) < 1e-15
    w = mlp.unpack(g)
    onehot_mean = np.bincount(y, minlength=3) / len(y)
    assert np.allclose(w["b3"], 1 / 3 - onehot_mean)
    assert np.all(w["W1"] == 0) and np.all(w["W2"] == 0) and np.all(w["W3"] == 0)


def test_adam_first_step_is_signed_lr():
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    p, m, v = mlp.adam(np.zeros(4), g, np.zeros(4), np.zeros(4), t=1, lr=0.01)
    assert np.allclose(p[:3], -0.01 * np.sign(g[:3]), rtol=1e-4) and p[3] == 0
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_training_steps_reduce_the_loss():
    rng = np.random.default_rng(6)
    X = rng.standard_normal((256, 16))
    y = (X[:, 0] > 0).astype(int) + (X[:, 1] > 1).astype(int)
    p = _params(7, 0.1)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    L0 = mlp.loss(p, X, y)
    for t in range(1, 201):
        _, g = mlp.loss_and_grad(p, X, y)
        p, m, v = mlp.adam(p, g, m, v, t, lr=1e-2)
    assert mlp.loss(p, X, y) < 0.3 * L0


def test_forward_on_hand_computed_network():
    """A network worked out by hand, with one negative pre-activation in each
    hidden layer, so that a dropped or misplaced ReLU changes the output.

    x = (1, -2, 0, ..., 0)
    layer 1: a1[0] = x0 + 0.5 = 1.5, a1[1] = x1 = -2 -> h1 = (1.5, 0, 0, ...)
    layer 2: a2[0] = 2 h1[0] + 1 h1[1] = 3, a2[1] = -h1[0] = -1.5 -> h2 = (3, 0, ...)
    layer 3: z = (h2[0], 5 h2[1] + ln 2, -h2[0]) = (3, ln 2, -3)
    softmax: (e^3, 2, e^-3) / (e^3 + 2 + e^-3)
    Without the first ReLU, a2[0] would be 3 - 2 = 1; without the second, z[1]
    would be ln 2 - 7.5.
    """
    w = {name: np.zeros(shape) for name, shape in mlp.SHAPES}
    w["W1"][0, 0] = 1.0
    w["W1"][1, 1] = 1.0
    w["b1"][0] = 0.5
    w["W2"][0, 0] = 2.0
    w["W2"][1, 0] = 1.0
    w["W2"][0, 1] = -1.0
    w["W3"][0, 0] = 1.0
    w["W3"][1, 1] = 5.0
    w["W3"][0, 2] = -1.0
    w["b3"][1] = math.log(2.0)
    p = mlp.pack(w)
    X = np.zeros((1, 16))
    X[0, 0], X[0, 1] = 1.0, -2.0
    probs, c = mlp.forward(p, X)
    den = math.exp(3) + 2.0 + math.exp(-3)
    expect = np.array([math.exp(3) / den, 2.0 / den, math.exp(-3) / den])
    assert np.allclose(probs[0], expect, rtol=1e-14, atol=0)
    assert c["h1"][0, 1] == 0.0 and c["h2"][0, 1] == 0.0
    # the loss of class 1 is -ln(2 / den)
    assert abs(mlp.loss(p, X, np.array([1])) - (math.log(den) - math.log(2.0))) < 1e-14
    # standardisation is applied before layer 1: x' = (x - mean) / std
    mean = np.full(16, 1.0)
    std = np.full(16, 2.0)
    probs2, _ = mlp.forward(p, X * 2.0 + 1.0, mean, std)
    assert np.allclose(probs2, probs, rtol=1e-14, atol=0)
