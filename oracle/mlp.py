"""Oracle of the strategy-selector network (test infrastructure only), float64 NumPy.

A 16 -> 64 -> 64 -> 3 multilayer perceptron with ReLU hidden layers and a
softmax output, trained on the mean cross-entropy with Adam (Kingma and Ba,
ICLR 2015). The selector stands in for the processing-time model of the
related work (Sec. 7). Parameters are one flat vector of 5443 values:
W1[16][64], b1[64], W2[64][64], b2[64], W3[64][3], b3[3] (W[in][out]).
"""
from __future__ import annotations

import numpy as np

SHAPES = [("W1", (16, 64)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (64, 3)), ("b3", (3,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(p: np.ndarray) -> dict:
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = p[o:o + k].reshape(shape)
        o += k
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def standardise(X, mean=None, std=None):
    X = np.asarray(X, dtype=np.float64)
    if mean is None:
        return X
    return (X - np.asarray(mean, dtype=np.float64)) / np.asarray(std, dtype=np.float64)


def forward(p, X, mean=None, std=None):
    """Class probabilities and the intermediate activations."""
    w = unpack(p)
    x = standardise(X, mean, std)
    a1 = x @ w["W1"] + w["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ w["W2"] + w["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ w["W3"] + w["b3"]
    zs = z - z.max(axis=1, keepdims=True)
    e = np.exp(zs)
    probs = e / e.sum(axis=1, keepdims=True)
    return probs, dict(x=x, a1=a1, h1=h1, a2=a2, h2=h2, z=z)


def loss(p, X, y, mean=None, std=None) -> float:
    probs, _ = forward(p, X, mean, std)
    y = np.asarray(y)
    return float(-np.mean(np.log(probs[np.arange(len(y)), y])))


def loss_and_grad(p, X, y, mean=None, std=None):
    """Mean cross-entropy and its gradient, by the chain rule layer by layer."""
    w = unpack(p)
    probs, c = forward(p, X, mean, std)
    y = np.asarray(y)
    B = len(y)
    onehot = np.zeros_like(probs)
    onehot[np.arange(B), y] = 1.0
    L = float(-np.mean(np.log(probs[np.arange(B), y])))
    dz = (probs - onehot) / B
    g = {"W3": c["h2"].T @ dz, "b3": dz.sum(axis=0)}
    dh2 = (dz @ w["W3"].T) * (c["a2"] > 0)
    g["W2"] = c["h1"].T @ dh2
    g["b2"] = dh2.sum(axis=0)
    dh1 = (dh2 @ w["W2"].T) * (c["a1"] > 0)
    g["W1"] = c["x"].T @ dh1
    g["b1"] = dh1.sum(axis=0)
    return L, pack(g)


def adam(p, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One bias-corrected Adam step at step t >= 1; returns (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
