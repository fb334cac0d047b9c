"""Float64 oracle of the learned cost model: a 10 -> 64 -> 64 -> 64 -> 1 MLP
with exact (erf) GELU, mean-squared error on log time, and Adam.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper chooses the group count by sampling a few runs (Section V-A-1,
Section VI); the learned model that proposes (P, Q, G, b, B) instead is a
requirement of the method as specified here, not of the paper.  Parameter vector layout (also the
layout of the device kernels' weight buffer):
  W1[64][10], b1[64], W2[64][64], b2[64], W3[64][64], b3[64], W4[1][64], b4[1]
(row-major, W[out][in]); y = W x + b per layer.
"""
from __future__ import annotations

import math

import numpy as np

LAYERS = ((10, 64), (64, 64), (64, 64), (64, 1))
N_PARAMS = sum(i * o + o for i, o in LAYERS)


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.size == N_PARAMS
    out, off = [], 0
    for fi, fo in LAYERS:
        W = theta[off:off + fi * fo].reshape(fo, fi)
        off += fi * fo
        b = theta[off:off + fo]
        off += fo
        out.append((W, b))
    return out


def pack(layers):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers])


_erf = np.vectorize(math.erf, otypes=[np.float64])


def gelu(x):
    """GELU(x) = x Phi(x) = x (1 + erf(x / sqrt 2)) / 2 (Hendrycks and Gimpel)."""
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    """d GELU / dx = Phi(x) + x phi(x)."""
    return 0.5 * (1.0 + _erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def forward(theta, X):
    """Returns predictions (batch,) and the cache of pre-activations."""
    X = np.asarray(X, dtype=np.float64)
    h, cache = X, []
    layers = unpack(theta)
    for li, (W, b) in enumerate(layers):
        z = h @ W.T + b
        cache.append((h, z))
        h = gelu(z) if li < len(layers) - 1 else z
    return h[:, 0], cache


def loss_and_grad(theta, X, y):
    """MSE loss mean_i (f(x_i) - y_i)^2 and its gradient by backpropagation."""
    pred, cache = forward(theta, X)
    y = np.asarray(y, dtype=np.float64)
    B = pred.size
    loss = float(np.mean((pred - y) ** 2))
    g = (2.0 / B) * (pred - y)[:, None]           # dL / d(output)
    layers = unpack(theta)
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        h, z = cache[li]
        dz = g if li == len(layers) - 1 else g * gelu_grad(z)
        grads[li] = (dz.T @ h, dz.sum(axis=0))
        g = dz @ W
    return loss, pack(grads)


def adam_step(theta, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba), step number t >= 1."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    theta = theta - lr * mh / (np.sqrt(vh) + eps)
    return theta, m, v
