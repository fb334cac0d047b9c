"""Pins of the float64 MLP oracle (no GPU): GELU special values and the
identity GELU(x) - GELU(-x) = x, backpropagated gradients against central
finite differences, Adam's first step, and a training run that fits."""
import math

import numpy as np
import pytest

import workloads
from oracle import mlp


def theta0(seed=5):
    return 0.3 * workloads.matrix(1, mlp.N_PARAMS, seed, "uniform")[0]


def test_gelu_values():
    x = np.array([-30.0, -1.0, 0.0, 1.0, 30.0])
    g = mlp.gelu(x)
    assert g[2] == 0.0 and g[4] == 30.0 and abs(g[0]) < 1e-100
    # Phi(1) = 0.841344746068543 (standard normal table)
    assert g[3] == pytest.approx(0.841344746068543, rel=1e-14)
    xs = np.linspace(-4, 4, 33)
    assert np.allclose(mlp.gelu(xs) - mlp.gelu(-xs), xs, rtol=0, atol=1e-15)


def test_gelu_grad_finite_difference():
    xs = np.linspace(-5, 5, 41)
    h = 1e-6
    fd = (mlp.gelu(xs + h) - mlp.gelu(xs - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(xs), fd, rtol=1e-8, atol=1e-9)


def test_gradient_central_differences():
    th = theta0()
    X = workloads.matrix(7, 10, 6, "uniform")
    y = workloads.matrix(1, 7, 7, "uniform")[0]
    loss, g = mlp.loss_and_grad(th, X, y)
    rng_idx = np.unique(np.concatenate([np.arange(0, mlp.N_PARAMS, 97),
                                        [mlp.N_PARAMS - 1, mlp.N_PARAMS - 2, 639, 640, 704]]))
    h = 1e-6
    for i in rng_idx:
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss_and_grad(tp, X, y)[0] - mlp.loss_and_grad(tm, X, y)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-9), i


def test_pack_unpack_layout():
    th = np.arange(mlp.N_PARAMS, dtype=np.float64)
    layers = mlp.unpack(th)
    assert layers[0][0].shape == (64, 10) and layers[0][0][1, 0] == 10.0
    assert layers[0][1][0] == 640.0
    assert layers[3][0].shape == (1, 64) and layers[3][1][0] == mlp.N_PARAMS - 1
    assert np.array_equal(mlp.pack(layers), th)
    assert mlp.N_PARAMS == 9089


def test_adam_first_step_is_signed_lr():
    th = theta0()
    g = workloads.matrix(1, mlp.N_PARAMS, 8, "uniform")[0]
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    t1, _, _ = mlp.adam_step(th, g, m, v, 1, lr=1e-3)
    # m^ = g, v^ = g^2: step = lr g / (|g| + eps)
    assert np.allclose(t1 - th, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)


def test_training_fits_a_smooth_target():
    X = workloads.matrix(128, 10, 9, "uniform")
    y = np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2]
    th = theta0(10) * 0.5
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    first = mlp.loss_and_grad(th, X, y)[0]
    for t in range(1, 301):
        loss, g = mlp.loss_and_grad(th, X, y)
        th, m, v = mlp.adam_step(th, g, m, v, t, lr=3e-3)
    assert loss < 0.05 * first
