"""Pins of the surrogate network's CPU reference (oracle/mlp.py): the analytic
backpropagation gradient against central finite differences in FP64, GELU
against its closed-form values, and the loss at a point where it is known."""
import math

import numpy as np
import pytest

from oracle import mlp


def test_gelu_closed_form():
    a = np.array([0.0, 1.0, -1.0, 3.0])
    want = a * 0.5 * (1 + np.array([math.erf(v / math.sqrt(2)) for v in a]))
    assert np.allclose(mlp.gelu(a), want, rtol=1e-15)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    # Phi(1) = 0.841344746..., so gelu(1) = 0.841344746...
    assert mlp.gelu(np.array([1.0]))[0] == pytest.approx(0.8413447460685429, rel=1e-13)
    h = 1e-6
    for v in (-2.0, -0.3, 0.0, 0.7, 2.5):
        fd = (mlp.gelu(np.array([v + h]))[0] - mlp.gelu(np.array([v - h]))[0]) / (2 * h)
        assert mlp.gelu_grad(np.array([v]))[0] == pytest.approx(fd, rel=1e-8, abs=1e-10)


def test_backprop_matches_central_differences():
    rng = np.random.default_rng(3)
    theta = mlp.init(1) * 0.7
    x = rng.normal(0, 1, (17, mlp.N_IN))
    t = rng.normal(0, 1, (17, mlp.N_OUT))
    g = mlp.grad(theta, x, t)
    idx = rng.choice(mlp.N_PARAMS, 300, replace=False)
    h = 1e-5
    for i in idx:
        e = np.zeros(mlp.N_PARAMS)
        e[i] = h
        fd = (mlp.loss(theta + e, x, t) - mlp.loss(theta - e, x, t)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_loss_zero_at_exact_targets_and_bias_only_net():
    theta = np.zeros(mlp.N_PARAMS)
    p = mlp.unpack(theta)
    p["b3"][:] = [0.25, -1.5]
    theta = mlp.pack(p)
    x = np.random.default_rng(0).normal(size=(5, mlp.N_IN))
    y, _ = mlp.forward(theta, x)
    assert np.all(y == np.array([0.25, -1.5]))   # zero weights: output is the bias
    assert mlp.loss(theta, x, np.tile([0.25, -1.5], (5, 1))) == 0.0
    # moving the target by 1 in one output costs exactly 1 per sample
    assert mlp.loss(theta, x, np.tile([1.25, -1.5], (5, 1))) == pytest.approx(1.0, rel=1e-15)
