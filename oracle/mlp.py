"""CPU oracle of the surrogate network (TEST INFRASTRUCTURE ONLY).

The surrogate maps a bin's first-pass features to its clipped mean and
log-deviation: x (20) -> 64 -> GELU -> 64 -> GELU -> 2, mean-squared-error
loss. This is the plain FP64 statement the GPU kernels are checked against:
forward, loss and the analytic gradient by backpropagation, each written out
layer by layer. GELU is the exact form x * Phi(x) = x (1 + erf(x / sqrt 2)) / 2.
The paper has no surrogate; the network is this project's addition and its
only reference is this file (pinned by central finite differences in
tests/test_oracle_mlp.py).

Parameter layout (flat, FP64 here, float on the GPU):
  W1 [64][20], b1 [64], W2 [64][64], b2 [64], W3 [2][64], b3 [2]
"""
from __future__ import annotations

import math

import numpy as np

N_IN, N_H, N_OUT = 20, 64, 2
SHAPES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)), ("W3", (N_OUT, N_H)),
          ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(theta[o:o + n], np.float64).reshape(shp)
        o += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], np.float64).ravel() for name, _ in SHAPES])


_erf = np.vectorize(math.erf)


def gelu(a):
    return 0.5 * a * (1.0 + _erf(a / math.sqrt(2.0)))


def gelu_grad(a):
    # d/da [a Phi(a)] = Phi(a) + a phi(a)
    return 0.5 * (1.0 + _erf(a / math.sqrt(2.0))) + a * np.exp(-0.5 * a * a) / math.sqrt(2.0 * math.pi)


def forward(theta, x):
    """x: [n][20] -> outputs [n][2] and the intermediate activations."""
    p = unpack(theta)
    x = np.asarray(x, np.float64)
    a1 = x @ p["W1"].T + p["b1"]
    h1 = gelu(a1)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(a2)
    y = h2 @ p["W3"].T + p["b3"]
    return y, (x, a1, h1, a2, h2)


def loss(theta, x, t):
    """Mean over samples of the summed squared error of the two outputs."""
    y, _ = forward(theta, x)
    return float(np.mean(np.sum((y - np.asarray(t, np.float64)) ** 2, axis=1)))


def grad(theta, x, t):
    """Analytic gradient of loss() by backpropagation."""
    p = unpack(theta)
    y, (x, a1, h1, a2, h2) = forward(theta, x)
    n = x.shape[0]
    d3 = 2.0 * (y - np.asarray(t, np.float64)) / n          # dL/dy
    g = {"W3": d3.T @ h2, "b3": d3.sum(0)}
    d2 = (d3 @ p["W3"]) * gelu_grad(a2)                      # dL/da2
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(0)
    d1 = (d2 @ p["W2"]) * gelu_grad(a1)                      # dL/da1
    g["W1"] = d1.T @ x
    g["b1"] = d1.sum(0)
    return pack(g)


def init(seed=0):
    """He-style uniform initialisation (the same recipe as the GPU's)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in SHAPES:
        if name.startswith("W"):
            lim = math.sqrt(6.0 / shp[1])
            p[name] = rng.uniform(-lim, lim, shp)
        else:
            p[name] = np.zeros(shp)
    return pack(p)
