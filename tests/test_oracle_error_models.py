"""Pins of the Poisson and hybrid error models (Section 2.2, Eqs. 3-4;
Section 2.4.1): the two-pixel example the paper prints (with the Poisson
deviation both pixels lie ~10 sigma away and sigma-clipping empties the bin;
the hybrid model keeps both and reports the Poisson deviation of 10), the
closed form sqrt(mean + dark) for unit coefficients, the c^2-weighted form
with split pixels, and a brute force of the Poisson clip loop."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from test_oracle_moments import GOLD, one_bin


def test_two_pixel_example_under_each_model():
    g = json.load(open(os.path.join(GOLD, "paper_two_pixel.json")))
    W, v = one_bin(g["values"])
    # Poisson: both pixels ~10 sigma from the mean, k = 3 discards them: an empty bin
    r = oracle.integrate_clip(W, v, n_iter=5, k=3.0, model=oracle.ERROR_POISSON)
    assert r["count"][0] == 0 and r["mean"][0] == 0.0
    # hybrid: the azimuthal deviation keeps both, the Poisson one is reported
    r = oracle.integrate_clip(W, v, n_iter=5, k=3.0, model=oracle.ERROR_HYBRID)
    assert r["count"][0] == 2 and r["mean"][0] == 100.0
    assert r["sigma"][0] == pytest.approx(10.0, rel=1e-15)
    assert abs(r["sigma"][0] - math.sqrt(g["mean"])) < 1e-12


@pytest.mark.parametrize("dark", [0.0, 2.5])
def test_unit_coefficients_closed_form(dark):
    rng = np.random.default_rng(1)
    v = rng.poisson(7.0, 500).astype(np.float32)
    W, v = one_bin(v)
    r = oracle.integrate_clip(W, v, n_iter=0, model=oracle.ERROR_POISSON, dark=dark)
    assert r["sigma"][0] == pytest.approx(math.sqrt(float(np.mean(v.astype(np.float64))) + dark), rel=1e-12)
    assert r["mean"][0] == pytest.approx(float(np.mean(v.astype(np.float64))), rel=1e-12)


def test_split_coefficients_weight_the_variance_by_c_squared():
    rng = np.random.default_rng(2)
    n = 300
    v = rng.uniform(1, 50, n).astype(np.float32)
    c = rng.choice([0.25, 0.5, 0.75, 1.0], n)
    W, v = one_bin(v, c=c)
    r = oracle.integrate_clip(W, v, n_iter=0, model=oracle.ERROR_POISSON, dark=1.0)
    x = v.astype(np.float64)
    want = math.sqrt(float(np.sum(c * c * (x + 1.0)) / np.sum(c * c)))
    assert r["sigma"][0] == pytest.approx(want, rel=1e-12)
    assert r["mean"][0] == pytest.approx(float(np.sum(c * x) / np.sum(c)), rel=1e-12)


@pytest.mark.parametrize("seed", range(5))
def test_poisson_clip_against_brute_force(seed):
    rng = np.random.default_rng(10 + seed)
    n = int(rng.integers(20, 120))
    v = rng.poisson(20.0, n).astype(np.float64)
    v[rng.integers(0, n, 4)] += rng.uniform(30, 200, 4)
    v = v.astype(np.float32)
    W, v = one_bin(v)
    r = oracle.integrate_clip(W, v, n_iter=10, k=3.0, model=oracle.ERROR_POISSON, dark=0.5)
    s = np.ones(n, bool)
    x = v.astype(np.float64)
    for _ in range(10):
        mu = x[s].mean()
        sp = math.sqrt(x[s].mean() + 0.5)
        new = s & (np.abs(x - mu) <= 3.0 * sp)
        if np.array_equal(new, s):
            break
        s = new
    assert r["count"][0] == int(s.sum())
    assert r["mean"][0] == pytest.approx(x[s].mean(), rel=1e-12)
    assert r["sigma"][0] == pytest.approx(math.sqrt(x[s].mean() + 0.5), rel=1e-12)
