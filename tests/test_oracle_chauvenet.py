"""Pins of the Chauvenet cut-off (Eq. 20, Section 2.4): the values the paper
prints (2.7 for 100 entries, 3.5 for 1000; on a Poisson background of mean 1
the discarded intensities start at 4 and at 5), the closed form behind the
criterion (n times the normal density at the cut-off is one), the
two-pixel example (no clipping of a set of two), and the oracle's clip loop
against an independent brute force on small sets."""
import math

import numpy as np
import pytest

import oracle
from test_oracle_moments import one_bin


def test_cutoffs_the_paper_prints():
    assert oracle.chauvenet_k(100) == pytest.approx(2.7, abs=0.05)
    assert oracle.chauvenet_k(1000) == pytest.approx(3.5, abs=0.05)
    # lambda = mu = sigma^2 = 1: the threshold mu + k sigma lies between 3 and 4
    # for 100 entries, between 4 and 5 for 1000
    assert 3 < 1 + oracle.chauvenet_k(100) < 4
    assert 4 < 1 + oracle.chauvenet_k(1000) < 5
    # "typically from 2 to 4" over ring sizes of tens to thousands
    assert 2 < oracle.chauvenet_k(40) < oracle.chauvenet_k(5000) < 4


@pytest.mark.parametrize("n", [3, 10, 100, 4321, 10 ** 6])
def test_one_expected_entry_beyond_the_cutoff(n):
    # the criterion: n * phi(k) = 1, phi the standard normal density
    k = oracle.chauvenet_k(n)
    assert n * math.exp(-k * k / 2) / math.sqrt(2 * math.pi) == pytest.approx(1.0, rel=1e-12)


def test_sets_of_two_are_not_clipped():
    W, v = one_bin([1.0, 199.0])
    r = oracle.integrate_clip(W, v, n_iter=5, chauvenet=True)
    assert r["count"][0] == 2 and r["mean"][0] == 100.0 and r["iters"][0] == 0
    assert oracle.chauvenet_k(2) is None and oracle.chauvenet_k(3) is not None


def _brute(v, n_iter):
    s = np.ones(v.size, bool)
    steps = 0
    for _ in range(n_iter):
        x = v[s].astype(np.float64)
        if x.size <= 2:
            break
        mu = x.mean()
        sd = math.sqrt(((x - mu) ** 2).mean())
        k = math.sqrt(2 * math.log(x.size / math.sqrt(2 * math.pi)))
        new = s & (np.abs(v.astype(np.float64) - mu) <= k * sd)
        if np.array_equal(new, s):
            break
        s = new
        steps += 1
    x = v[s].astype(np.float64)
    return x.mean(), math.sqrt(((x - x.mean()) ** 2).mean()), int(s.sum()), steps


@pytest.mark.parametrize("seed", range(6))
def test_clip_loop_against_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 80))
    v = rng.normal(10, 2, n)
    v[rng.integers(0, n, 3)] += rng.uniform(10, 40, 3)        # a few outliers
    v = v.astype(np.float32)
    W, v = one_bin(v)
    r = oracle.integrate_clip(W, v, n_iter=20, chauvenet=True)
    mu, sd, cnt, steps = _brute(v, 20)
    assert r["count"][0] == cnt and r["iters"][0] == steps
    assert r["mean"][0] == pytest.approx(mu, rel=1e-12) and r["sigma"][0] == pytest.approx(sd, rel=1e-9, abs=1e-12)
