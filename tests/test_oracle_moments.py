"""Pins of the oracle's moments and sigma-clipping (Eqs. 2, 6, 8-13, 17, 19;
Section 2.4) against values the paper prints, closed forms, special cases
and an independent interval-based brute force."""
import json
import math
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def one_bin(values, c=None, nbins=1, bins=None):
    v = np.asarray(values, np.float32)
    n = v.size
    pix = np.arange(n, dtype=np.int32)
    b = np.zeros(n, np.int32) if bins is None else np.asarray(bins, np.int32)
    cc = np.ones(n) if c is None else np.asarray(c, np.float64)
    W = oracle.Weights(pix, b, cc, np.zeros(n, np.int32), (0.0, 1.0), nbins, n)
    return W, v


def test_two_pixel_example_of_the_paper():
    g = json.load(open(os.path.join(GOLD, "paper_two_pixel.json")))
    W, v = one_bin(g["values"])
    r = oracle.integrate_clip(W, v, n_iter=5, k=3.0)
    assert r["mean"][0] == g["mean"]
    # "close to 100": the population deviation (Eq. 13, no Bessel correction) is 99
    assert r["sigma"][0] == pytest.approx(99.0, abs=1e-12)
    assert abs(r["sigma"][0] - g["azimuthal_std_close_to"]) < 2
    # both pixels lie at 1 sigma with the azimuthal model: k = 3 rejects neither
    assert r["count"][0] == 2 and r["iters"][0] == 0
    dist = abs(v - r["mean"][0]) / r["sigma"][0]
    assert np.allclose(dist, g["distance_in_azimuthal_sigmas"], atol=0.02)
    # with the Poisson deviation sqrt(<I>) they would be ~10 sigma away
    assert np.allclose(abs(v - 100.0) / math.sqrt(100.0), g["distance_in_poisson_sigmas"], atol=0.2)


def test_boundary_equality_is_kept():
    g = json.load(open(os.path.join(GOLD, "boundary_equality.json")))
    W, v = one_bin(g["values"])
    r = oracle.integrate_clip(W, v, n_iter=5, k=g["k_equal"])
    assert (r["mean"][0], r["sigma"][0], r["count"][0]) == (g["at_k_equal"]["mean"], g["at_k_equal"]["sigma"],
                                                         g["at_k_equal"]["count"])
    r = oracle.integrate_clip(W, v, n_iter=5, k=g["k_below"])
    assert (r["mean"][0], r["sigma"][0], r["count"][0]) == (g["at_k_below"]["mean"], g["at_k_below"]["sigma"],
                                                         g["at_k_below"]["count"])
    assert r["iters"][0] == 1


@pytest.mark.parametrize("n", [2, 3, 10, 101, 1000])
def test_arithmetic_progression_closed_form(n):
    W, v = one_bin(np.arange(1, n + 1))
    r = oracle.integrate_clip(W, v, n_iter=0)
    assert r["mean"][0] == pytest.approx((n + 1) / 2, rel=1e-15)
    assert r["sigma"][0] ** 2 == pytest.approx((n * n - 1) / 12.0, rel=1e-12)
    # a uniform set never has a member beyond sqrt(3) sigma: k = 3 keeps all
    r = oracle.integrate_clip(W, v, n_iter=5, k=3.0)
    assert r["count"][0] == n and r["iters"][0] == 0


def test_constant_bin_and_degenerate_bins():
    W, v = one_bin([7.25] * 50 + [3.0], bins=[0] * 50 + [1], nbins=3)
    r = oracle.integrate_clip(W, v, n_iter=5, k=3.0)
    # constant bin: mean = constant, sigma = 0, nothing rejected
    assert r["mean"][0] == 7.25 and r["sigma"][0] == 0.0 and r["count"][0] == 50
    # single entry: sigma = 0, never rejected
    assert r["mean"][1] == 3.0 and r["sigma"][1] == 0.0 and r["count"][1] == 1
    # empty bin: mean = sigma = 0, count 0
    assert r["mean"][2] == 0.0 and r["sigma"][2] == 0.0 and r["count"][2] == 0


def test_incremental_union_update_matches_two_pass():
    """Eq. 17 (adding one member b to a partition A) built up pixel by pixel
    gives the same VV as the two-pass Eq. 6 for unit weights."""
    rng = np.random.default_rng(3)
    vals = rng.normal(5.0, 2.0, 500).astype(np.float32).astype(np.float64)
    Om = V = VV = 0.0
    for x in vals:
        if Om == 0:
            Om, V, VV = 1.0, x, 0.0
            continue
        muA = V / Om
        Om2, V2 = Om + 1.0, V + x
        VV = VV + (x - muA) * (x - V2 / Om2)
        Om, V = Om2, V2
    W, v = one_bin(vals)
    r = oracle.integrate_clip(W, v, n_iter=0)
    assert r["mean"][0] == pytest.approx(V / Om, rel=1e-13)
    assert r["sigma"][0] == pytest.approx(math.sqrt(VV / Om), rel=1e-11)


def test_invariances_scale_shift_and_norm():
    rng = np.random.default_rng(5)
    vals = rng.normal(10.0, 3.0, 400).astype(np.float32)
    c = rng.choice([0.25, 0.5, 0.75, 1.0], 400)
    W, v = one_bin(vals, c=c)
    base = oracle.integrate_clip(W, v, n_iter=5, k=2.5)
    # scaling by a power of two is exact in binary floating point
    r = oracle.integrate_clip(W, v * np.float32(4.0), n_iter=5, k=2.5)
    assert r["mean"][0] == pytest.approx(4 * base["mean"][0], rel=1e-14)
    assert r["sigma"][0] == pytest.approx(4 * base["sigma"][0], rel=1e-14)
    assert r["count"][0] == base["count"][0]
    # Eq. 1: signal and norm scaled together leave v = signal / norm and the
    # relative weights unchanged
    s = np.float32(2.0)
    r = oracle.integrate_clip(W, v * s, norm=np.full(400, s, np.float32), n_iter=5, k=2.5)
    assert r["mean"][0] == pytest.approx(base["mean"][0], rel=1e-14)
    assert r["sigma"][0] == pytest.approx(base["sigma"][0], rel=1e-14)


def test_norm_weights_the_mean_eq2():
    """Eq. 2: <I> = sum c signal / sum c norm, not the plain mean of v."""
    sig = np.array([2.0, 8.0], np.float32)
    nrm = np.array([1.0, 4.0], np.float32)  # v = 2, 2 -> mean 2 regardless
    W, _ = one_bin(sig)
    r = oracle.integrate_clip(W, sig, norm=nrm, n_iter=0)
    assert r["mean"][0] == 2.0 and r["sigma"][0] == 0.0
    sig = np.array([1.0, 8.0], np.float32)  # v = 1, 2 -> (1 + 8) / (1 + 4) = 1.8
    r = oracle.integrate_clip(W, sig, norm=nrm, n_iter=0)
    assert r["mean"][0] == pytest.approx(1.8, rel=1e-15)
    # Eq. 6: sigma^2 = (1^2 (1 - 1.8)^2 + 4^2 (2 - 1.8)^2) / (1 + 16) = 1.28 / 17
    assert r["sigma"][0] ** 2 == pytest.approx((0.64 + 16 * 0.04) / 17.0, rel=1e-13)


def truncated_normal_sequence(k, steps):
    """Deviation ratio after each cumulative clip of a normal distribution:
    x_{t+1}^2 = 1 - 2 a phi(a) / (2 Phi(a) - 1), a = k x_t, x_0 = 1."""
    from scipy.stats import norm as N
    xs = [1.0]
    for _ in range(steps):
        a = k * xs[-1]
        xs.append(math.sqrt(1.0 - 2.0 * a * N.pdf(a) / (2.0 * N.cdf(a) - 1.0)))
    return xs


def test_truncated_normal_closed_form():
    xs = truncated_normal_sequence(3.0, 60)
    assert xs[1] == pytest.approx(0.98658, abs=2e-5)
    assert xs[-1] == pytest.approx(0.984846, abs=2e-6)
    rng = np.random.default_rng(11)
    m, s, n = 40.0, 2.5, 400_000
    vals = rng.normal(m, s, n).astype(np.float32)
    W, v = one_bin(vals)
    r = oracle.integrate_clip(W, v, n_iter=5, k=3.0)
    ratio = r["sigma"][0] / s
    # sampling error of a deviation estimate ~ 1/sqrt(2n) ~ 1.1e-3
    assert ratio == pytest.approx(xs[5], abs=6e-3)
    assert r["mean"][0] == pytest.approx(m, abs=6 * s / math.sqrt(n))
    # the clipped share agrees with 2 Phi(3 x_4) - 1
    from scipy.stats import norm as N
    frac = r["count"][0] / n
    assert frac == pytest.approx(2 * N.cdf(3 * xs[4]) - 1, abs=6 * math.sqrt(0.003 / n))


def test_poisson_bins_approach_truncated_normal():
    rng = np.random.default_rng(12)
    lam = 80.0
    vals = rng.poisson(lam, 300_000).astype(np.float32)
    W, v = one_bin(vals)
    r = oracle.integrate_clip(W, v, n_iter=5, k=3.0)
    xs = truncated_normal_sequence(3.0, 5)
    assert r["sigma"][0] / math.sqrt(lam) == pytest.approx(xs[5], abs=0.02)


def test_early_exit_makes_iteration_cap_irrelevant():
    rng = np.random.default_rng(13)
    vals = np.concatenate([rng.normal(0, 1, 3000), [40, 55, -30]]).astype(np.float32)
    W, v = one_bin(vals)
    r50 = oracle.integrate_clip(W, v, n_iter=50, k=3.0)
    assert r50["iters"][0] < 50
    r = oracle.integrate_clip(W, v, n_iter=int(r50["iters"][0]) + 1, k=3.0)
    assert (r["mean"][0], r["sigma"][0], r["count"][0]) == (r50["mean"][0], r50["sigma"][0], r50["count"][0])
    # one step fewer than needed gives a different (larger) set
    r = oracle.integrate_clip(W, v, n_iter=int(r50["iters"][0]) - 1, k=3.0)
    assert r["count"][0] > r50["count"][0]


def interval_clip(vals, c, n_iter, k):
    """Brute force by a different route: with cumulative rejection every set
    S_t is the set of entries whose value lies in an interval [L_t, H_t],
    so track the interval on sorted values instead of per-entry flags."""
    order = np.argsort(vals, kind="stable")
    x = vals[order].astype(np.float64)
    w = c[order].astype(np.float64)
    L, H = -np.inf, np.inf

    def mom(L, H):
        sel = (x >= L) & (x <= H) & (w > 0)
        if not sel.any():
            return 0.0, 0.0, 0
        ww, xx = w[sel], x[sel]
        mu = (ww * xx).sum() / ww.sum()
        return mu, math.sqrt((ww * ww * (xx - mu) ** 2).sum() / (ww * ww).sum()), int(sel.sum())

    for _ in range(n_iter):
        mu, sd, n = mom(L, H)
        L2, H2 = max(L, mu - k * sd), min(H, mu + k * sd)
        if mom(L2, H2)[2] == n:
            break
        L, H = L2, H2
    return mom(L, H)


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_32x32_interval_route(seed):
    """A 32 x 32 frame with 6 bins of mixed coefficients and outliers: the
    oracle's per-entry clipping equals the interval brute force."""
    rng = np.random.default_rng(100 + seed)
    npix = 32 * 32
    sig = rng.normal(3.0, 1.0, npix)
    hot = rng.choice(npix, 20, replace=False)
    sig[hot] += rng.uniform(5, 50, 20)
    sig = sig.astype(np.float32)
    # each pixel in one or two bins with coefficients summing to 1
    pix, b, c = [], [], []
    for i in range(npix):
        b0 = i * 6 // npix
        if i % 3 == 0 and b0 < 5:
            pix += [i, i]; b += [b0, b0 + 1]; c += [0.75, 0.25]
        else:
            pix += [i]; b += [b0]; c += [1.0]
    W = oracle.Weights(np.array(pix, np.int32), np.array(b, np.int32), np.array(c), np.zeros(npix, np.int32),
                       (0, 1), 6, npix)
    r = oracle.integrate_clip(W, sig, n_iter=5, k=2.5)
    for bb in range(6):
        sel = W.bin == bb
        mu, sd, n = interval_clip(sig[W.pix[sel]], W.c[sel], 5, 2.5)
        assert r["mean"][bb] == pytest.approx(mu, rel=1e-12, abs=1e-12)
        assert r["sigma"][bb] == pytest.approx(sd, rel=1e-10, abs=1e-12)
        assert r["count"][bb] == n


def test_exact_weighted_merge_identity():
    """The exact merge of two partial moment sets with omega^2 weights used by
    the GPU's cross-block reduction: with U = sum w^2 v and VV about each
    part's own mean, VV_{A+B} = sum_X VV_X + 2 (mu_X - mu)(U_X - OO_X mu_X)
    + OO_X (mu_X - mu)^2. It reduces to Eq. 18's Chan form when w^2 = w."""
    rng = np.random.default_rng(21)
    v = rng.normal(2.0, 3.0, 1000)
    w = rng.choice([0.25, 0.5, 0.75, 1.0], 1000) * rng.uniform(0.5, 2.0, 1000)

    def part(vv, ww):
        Om, OO, V, U = ww.sum(), (ww * ww).sum(), (ww * vv).sum(), (ww * ww * vv).sum()
        mu = V / Om
        return Om, OO, V, U, (ww * ww * (vv - mu) ** 2).sum()

    for cut in (1, 17, 500, 999):
        A, B = part(v[:cut], w[:cut]), part(v[cut:], w[cut:])
        mu = (A[2] + B[2]) / (A[0] + B[0])
        VV = 0.0
        for X in (A, B):
            muX = X[2] / X[0]
            VV += X[4] + 2 * (muX - mu) * (X[3] - X[1] * muX) + X[1] * (muX - mu) ** 2
        full = part(v, w)
        assert VV == pytest.approx(full[4], rel=1e-11)
    # with unit weights it is Eq. 18 (Chan et al.)
    A, B = part(v[:300], np.ones(300)), part(v[300:], np.ones(700))
    chan = A[4] + B[4] + B[1] * (A[2] * B[0] - B[2] * A[0]) ** 2 / ((A[0] + B[0]) * A[0] * B[0] ** 2)
    assert chan == pytest.approx(part(v, np.ones(1000))[4], rel=1e-11)
