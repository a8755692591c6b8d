"""Pins of the sparsification threshold taken from the smooth background
(Section 3: the compressed format keeps the background level and its
deviation as a function of the distance to the beam centre, and every
pixel's distance; the threshold of a pixel is that profile at the pixel,
mu(x_i) + k_pick sigma(x_i), interpolated linearly between bin centres).

Pinned against closed forms: on a profile linear in the radial value the
interpolated threshold is that line at the pixel centre's own radial value
(computed here from the geometry, not by the oracle), so pixels placed a
relative 1e-6 above / below it are kept / dropped exactly; beyond the outer
bin centres the end bins' levels hold; a constant profile gives the per-bin
result; the peak records subtract the interpolated background."""
import math

import numpy as np

import oracle
import synth


def _radial_2theta_deg(det):
    """Pixel-centre 2theta in degrees straight from the flat geometry."""
    py, px = det.pixel_m
    cx, cy = det.center_px
    r, c = np.divmod(np.arange(det.npix), det.cols)
    dy = (r + 0.5 - cy) * py
    dx = (c + 0.5 - cx) * px
    return np.degrees(np.arctan2(np.hypot(dx, dy), det.dist_m))


def _linear_setup(alpha=40.0, beta=-3.0, gamma=2.0, delta=0.25):
    det = synth.det_config1()
    W = oracle.weights(det)
    lo, hi = W.range
    B = W.nbins
    centres = lo + (np.arange(B) + 0.5) * (hi - lo) / B
    mean = alpha + beta * centres
    sigma = gamma + delta * centres
    x = _radial_2theta_deg(det)
    xc = np.clip(x, centres[0], centres[-1])          # end bins' levels beyond the outer centres
    return det, W, mean, sigma, alpha + beta * xc, gamma + delta * xc


def test_linear_profile_threshold_is_the_line_at_each_pixel():
    det, W, mean, sigma, mu_x, sd_x = _linear_setup()
    k = 3.0
    thr = mu_x + k * sd_x
    rng = np.random.default_rng(4)
    above = rng.random(det.npix) < 0.5
    sig = np.where(above, thr * (1 + 1e-6), thr * (1 - 1e-6)).astype(np.float32)
    interp = oracle.interpolation(det, W, exact=True)
    idx, val = oracle.sparsify(W, sig, mean, sigma, k, interp=interp)
    assert np.array_equal(idx, np.flatnonzero(above))
    assert np.array_equal(val, sig[idx].astype(np.float64))
    # the per-bin threshold misses the line by up to half a bin's slope
    idx_bin, _ = oracle.sparsify(W, sig, mean, sigma, k)
    assert not np.array_equal(idx_bin, idx)


def test_end_bins_hold_beyond_the_outer_centres():
    det, W, mean, sigma, _, _ = _linear_setup()
    lo, hi = W.range
    B = W.nbins
    x = _radial_2theta_deg(det)
    interp = oracle.interpolation(det, W, exact=True)
    mu = oracle.profile_at(interp, mean, B)
    first = x <= lo + 0.5 * (hi - lo) / B
    last = x >= lo + (B - 0.5) * (hi - lo) / B
    assert first.any() and last.any()
    assert np.all(mu[first] == mean[0]) and np.all(mu[last] == mean[-1])
    # and a pixel centre on a bin centre takes that bin's level
    a, t = interp
    inner = ~first & ~last
    assert np.all((a[inner] >= 0) & (a[inner] < B - 1) & (t[inner] >= 0) & (t[inner] < 1))


def test_constant_profile_gives_the_per_bin_result():
    det = synth.det_config1()
    mask = np.zeros(det.npix, np.uint8)
    mask[::97] = 1
    W = oracle.weights(det, mask)
    fr = synth.frames(det, synth.spec_config1(2), 0, 1)[0][0].astype(np.float32)
    mean = np.full(W.nbins, 31.0)
    sigma = np.full(W.nbins, 6.0)
    interp = oracle.interpolation(det, W, exact=True)
    i0, v0 = oracle.sparsify(W, fr, mean, sigma, 3.0)
    i1, v1 = oracle.sparsify(W, fr, mean, sigma, 3.0, interp=interp)
    assert i0.size > 0 and np.array_equal(i0, i1) and np.array_equal(v0, v1)
    assert not np.isin(np.flatnonzero(mask), i1).any()
    p0 = oracle.peaks(det, W, fr, mean, sigma)
    p1 = oracle.peaks(det, W, fr, mean, sigma, interp=interp)
    assert p0.size > 0 and np.array_equal(p0, p1)


def test_peak_record_subtracts_the_interpolated_background():
    det, W, mean, sigma, mu_x, sd_x = _linear_setup(alpha=10.0, beta=-1.0, gamma=1.0, delta=0.1)
    sig = np.asarray(mu_x, np.float32)                  # background exactly on the line: nothing kept
    r0, c0 = 100, 60
    block = [(r, c) for r in range(r0 - 1, r0 + 2) for c in range(c0 - 1, c0 + 2)]
    for (r, c) in block:
        sig[r * det.cols + c] = np.float32(500.0 + (r - r0) * 3 + (c - c0) * 7)
    sig[r0 * det.cols + c0] = np.float32(900.0)
    interp = oracle.interpolation(det, W, exact=True)
    pk = oracle.peaks(det, W, sig, mean, sigma, k_pick=3.0, patch=3, min_count=3, interp=interp)
    assert pk.size == 1 and pk["idx"][0] == r0 * det.cols + c0 and pk["npix"][0] == 9
    js = [r * det.cols + c for (r, c) in block]
    w = np.array([float(sig[j]) - mu_x[j] for j in js])
    I = w.sum()
    y = sum(wk * (r + 0.5) for wk, (r, c) in zip(w, block)) / I
    x = sum(wk * (c + 0.5) for wk, (r, c) in zip(w, block)) / I
    s = math.sqrt(sum(sd_x[j] ** 2 for j in js))
    for got, want in ((pk["I"][0], I), (pk["y"][0], y), (pk["x"][0], x), (pk["sigma"][0], s)):
        assert abs(got - want) <= 1e-9 * abs(want)
