"""Oracle of the densification (Section 3, "Densification / Decompression")
pinned against what the paper and the mathematics fix: the round trip
restores every kept pixel exactly and the background of every other binned
pixel; the noisy background has its bin's mean and deviation (closed form
for standard normal deviates); a zero deviation gives a noise-free
background; and on normal data the share of kept pixels is the normal tail
the paper prints (about 16 %, 2.3 % and 0.13 % above 1, 2 and 3 deviations)."""
import math

import numpy as np

import oracle
import synth


def _frame(seed=3):
    det = synth.det_config1()
    fr = synth.frames(det, synth.spec_config1(seed), 0, 1)[0][0].astype(np.float32)
    return det, fr


def test_round_trip_restores_kept_pixels_and_the_binned_background():
    det, fr = _frame()
    mask = np.zeros(det.npix, np.uint8)
    mask[::53] = 1
    W = oracle.weights(det, mask)
    ref = oracle.integrate_clip(W, fr)
    idx, val = oracle.sparsify(W, fr, ref["mean"], ref["sigma"], 3.0)
    assert idx.size > 0
    out = oracle.densify(W, ref["mean"], ref["sigma"], idx, val)
    assert np.array_equal(out[idx], fr[idx])                 # exact values back
    bop = W.bin_of_pixel
    rest = np.ones(det.npix, bool)
    rest[idx] = False
    binned = rest & (bop >= 0)
    assert np.array_equal(out[binned], ref["mean"][bop[binned]].astype(np.float32))
    assert np.all(np.isnan(out[bop < 0])) and np.all(bop[mask == 1] < 0)
    out0 = oracle.densify(W, ref["mean"], ref["sigma"], idx, val, fill=-1.0)
    assert np.all(out0[bop < 0] == -1.0)


def test_noisy_background_has_the_bin_mean_and_deviation():
    det = synth.det_config1()
    W = oracle.weights(det)
    mean = np.full(W.nbins, 10.0, np.float32)
    sigma = np.full(W.nbins, 2.0, np.float32)
    z = np.random.default_rng(11).standard_normal(det.npix).astype(np.float32)
    out = oracle.densify(W, mean, sigma, np.empty(0, np.int32), np.empty(0, np.float32), noise=z)
    has = W.bin_of_pixel >= 0
    n = int(has.sum())
    m, s = float(out[has].mean()), float(out[has].std())
    assert abs(m - 10.0) < 5 * 2.0 / math.sqrt(n)
    assert abs(s - 2.0) < 5 * 2.0 / math.sqrt(2 * n)
    # zero deviation: the background is the mean whatever the deviates
    out0 = oracle.densify(W, mean, np.zeros_like(sigma), np.empty(0, np.int32), np.empty(0, np.float32), noise=z)
    assert np.all(out0[has] == 10.0)


def test_kept_share_of_normal_data_is_the_normal_tail():
    det = synth.det_small_jf(split=1, nbins=40)
    W = oracle.weights(det)
    rng = np.random.default_rng(5)
    fr = (100.0 + 5.0 * rng.standard_normal(det.npix)).astype(np.float32)
    mean = np.full(W.nbins, 100.0)
    sigma = np.full(W.nbins, 5.0)
    n = int((W.bin_of_pixel >= 0).sum())
    for k, printed in ((1, 0.16), (2, 0.023), (3, 0.0013)):
        idx, _ = oracle.sparsify(W, fr, mean, sigma, float(k))
        p = 0.5 * math.erfc(k / math.sqrt(2))          # the normal tail above k deviations
        assert abs(idx.size - n * p) < 5 * math.sqrt(n * p * (1 - p))
        assert abs(p - printed) / printed < 0.05          # the values the paper prints


def test_interpolated_background_reproduces_a_linear_profile():
    # the smooth background of Section 3: a profile linear in the radial
    # value is reproduced at every pixel between the outer bin centres
    det = synth.det_config1()
    W = oracle.weights(det)
    lo, hi = W.range
    B = W.nbins
    centres = lo + (np.arange(B) + 0.5) * (hi - lo) / B
    alpha, beta = 3.0, 0.7
    mean = (alpha + beta * centres).astype(np.float32)
    interp = oracle.interpolation(det, W)
    out = oracle.densify(W, mean, None, np.empty(0, np.int32), np.empty(0, np.float32), interp=interp)
    x = oracle.pixel_unit(det)
    inner = (x > centres[0]) & (x < centres[-1]) & (W.bin_of_pixel >= 0)
    assert np.allclose(out[inner], alpha + beta * x[inner], rtol=2e-6, atol=1e-5)
    # beyond the outer centres: the end bins' levels
    below = (x <= centres[0]) & (W.bin_of_pixel >= 0)
    above = (x >= centres[-1]) & (W.bin_of_pixel >= 0)
    assert below.any() and np.all(out[below] == mean[0])
    assert above.any() and np.all(out[above] == mean[-1])
    # the weights: in [0, 1), and the lower bin within one of the centre bin
    a, t = interp
    assert np.all((t >= 0) & (t < 1)) and np.all(np.abs(a - W.bin_of_pixel) <= 1)
