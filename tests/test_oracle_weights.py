"""Pins of the oracle's pixel-to-bin coefficients c_{i,r} (Section 2.2):
coefficients sum to one per pixel, splitting off gives ones only, mirror
pixels get the same bins, the automatic range follows the farthest corner in
closed form, and every sub-pixel lands in the bin that the *inverse* unit
mapping (radius of each bin edge) assigns to it."""
import math

import numpy as np
import pytest

import oracle
import synth


def small_det(unit, split, nbins=37, rows=40, cols=52, center=(23.3, 17.8), dist=0.05):
    return synth.Detector("t", rows, cols, dist_m=dist, center_px=center, unit=unit, nbins=nbins, split=split)


@pytest.mark.parametrize("split", [1, 2, 3])
def test_coefficients_sum_to_one(split):
    d = small_det(synth.UNIT_Q_NM, split)
    mask = np.zeros(d.npix, np.uint8)
    mask[::7] = 1
    W = oracle.weights(d, mask)
    tot = np.bincount(W.pix, weights=W.c, minlength=d.npix)
    # exact for s = 1, 2 (dyadic fractions); to rounding for s = 3
    tol = 0.0 if split in (1, 2) else 4e-16
    assert np.all(np.abs(tot[mask == 0] - 1.0) <= tol)
    assert np.all(tot[mask == 1] == 0.0)
    assert np.all(W.bin_of_pixel[mask == 1] == -1)
    assert abs(W.c.sum() - (mask == 0).sum()) <= tol * W.c.size
    if split == 1:
        assert np.all(W.c == 1.0) and W.pix.size == (mask == 0).sum()
    # coefficients are multiples of 1/s^2
    k = W.c * split * split
    assert np.all(np.abs(k - np.round(k)) <= 1e-12)


@pytest.mark.parametrize("unit", [synth.UNIT_2TH_DEG, synth.UNIT_Q_NM, synth.UNIT_R_MM])
def test_mirror_pixels_share_bins(unit):
    rows, cols = 30, 44
    d = small_det(unit, 2, rows=rows, cols=cols, center=(cols / 2, rows / 2))
    W = oracle.weights(d)
    ent = {}
    for p, b, c in zip(W.pix, W.bin, W.c):
        ent.setdefault(int(p), []).append((int(b), float(c)))
    for r in range(rows):
        for c in range(cols):
            i = r * cols + c
            for j in ((rows - 1 - r) * cols + c, r * cols + (cols - 1 - c), (rows - 1 - r) * cols + cols - 1 - c):
                assert ent[i] == ent[j]


def test_auto_range_config1_closed_form():
    d = synth.det_config1()
    lo, hi = oracle.unit_range(d)
    # farthest pixel centre from (x, y) = (128.3, 120.7): column 0 (x = 0.5) and row 255 (y = 255.5)
    rmax = math.hypot(128.3 - 0.5, 255.5 - 120.7) * 75e-6
    assert hi == pytest.approx(math.degrees(math.atan(rmax / 0.1)), rel=1e-12)
    assert hi == pytest.approx(7.93, abs=0.01)
    # nearest pixel centre: (128.5, 120.5)
    rmin = math.hypot(0.2, 0.2) * 75e-6
    assert lo == pytest.approx(math.degrees(math.atan(rmin / 0.1)), rel=1e-9)
    W = oracle.weights(d)
    assert W.bin.min() == 0 and W.bin.max() == 63
    assert W.range == (lo, hi)


def edge_radii(det, lo, hi):
    B = det.nbins
    x = lo + (hi - lo) * np.arange(B + 1) / B
    if det.unit == synth.UNIT_2TH_DEG:
        return det.dist_m * np.tan(np.radians(x))
    if det.unit == synth.UNIT_Q_NM:
        lam_nm = det.wavelength_m * 1e9
        return det.dist_m * np.tan(2.0 * np.arcsin(x * lam_nm / (4 * np.pi)))
    return x / 1e3


@pytest.mark.parametrize("unit,split", [(synth.UNIT_2TH_DEG, 1), (synth.UNIT_Q_NM, 2), (synth.UNIT_R_MM, 2),
                                        (synth.UNIT_Q_NM, 3)])
def test_bins_from_inverse_unit(unit, split):
    d = small_det(unit, split)
    W = oracle.weights(d)
    lo, hi = W.range
    R = edge_radii(d, lo, hi)
    rows, cols, s = d.rows, d.cols, split
    off = (np.arange(s) + 0.5) / s
    rr, cc = np.meshgrid(np.arange(rows), np.arange(cols), indexing="ij")
    want = np.zeros((d.npix, d.nbins))
    near_edge = np.zeros(d.npix, bool)
    for fy in off:
        for fx in off:
            dy = (rr + fy - d.center_px[1]) * d.pixel_m[0]
            dx = (cc + fx - d.center_px[0]) * d.pixel_m[1]
            r = np.hypot(dx, dy).ravel()
            b = np.clip(np.searchsorted(R, r, side="right") - 1, 0, d.nbins - 1)
            want[np.arange(d.npix), b] += 1.0 / (s * s)
            rel = np.min(np.abs(r[:, None] - R[None, 1:-1]), axis=1) / r.max()
            near_edge |= rel < 1e-9
    got = np.zeros((d.npix, d.nbins))
    got[W.pix, W.bin] = W.c
    bad = np.any(np.abs(got - want) > 1e-12, axis=1)
    assert not np.any(bad & ~near_edge)
    assert bad.sum() <= max(2, d.npix // 1000)


def test_bin_of_pixel_is_centre_bin():
    d = small_det(synth.UNIT_2TH_DEG, 1)
    W = oracle.weights(d)
    # without splitting the only coefficient of a pixel is its centre's bin
    assert np.array_equal(W.bin_of_pixel[W.pix], W.bin)
    d2 = small_det(synth.UNIT_2TH_DEG, 2)
    W2 = oracle.weights(d2)
    lo, hi = W2.range
    R = edge_radii(d2, lo, hi)
    rr, cc = np.meshgrid(np.arange(d2.rows), np.arange(d2.cols), indexing="ij")
    r = np.hypot((cc + 0.5 - d2.center_px[0]) * 75e-6, (rr + 0.5 - d2.center_px[1]) * 75e-6).ravel()
    b = np.clip(np.searchsorted(R, r, side="right") - 1, 0, d2.nbins - 1)
    assert np.mean(b == W2.bin_of_pixel) > 0.999
