"""Exact-area coefficients (Section 2.2: c_{i,r} is the fraction of pixel
i's area in radial bin r). The oracle's fractions are pinned by a brute-force
count over a fine sub-pixel grid, by the partition of every pixel's area
(the fractions of a pixel inside the range sum to one) and by the symmetry
of pixels mirrored about the beam centre; the library's host-built matrix
(split 0) then matches the oracle entry by entry."""
import math

import numpy as np
import pytest

import oracle
import synth
from paper_2411_09515_gb300 import _binding as B


def _det(unit, nbins=9, center=(6.3, 5.7), rng=(math.nan, math.nan)):
    d = synth.Detector("exact", 12, 14, dist_m=0.05, center_px=center, nbins=nbins, split=0, unit=unit)
    d.range = rng
    return d


def _brute(det, W, n=160):
    """Fraction of n x n sub-pixel centres per (pixel, bin), same range."""
    lo, hi = W.range
    out = {}
    f = (np.arange(n) + 0.5) / n
    for i in np.unique(W.pix):
        r, c = divmod(int(i), det.cols)
        yy = (r + f[:, None] - det.center_px[1]) * det.pixel_m[0]
        xx = (c + f[None, :] - det.center_px[0]) * det.pixel_m[1]
        R = np.hypot(xx, yy)
        if det.unit == synth.UNIT_R_MM:
            x = R * 1e3
        else:
            tth = np.arctan2(R, det.dist_m)
            x = np.degrees(tth) if det.unit == synth.UNIT_2TH_DEG else \
                4 * np.pi * np.sin(tth / 2) / (det.wavelength_m * 1e9)
        b = np.floor((x - lo) / (hi - lo) * det.nbins).astype(int)
        inside = (x >= lo) & (x <= hi)
        b = np.clip(b, 0, det.nbins - 1)[inside]
        for k, cnt in zip(*np.unique(b, return_counts=True)):
            out[(int(i), int(k))] = cnt / (n * n)
    return out


@pytest.mark.parametrize("unit", [synth.UNIT_R_MM, synth.UNIT_2TH_DEG, synth.UNIT_Q_NM])
def test_fractions_against_a_fine_grid(unit):
    det = _det(unit)
    W = oracle.weights_exact(det)
    brute = _brute(det, W)
    got = {(int(p), int(b)): c for p, b, c in zip(W.pix, W.bin, W.c)}
    for key in set(got) | set(brute):
        assert abs(got.get(key, 0.0) - brute.get(key, 0.0)) < 0.02, key   # sub-sampling error ~ 1/n per edge


def test_fractions_partition_each_pixel():
    det = _det(synth.UNIT_2TH_DEG, nbins=23)
    W = oracle.weights_exact(det)
    tot = np.bincount(W.pix, weights=W.c, minlength=det.npix)
    assert np.allclose(tot, 1.0, atol=1e-12)
    # a range that cuts the pixels: fractions outside it are dropped
    lo, hi = W.range
    det2 = _det(synth.UNIT_2TH_DEG, nbins=23, rng=(lo + 0.3 * (hi - lo), hi))
    W2 = oracle.weights_exact(det2)
    tot2 = np.bincount(W2.pix, weights=W2.c, minlength=det.npix)
    assert np.all(tot2 <= 1 + 1e-12) and np.any((tot2 > 0) & (tot2 < 1 - 1e-6))


def test_mirror_symmetry_about_a_pixel_corner():
    det = _det(synth.UNIT_R_MM, nbins=7, center=(7.0, 6.0))    # the beam on a pixel corner
    W = oracle.weights_exact(det)
    got = {(int(p), int(b)): c for p, b, c in zip(W.pix, W.bin, W.c)}
    for (p, b), c in got.items():
        r, cl = divmod(p, det.cols)
        rm, cm = 2 * 6 - 1 - r, 2 * 7 - 1 - cl                   # mirrored through the corner
        if 0 <= rm < det.rows and 0 <= cm < det.cols:
            assert got.get((rm * det.cols + cm, b), 0.0) == pytest.approx(c, abs=1e-12)


@pytest.mark.parametrize("unit", [synth.UNIT_R_MM, synth.UNIT_Q_NM])
def test_library_matrix_matches_the_oracle(unit):
    det = _det(unit, nbins=11)
    mask = np.zeros(det.npix, np.uint8)
    mask[::17] = 1
    geo = B.make_geometry(det.rows, det.cols, det.pixel_m, det.dist_m, det.center_px, det.wavelength_m, det.unit,
                          det.nbins, det.split, det.range)
    csr = B.sep_build_csr(None, geo, mask)
    try:
        ex = B.sep_csr_export(csr)
    finally:
        B.sep_csr_destroy(csr)
    W = oracle.weights_exact(det, mask)
    assert ex["range"][0] == pytest.approx(W.range[0], abs=1e-12) and ex["range"][1] == pytest.approx(W.range[1],
                                                                                                     rel=1e-12)
    assert np.array_equal(ex["bin_of_pixel"], W.bin_of_pixel)
    rows = np.repeat(np.arange(det.nbins), np.diff(ex["rowptr"]))
    nz = ex["coef"] != 0
    got = {(int(p), int(b)): float(c) for p, b, c in zip(ex["col"][nz], rows[nz], ex["coef"][nz])}
    want = {(int(p), int(b)): float(c) for p, b, c in zip(W.pix, W.bin, W.c)}
    assert set(got) == set(want)
    for k in want:
        assert got[k] == pytest.approx(want[k], rel=2e-7, abs=1e-12)   # binary32 coefficients


def test_library_refuses_bins_far_narrower_than_pixels():
    det = _det(synth.UNIT_R_MM, nbins=4000)
    geo = B.make_geometry(det.rows, det.cols, det.pixel_m, det.dist_m, det.center_px, det.wavelength_m, det.unit,
                          det.nbins, det.split, det.range)
    with pytest.raises(B.SepError) as e:
        B.sep_build_csr(None, geo, None)
    assert e.value.status == B.SEP_ERR_ARG
