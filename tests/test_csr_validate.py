"""Host-side validation of integration matrices (no GPU): a matrix the
library builds passes; every kind of corruption a kernel could follow out
of bounds (a non-monotone row pointer, a column or bin out of range, a
coefficient outside [0, 1] or a pixel's coefficients summing above its
area, Section 2.2) and a calibration of another size are refused before any
launch."""
import numpy as np
import pytest

import synth
from paper_2411_09515_gb300 import _binding as B
from tests.test_lib_host import geom_of


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2411_09515_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def small():
    det = synth.det_small_jf(split=2, nbins=64)
    csr = B.sep_build_csr(None, geom_of(det), det.mask())
    ex = B.sep_csr_export(csr)
    yield det, csr, ex
    B.sep_csr_destroy(csr)


def _validate(ex, npix, calib_npix=-1, **over):
    a = {k: ex[k].copy() for k in ("rowptr", "col", "coef", "bin_of_pixel")}
    a.update(over)
    return B.sep_csr_validate(a["rowptr"], a["col"], a["coef"], a["bin_of_pixel"], npix, calib_npix)


def test_built_matrix_passes(small):
    det, csr, ex = small
    st, msg = _validate(ex, det.npix, calib_npix=det.npix)
    assert st == B.SEP_OK and msg == ""
    assert B.sep_csr_check(csr) == B.SEP_OK


def test_non_monotone_rowptr_refused(small):
    det, _, ex = small
    rp = ex["rowptr"].copy()
    b = int(np.argmax(np.diff(rp) > 0))
    rp[b + 1], rp[b + 2] = rp[b + 2], rp[b + 1]   # one row pointer runs backwards
    assert np.any(np.diff(rp) < 0)
    st, msg = _validate(ex, det.npix, rowptr=rp)
    assert st == B.SEP_ERR_ARG and "non-monotone" in msg


def test_row_pointer_total_must_match(small):
    det, _, ex = small
    rp = ex["rowptr"].copy()
    rp[-1] -= 4
    st, msg = _validate(ex, det.npix, rowptr=rp)
    assert st == B.SEP_ERR_ARG and "nnz" in msg


@pytest.mark.parametrize("value", [-2, "npix"])
def test_column_out_of_range_refused(small, value):
    det, _, ex = small
    col = ex["col"].copy()
    e = int(np.flatnonzero(col >= 0)[7])
    col[e] = det.npix if value == "npix" else value
    st, msg = _validate(ex, det.npix, col=col)
    assert st == B.SEP_ERR_ARG and "column out of range" in msg


def test_bin_of_pixel_out_of_range_refused(small):
    det, _, ex = small
    bop = ex["bin_of_pixel"].copy()
    bop[int(np.flatnonzero(bop >= 0)[3])] = len(ex["rowptr"]) - 1   # == nbins
    st, msg = _validate(ex, det.npix, bin_of_pixel=bop)
    assert st == B.SEP_ERR_ARG and "bin_of_pixel" in msg


@pytest.mark.parametrize("value", [1.5, -0.25, np.nan])
def test_coefficient_outside_unit_interval_refused(small, value):
    det, _, ex = small
    coef = ex["coef"].copy()
    coef[int(np.flatnonzero(coef > 0)[5])] = value
    st, msg = _validate(ex, det.npix, coef=coef)
    assert st == B.SEP_ERR_ARG and "coefficient" in msg


def test_pixel_area_above_one_refused(small):
    """A pixel split over two bins whose shares are each raised to 0.75
    covers more than its own area (the coefficients of Section 2.2 are area
    fractions)."""
    det, _, ex = small
    col, coef = ex["col"], ex["coef"].copy()
    half = np.flatnonzero((coef == 0.5) & (col >= 0))
    pix, first = np.unique(col[half], return_index=True)
    cnt = np.bincount(col[half], minlength=det.npix)
    p = pix[np.argmax(cnt[pix] == 2)]
    coef[(col == p) & (coef == 0.5)] = 0.75
    st, msg = _validate(ex, det.npix, coef=coef)
    assert st == B.SEP_ERR_ARG and "sum above 1" in msg


def test_padding_with_weight_refused(small):
    det, _, ex = small
    col, coef = ex["col"], ex["coef"].copy()
    pads = np.flatnonzero(col < 0)
    assert pads.size
    coef[pads[0]] = 0.25
    st, msg = _validate(ex, det.npix, coef=coef)
    assert st == B.SEP_ERR_ARG and "padding" in msg


def test_calibration_of_another_size_refused(small):
    det, _, ex = small
    st, msg = _validate(ex, det.npix, calib_npix=det.npix - 1)
    assert st == B.SEP_ERR_ARG and "calibration" in msg
