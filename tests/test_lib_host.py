"""Host-side checks of libsep that need no GPU: the library loads and
exports every symbol include/sep.h declares, argument errors are reported
before any launch, and the host-built integration matrix equals the oracle's
independently computed coefficients entry for entry."""
import os
import re

import numpy as np
import pytest

import oracle
import synth
from paper_2411_09515_gb300 import _binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2411_09515_gb300 import build
    build.build()


def header_functions():
    src = open(os.path.join(ROOT, "include", "sep.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sep_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    names = header_functions()
    assert sorted(B.EXPORTS) == names
    L = B.lib()
    for n in names:
        assert hasattr(L, n), n
    assert "sm_103a" in B.sep_version()


def test_constants_match_header():
    """Every numeric #define of the header has the same value in the binding."""
    src = open(os.path.join(ROOT, "include", "sep.h")).read()
    found = 0
    for name, val in re.findall(r"^#define[ \t]+(SEP_[A-Z_0-9]+)[ \t]+([^/\n]+)", src, flags=re.M):
        val = val.strip()
        if not val:
            continue
        assert hasattr(B, name), name
        assert getattr(B, name) == eval(val.replace("<<", " << "), {}), name
        found += 1
    assert found >= 30


def header_structs():
    """{name: [(field, c type, array length or 0), ...]} of the header's
    plain structs, in declaration order."""
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "sep.h")).read(), flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct\s*\{(.*?)\}\s*(\w+)\s*;", src, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            m = re.match(r"((?:const )?\w+\s*\*?)\s*(.*)", decl)
            ctype = m.group(1).replace(" ", "")
            for item in m.group(2).split(","):
                item = item.strip()
                if item.startswith("*"):
                    ctype, item = ctype + "*", item[1:]
                a = re.match(r"(\w+)(?:\[(\d+)\])?$", item)
                fields.append((a.group(1), ctype, int(a.group(2) or 0)))
        out[name] = fields
    return out


def test_struct_fields_match_header():
    """Field names, order and types of every ctypes struct equal the header's."""
    import ctypes as C
    cmap = {"int32_t": C.c_int32, "float": C.c_float, "double": C.c_double, "uint64_t": C.c_uint64,
            "constvoid*": C.c_void_p}
    hs = header_structs()
    for cls in (B.sep_geometry, B.sep_params, B.sep_train_cfg, B.sep_frame_desc):
        want = hs[cls.__name__]
        got = cls._fields_
        assert [f[0] for f in got] == [w[0] for w in want], cls.__name__
        for (name, ct), (_, htype, n) in zip(got, want):
            base = cmap[htype]
            assert ct == (base * n if n else base), (cls.__name__, name)
    assert list(B.PEAK_DTYPE.names) == [w[0] for w in hs["sep_peak"]]


def test_struct_layouts_match_header():
    import ctypes as C
    assert C.sizeof(B.sep_geometry) == 4 * 2 + 8 * 2 + 8 + 8 * 2 + 8 + 4 * 3 + 4 + 8 * 2  # padded before range
    assert C.sizeof(B.sep_params) == 44
    assert B.PEAK_DTYPE.itemsize == B.PEAK_BYTES == 24


def geom_of(det):
    return B.make_geometry(det.rows, det.cols, det.pixel_m, det.dist_m, det.center_px, det.wavelength_m, det.unit,
                           det.nbins, det.split, det.range)


@pytest.mark.parametrize("bad", [dict(rows=0), dict(nbins=0), dict(split=3), dict(unit=7), dict(dist_m=0.0),
                                 dict(rows=8192, cols=8192)])
def test_invalid_geometry_rejected(bad):
    det = synth.det_config1()
    for k, v in bad.items():
        setattr(det, k, v)
    with pytest.raises(B.SepError) as e:
        B.sep_build_csr(None, geom_of(det))
    assert e.value.status == B.SEP_ERR_ARG


TILE = (64, 64)   # staging tile (rows, columns) of the library


def compare_with_oracle(det, mask=None):
    csr = B.sep_build_csr(None, geom_of(det), mask)
    try:
        ex = B.sep_csr_export(csr)
        perm_inv = B.sep_csr_staging(csr)
    finally:
        B.sep_csr_destroy(csr)
    W = oracle.weights(det, mask)
    assert ex["range"] == W.range
    assert np.array_equal(ex["bin_of_pixel"], W.bin_of_pixel)
    rows = np.repeat(np.arange(det.nbins), np.diff(ex["rowptr"]))
    assert np.all(ex["rowptr"] % 4 == 0)
    pad = ex["col"] < 0
    assert np.all(ex["coef"][pad] == 0)
    nz = ex["coef"] != 0
    got = sorted(zip(ex["col"][nz].tolist(), rows[nz].tolist(), ex["coef"][nz].astype(np.float64).tolist()))
    want = sorted(zip(W.pix.tolist(), W.bin.tolist(), W.c.tolist()))
    assert got == want
    # staging order: a permutation of the pixels with entries, tiles in
    # row-major order, by centre bin inside a tile (then radius)
    used = np.unique(ex["col"][ex["col"] >= 0])
    assert np.array_equal(np.sort(perm_inv), used)
    r, cl = perm_inv // det.cols, perm_inv % det.cols
    th, tw = TILE
    tiles_x = (det.cols + tw - 1) // tw
    tile = (r // th) * tiles_x + cl // tw
    key = tile.astype(np.int64) * 100000 + W.bin_of_pixel[perm_inv]
    assert np.all(np.diff(key) >= 0)
    # inside a (tile, bin) group the radius grows
    yy, xx = r + 0.5 - det.center_px[1], cl + 0.5 - det.center_px[0]
    rad = np.hypot(yy, xx)
    same = np.diff(key) == 0
    assert np.all(np.diff(rad)[same] >= -1e-3)   # float32 keys: ties within a rounding
    pos_of = np.full(det.rows * det.cols, -1, np.int64)
    pos_of[perm_inv] = np.arange(perm_inv.size)
    # within a row: coefficient groups, largest first, staging positions ascending in a group
    for b in range(det.nbins):
        sl = slice(ex["rowptr"][b], ex["rowptr"][b + 1])
        c, k = ex["col"][sl], ex["coef"][sl]
        real = c >= 0
        kk = np.where(k[real] == 0, -1.0, k[real])
        assert np.all(np.diff(kk) <= 0)
        for val in np.unique(kk):
            assert np.all(np.diff(pos_of[c[real][kk == val]]) > 0)
    # zero-coefficient entries exist only to carry a pixel's centre bin
    zc, zr = ex["col"][~nz & ~pad], rows[~nz & ~pad]
    assert np.array_equal(W.bin_of_pixel[zc], zr)
    have = set(zip(W.pix.tolist(), W.bin.tolist()))
    assert all((int(p), int(b)) not in have for p, b in zip(zc, zr))
    valid = np.flatnonzero(W.bin_of_pixel >= 0)
    centre_pairs = set(zip(ex["col"].tolist(), rows.tolist()))
    assert all((int(i), int(W.bin_of_pixel[i])) in centre_pairs for i in valid[:: max(1, valid.size // 5000)])
    return ex


def test_csr_config1_equals_oracle():
    ex = compare_with_oracle(synth.det_config1())
    assert (ex["col"] >= 0).sum() == 65536 and ex["max_row"] > 0


@pytest.mark.parametrize("unit", [synth.UNIT_2TH_DEG, synth.UNIT_Q_NM, synth.UNIT_R_MM])
def test_csr_split2_equals_oracle(unit):
    det = synth.det_small_jf(split=2, nbins=150)
    det.unit = unit
    compare_with_oracle(det, det.mask())


def test_csr_centre_only_entries_near_beam_centre():
    # many narrow bins around a centre inside the image force pixels whose
    # centre bin holds none of their sub-pixels
    det = synth.Detector("c", 24, 24, dist_m=0.05, center_px=(12.0, 12.0), unit=synth.UNIT_R_MM, nbins=200, split=2)
    ex = compare_with_oracle(det)
    assert ((ex["coef"] == 0) & (ex["col"] >= 0)).sum() > 0


def test_csr_explicit_range_drops_outside():
    det = synth.det_config1()
    det.range = (1.0, 5.0)
    det.nbins = 20
    compare_with_oracle(det)


@pytest.mark.parametrize("case", ["config1", "jf_mask_split2", "r_mm_user_range", "exact"])
def test_interpolation_table_matches_the_oracle(case):
    """The host-built table of the smooth background (lower bin, binary32
    weight) equals the oracle's, bit for bit, in three units, with a mask,
    a user range that leaves pixels beyond the outer bin centres, and exact
    area fractions (whose automatic range spans the pixels' extents)."""
    mask = None
    if case == "config1":
        det = synth.det_config1()
    elif case == "jf_mask_split2":
        det = synth.det_small_jf(split=2, nbins=120, rows=300, cols=260)
        det.layout = None
        mask = np.zeros(det.npix, np.uint8)
        mask[::13] = 1
    elif case == "r_mm_user_range":
        det = synth.Detector("r", 60, 70, dist_m=0.05, center_px=(30.3, 25.7), nbins=25, split=1,
                             unit=synth.UNIT_R_MM, range=(0.5, 2.0))
    else:
        det = synth.Detector("x", 40, 44, dist_m=0.05, center_px=(20.3, 18.7), nbins=16, split=0,
                             unit=synth.UNIT_2TH_DEG)
    csr = B.sep_build_csr(None, geom_of(det), mask)
    try:
        a, t = B.sep_csr_interp(csr)
    finally:
        B.sep_csr_destroy(csr)
    W = oracle.weights_exact(det, mask) if det.split == 0 else oracle.weights(det, mask)
    oa, ot = oracle.interpolation(det, W)
    valid = W.bin_of_pixel >= 0
    assert np.array_equal(a[valid], oa[valid])
    assert np.array_equal(t[valid].view(np.uint32), np.asarray(ot, np.float32)[valid].view(np.uint32))
    assert np.all(a[~valid] == 0) and np.all(t[~valid] == 0)
    assert np.all((t >= 0) & (t < 1)) and np.all((a >= 0) & (a < det.nbins))
    lo, hi = W.range
    x = oracle.pixel_unit(det)
    u = (x - lo) / (hi - lo) * det.nbins - 0.5
    assert np.any(valid & (u <= 0)) or case != "r_mm_user_range"
    assert np.all(t[valid & ((u <= 0) | (u >= det.nbins - 1))] == 0)
