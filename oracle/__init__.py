"""CPU oracle for the signal-separation path (arXiv 2411.09515).

TEST INFRASTRUCTURE ONLY: the plain FP64 statement of what the GPU library
computes. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package. It shares no code with
``paper_2411_09515_gb300`` and never imports it.

The arithmetic of correction, coefficients, moments, clipping,
sparsification and peaks lives in ``sep_oracle.c`` (compiled to
``oracle/_build/liboracle.so``), for which this module marshals numpy
arrays; densification, the veto, the exact area fractions and the radial
interpolation (of the densified background and of the sparsification
threshold, fed to the C routines as one "bin" per pixel) are plain Python /
numpy statements here. Every function's
docstring names the passage of the paper it follows.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build_cmd():
    # -ffp-contract=off: no fused multiply-add anywhere (x86 and Arm alike);
    # no -ffast-math: IEEE semantics for the binary32 correction.
    return ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-ffp-contract=off", "-fno-fast-math",
            "-Wall", os.path.join(_HERE, "sep_oracle.c"), "-lm", "-o", _SO]


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    src = os.path.join(_HERE, "sep_oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.run(build_cmd(), check=True)
    return _SO


class Geom(C.Structure):
    _fields_ = [
        ("rows", C.c_int32), ("cols", C.c_int32),
        ("pixel_y", C.c_double), ("pixel_x", C.c_double),
        ("dist", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
        ("wavelength", C.c_double),
        ("unit", C.c_int32), ("nbins", C.c_int32), ("split", C.c_int32),
        ("lo", C.c_double), ("hi", C.c_double),
    ]


class Peak(C.Structure):
    _fields_ = [("idx", C.c_int32), ("y", C.c_double), ("x", C.c_double), ("I", C.c_double),
                ("sigma", C.c_double), ("npix", C.c_int32)]


PEAK_DTYPE = np.dtype([("idx", "<i4"), ("y", "<f8"), ("x", "<f8"), ("I", "<f8"), ("sigma", "<f8"),
                       ("npix", "<i4")], align=True)
assert PEAK_DTYPE.itemsize == C.sizeof(Peak)

vp = C.c_void_p


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(_SO):
            build()
        L = C.CDLL(_SO)
        L.oracle_jf_photons.argtypes = [C.c_int64, vp, vp, vp, C.c_int64, vp]
        L.oracle_jf_photons.restype = None
        L.oracle_unit_range.argtypes = [C.POINTER(Geom), vp, vp, vp]
        L.oracle_unit_range.restype = None
        L.oracle_weights.argtypes = [C.POINTER(Geom), vp, C.c_int64, vp, vp, vp, vp, vp]
        L.oracle_weights.restype = C.c_int64
        L.oracle_integrate_clip.argtypes = [C.c_int64, C.c_int64, vp, vp, vp, C.c_int32, vp, vp,
                                            C.c_int32, C.c_double, C.c_int32, C.c_int32, C.c_double,
                                            vp, vp, vp, vp, vp, vp]
        L.oracle_integrate_clip.restype = C.c_int
        L.oracle_pixel_unit.argtypes = [C.POINTER(Geom), vp]
        L.oracle_pixel_unit.restype = None
        L.oracle_moments_subset.argtypes = [C.c_int64, vp, vp, vp, vp, vp, C.c_int32, C.c_double, vp]
        L.oracle_moments_subset.restype = None
        L.oracle_sparsify.argtypes = [C.c_int64, vp, vp, vp, vp, vp, C.c_double, C.c_int64, vp, vp]
        L.oracle_sparsify.restype = C.c_int64
        L.oracle_peaks.argtypes = [C.c_int32, C.c_int32, vp, vp, vp, vp, vp, C.c_double, C.c_int32,
                                   C.c_int32, C.c_int64, vp]
        L.oracle_peaks.restype = C.c_int64
        L.oracle_process_frames.argtypes = [C.c_int32, C.c_int32, C.c_int64, vp, vp, vp, vp, C.c_int32,
                                            C.c_int32, C.c_int32, vp, vp, vp, vp, C.c_int32, C.c_double,
                                            C.c_double, C.c_int32, C.c_int32, vp, vp, vp, vp, C.c_int32]
        L.oracle_process_frames.restype = C.c_int
        L.oracle_max_threads.restype = C.c_int
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(vp)


def _c(a, dt):
    return None if a is None else np.ascontiguousarray(a, dtype=dt)


def geom_of(det) -> Geom:
    """Oracle geometry from a ``synth.Detector`` description."""
    lo, hi = det.range
    return Geom(det.rows, det.cols, det.pixel_m[0], det.pixel_m[1], det.dist_m, det.center_px[0],
                det.center_px[1], det.wavelength_m, det.unit, det.nbins, det.split, lo, hi)


def jf_photons(raw, ped, gain):
    """Detector correction of Section 1.2 (dark subtraction of Eq. 1 and the
    gain of the level in the raw word's top two bits), binary32."""
    raw = _c(raw, np.uint16).reshape(-1)
    n = raw.size
    ped = _c(ped, np.float32).reshape(3, -1)
    gain = _c(gain, np.float32).reshape(3, -1)
    assert ped.shape[1] == n and gain.shape[1] == n
    out = np.empty(n, np.float32)
    lib().oracle_jf_photons(n, _p(raw), _p(ped), _p(gain), n, _p(out))
    return out


def chauvenet_k(n):
    """Clip cut-off of Eq. 20 for a set of n entries: sqrt(2 ln(n / sqrt(2 pi)))
    (None for n <= 2, where the logarithm is not positive: no clipping)."""
    return math.sqrt(2.0 * math.log(n / math.sqrt(2.0 * math.pi))) if n > 2 else None


def unit_range(det, mask=None):
    g = geom_of(det)
    lo, hi = C.c_double(), C.c_double()
    lib().oracle_unit_range(C.byref(g), _p(_c(mask, np.uint8)), C.byref(lo), C.byref(hi))
    return lo.value, hi.value


class Weights:
    """Pixel-to-bin coefficients c_{i,r} of Section 2.2 (area fraction by
    s x s sub-pixel centres), pixel-major."""

    def __init__(self, pix, b, c, bin_of_pixel, rng, nbins, npix):
        self.pix, self.bin, self.c = pix, b, c
        self.bin_of_pixel, self.range, self.nbins, self.npix = bin_of_pixel, rng, nbins, npix


def _radius_of(det, x):
    """Detector-plane radius (m) of the radial value x in det's unit (the
    inverse of the radius -> 2theta / q / r mapping of the flat detector)."""
    x = float(x)
    if det.unit == 2:                                   # r in mm
        R = x * 1e-3
    else:
        if det.unit == 0:                               # 2theta in degrees
            tth = math.radians(x)
        else:                                           # q in nm^-1
            sarg = x * det.wavelength_m * 1e9 / (4 * math.pi)
            tth = math.pi if sarg >= 1 else 2 * math.asin(sarg)
        R = math.inf if tth >= math.pi / 2 else det.dist_m * math.tan(tth)
    return max(R, 0.0)


def _unit_of(det, R):
    if det.unit == 2:
        return R * 1e3
    tth = math.atan2(R, det.dist_m)
    if det.unit == 0:
        return tth * (180 / math.pi)
    return 4 * math.pi * math.sin(0.5 * tth) / (det.wavelength_m * 1e9)


def _rect_in_disc(x0, x1, y0, y1, R):
    """Area of [x0, x1] x [y0, y1] inside the disc of radius R about the
    origin: the integral over x of the chord of the rectangle's column inside
    the circle, split where the circle crosses the rectangle's top and bottom."""
    if R <= 0:
        return 0.0
    if math.isinf(R):
        return (x1 - x0) * (y1 - y0)
    a, b = max(x0, -R), min(x1, R)
    if a >= b:
        return 0.0

    def S(t):   # integral of sqrt(R^2 - u^2) from 0 to t
        t = min(max(t, -R), R)
        return 0.5 * (t * math.sqrt(max(R * R - t * t, 0.0)) + R * R * math.asin(t / R))

    cuts = [a, b]
    for y in (y0, y1):
        if abs(y) < R:
            u = math.sqrt(R * R - y * y)
            cuts += [u, -u]
    cuts = sorted(c for c in set(cuts) if a <= c <= b)
    area = 0.0
    for u, v in zip(cuts[:-1], cuts[1:]):
        m = 0.5 * (u + v)
        h = math.sqrt(max(R * R - m * m, 0.0))
        top_is_circle, bot_is_circle = h < y1, -h > y0
        top = h if top_is_circle else y1
        bot = -h if bot_is_circle else y0
        if top <= bot:
            continue
        seg = 0.0
        seg += (S(v) - S(u)) if top_is_circle else y1 * (v - u)
        seg -= -(S(v) - S(u)) if bot_is_circle else y0 * (v - u)
        area += seg
    return area


def weights_exact(det, mask=None) -> Weights:
    """c_{i,r} of Section 2.2 as the exact fraction of pixel i's area falling
    into radial bin r: the bin's edges (in det's unit) are circles on the
    detector plane, and c is the pixel's area between them over the pixel's
    area. The range is det.range, or (NaN) the span of the valid pixels'
    nearest and farthest points. The threshold bin of a pixel is the bin of
    its centre (clamped into the range). Plain Python, for small detectors."""
    rows, cols = det.rows, det.cols
    py, px = det.pixel_m
    cx, cy = det.center_px
    m = np.zeros(rows * cols, np.uint8) if mask is None else np.asarray(mask, np.uint8).reshape(-1)
    lo, hi = det.range

    def extent(r, c):
        x0, x1 = (c - cx) * px, (c + 1 - cx) * px
        y0, y1 = (r - cy) * py, (r + 1 - cy) * py
        nx = x0 if x0 > 0 else (x1 if x1 < 0 else 0.0)
        ny = y0 if y0 > 0 else (y1 if y1 < 0 else 0.0)
        fx, fy = max(abs(x0), abs(x1)), max(abs(y0), abs(y1))
        return (x0, x1, y0, y1), _unit_of(det, math.hypot(nx, ny)), _unit_of(det, math.hypot(fx, fy))

    if math.isnan(lo) or math.isnan(hi):
        ex = [extent(r, c)[1:] for r in range(rows) for c in range(cols) if not m[r * cols + c]]
        lo = min(e[0] for e in ex) if math.isnan(lo) else lo
        hi = max(e[1] for e in ex) if math.isnan(hi) else hi
    B = det.nbins
    edges_R = [_radius_of(det, lo + (hi - lo) * k / B) for k in range(B + 1)]
    pix, bins, cs = [], [], []
    for r in range(rows):
        for c in range(cols):
            i = r * cols + c
            if m[i]:
                continue
            (x0, x1, y0, y1), umin, umax = extent(r, c)
            if umax < lo or umin > hi:
                continue
            t0 = (max(umin, lo) - lo) / (hi - lo) * B
            t1 = (min(umax, hi) - lo) / (hi - lo) * B
            for b in range(max(int(math.floor(t0)), 0), min(int(math.floor(t1)), B - 1) + 1):
                f = (_rect_in_disc(x0, x1, y0, y1, edges_R[b + 1]) - _rect_in_disc(x0, x1, y0, y1, edges_R[b])) / (px * py)
                if f > 1e-12:
                    pix.append(i)
                    bins.append(b)
                    cs.append(min(f, 1.0))
    # threshold bins: the pixel centres' bins on the same range (the C oracle's radial values)
    import copy
    d1 = copy.copy(det)
    d1.split, d1.range = 1, (lo, hi)
    bop = weights(d1, mask).bin_of_pixel
    return Weights(np.asarray(pix, np.int32), np.asarray(bins, np.int32), np.asarray(cs, np.float64), bop, (lo, hi),
                   B, rows * cols)


def weights(det, mask=None) -> Weights:
    g = geom_of(det)
    m = _c(mask, np.uint8)
    npix = det.rows * det.cols
    cap = npix * det.split * det.split
    pix = np.empty(cap, np.int32)
    b = np.empty(cap, np.int32)
    c = np.empty(cap, np.float64)
    bop = np.empty(npix, np.int32)
    rng = np.empty(2, np.float64)
    n = lib().oracle_weights(C.byref(g), _p(m), cap, _p(pix), _p(b), _p(c), _p(bop), _p(rng))
    assert n <= cap
    return Weights(pix[:n].copy(), b[:n].copy(), c[:n].copy(), bop, (rng[0], rng[1]), det.nbins, npix)


ERROR_AZIMUTHAL, ERROR_POISSON, ERROR_HYBRID = 0, 1, 2


def integrate_clip(W: Weights, signal, norm=None, n_iter=5, k=3.0, want_keep=False, chauvenet=False,
                   model=ERROR_AZIMUTHAL, dark=0.0):
    """Integration (Eqs. 2, 8-13) and sigma-clipping (Eq. 19, Section 2.4) of one frame;
    with ``chauvenet`` the cut-off of every step is Eq. 20's for the size of the set;
    ``model``: the deviation that clips and is reported (Section 2.4.1: azimuthal
    Eq. 13, Poisson Eqs. 3-4 with dark variance ``dark``, or hybrid: azimuthal
    clipping, Poisson deviation of the final set).

    Returns dict(mean, sigma, count, iters, band[, keep]) per bin."""
    sig = _c(signal, np.float32).reshape(-1)
    nrm = _c(norm, np.float32)
    B = W.nbins
    out = {"mean": np.zeros(B), "sigma": np.zeros(B), "count": np.zeros(B, np.int32),
           "iters": np.zeros(B, np.int32), "band": np.zeros(B)}
    keep = np.zeros(W.pix.size, np.uint8) if want_keep else None
    rc = lib().oracle_integrate_clip(W.npix, W.pix.size, _p(W.pix), _p(W.bin), _p(W.c), B, _p(sig),
                                     _p(nrm), n_iter, k, int(bool(chauvenet)), int(model), float(dark),
                                     _p(out["mean"]), _p(out["sigma"]),
                                     _p(out["count"]), _p(out["iters"]), _p(out["band"]), _p(keep))
    assert rc == 0
    if want_keep:
        out["keep"] = keep
    return out


def moments_subset(pix, c, sel, signal, norm=None, model=ERROR_AZIMUTHAL, dark=0.0):
    """(mu, sigma, count) of an explicit set of entries (Eqs. 8-13; sigma of
    the error model, as integrate_clip reports it)."""
    pix = _c(pix, np.int32)
    c = _c(c, np.float64)
    sel = _c(sel, np.uint8)
    o = np.zeros(3)
    lib().oracle_moments_subset(pix.size, _p(pix), _p(c), _p(sel), _p(_c(signal, np.float32)),
                                _p(_c(norm, np.float32)), int(model), float(dark), _p(o))
    return o[0], o[1], int(o[2])


def per_pixel_background(W: Weights, mean, sigma, interp):
    """The background of every pixel as its own "bin": (bins, mean, sigma)
    with bins[i] = i for a pixel with a radial bin (-1 otherwise) and
    mean / sigma the per-bin profile interpolated in binary64 at the pixel
    centre's radial value (``interp`` = interpolation(det, W, exact=True)).
    Fed to the per-bin sparsification and peak routines it makes their
    threshold mu(x_i) + k_pick sigma(x_i) and their background mu(x_j)."""
    bop = np.asarray(W.bin_of_pixel)
    has = bop >= 0
    bins = np.where(has, np.arange(W.npix), -1).astype(np.int32)
    mu = np.zeros(W.npix)
    sd = np.zeros(W.npix)
    mu[has] = profile_at(interp, mean, W.nbins)[has]
    sd[has] = profile_at(interp, sigma, W.nbins)[has]
    return bins, mu, sd


def sparsify(W: Weights, signal, mean, sigma, k_pick=3.0, norm=None, interp=None):
    """Pixels above mu + k_pick sigma of their radial bin (Section 3),
    ascending; with ``interp`` (interpolation(det, W, exact=True)) the
    background at the pixel centre's radial value instead: the smooth
    profile of Section 3, interpolated between bin centres."""
    sig = _c(signal, np.float32).reshape(-1)
    bop = W.bin_of_pixel
    if interp is not None:
        bop, mean, sigma = per_pixel_background(W, mean, sigma, interp)
    bop = _c(bop, np.int32)
    mean = _c(mean, np.float64)
    sigma = _c(sigma, np.float64)
    nrm = _c(norm, np.float32)
    n = lib().oracle_sparsify(W.npix, _p(bop), _p(sig), _p(nrm), _p(mean), _p(sigma), k_pick, 0, None, None)
    idx = np.empty(n, np.int32)
    val = np.empty(n, np.float64)
    lib().oracle_sparsify(W.npix, _p(bop), _p(sig), _p(nrm), _p(mean), _p(sigma), k_pick, n, _p(idx), _p(val))
    return idx, val


def veto(n_peaks, min_peaks):
    """Section 4 ("Peak count as veto algorithm"): the frames kept are those
    with at least min_peaks peaks (fewer: discarded), in frame order."""
    return [f for f, n in enumerate(n_peaks) if n >= min_peaks]


def pixel_unit(det):
    """Radial value (det's unit) of every pixel centre, by the C oracle's
    binary64 sequence (radius, then 2theta / q / r)."""
    out = np.empty(det.rows * det.cols, np.float64)
    lib().oracle_pixel_unit(C.byref(geom_of(det)), _p(out))
    return out


def interpolation(det, W: Weights, exact=False):
    """Lower bin a and weight t (binary32; binary64 with ``exact``) of the
    linear interpolation of a per-bin profile at every pixel centre's radial
    value, between the two bin centres around it (lo + (b + 1/2)(hi - lo)/B);
    the end bins' levels beyond the outer centres."""
    lo, hi = W.range
    B = W.nbins
    u = (pixel_unit(det) - lo) / (hi - lo) * B - 0.5
    a = np.floor(u)
    t = u - a if exact else (u - a).astype(np.float32)
    low, high = ~(u > 0), u >= B - 1
    a = np.where(low, 0, np.where(high, B - 1, a)).astype(np.int64)
    t = np.where(low | high, t.dtype.type(0), t)
    return a, t


def profile_at(interp, profile, nbins):
    """A per-bin profile at every pixel centre, in binary64:
    (1 - t) p_a + t p_(a+1) (the upper term is 0 where a is the last bin,
    where t is 0 too)."""
    a, t = interp
    p = np.asarray(profile, np.float64)
    t = np.asarray(t, np.float64)
    upper = np.where(a + 1 < nbins, p[np.minimum(a + 1, nbins - 1)], 0.0)
    return (1.0 - t) * p[a] + t * upper


def densify(W: Weights, mean, sigma, idx, val, noise=None, fill=np.nan, interp=None):
    """Decompression of Section 3 ("Densification / Decompression"): the
    background of every pixel with a radial bin is its bin's mean level (with
    ``interp`` = interpolation(det, W): the smooth profile, (1 - t) m_a + t
    m_(a+1), each product and the sum rounded to binary32), with noise of the
    bin's (interpolated) deviation when standard normal deviates z are given
    (binary32, one rounding per operation: m + (s * z_i)); the pixels that were
    kept get their recorded values back; pixels without a bin get `fill`.
    Plain numpy statement (no arithmetic in the C library)."""
    bop = np.asarray(W.bin_of_pixel)
    out = np.full(W.npix, fill, np.float32)
    has = bop >= 0
    mean = np.asarray(mean, np.float32)
    sigma = None if sigma is None else np.asarray(sigma, np.float32)

    def level(p):
        if interp is None:
            return p[bop[has]]
        a, t = interp[0][has], interp[1][has]
        upper = np.where(a + 1 < W.nbins, p[np.minimum(a + 1, W.nbins - 1)], np.float32(0))
        return (np.float32(1) - t) * p[a] + t * upper      # binary32 throughout

    mu = level(mean)
    if noise is None:
        out[has] = mu
    else:
        z = np.asarray(noise, np.float32).reshape(-1)[has]
        out[has] = mu + level(sigma) * z   # float32 operands: each operation rounds to binary32
    idx = np.asarray(idx, np.int64)
    ok = (idx >= 0) & (idx < W.npix)
    out[idx[ok]] = np.asarray(val, np.float32)[ok]
    return out


def peaks(det, W: Weights, signal, mean, sigma, k_pick=3.0, patch=3, min_count=3, norm=None, interp=None):
    """Peak picking of Section 4 over the kept pixels; structured array.
    With ``interp`` the kept test and the background of the records use the
    profile interpolated at each pixel centre (as ``sparsify``)."""
    sig = _c(signal, np.float32).reshape(-1)
    bop = W.bin_of_pixel
    if interp is not None:
        bop, mean, sigma = per_pixel_background(W, mean, sigma, interp)
    bop = _c(bop, np.int32)
    mean = _c(mean, np.float64)
    sigma = _c(sigma, np.float64)
    nrm = _c(norm, np.float32)
    args = (det.rows, det.cols, _p(bop), _p(sig), _p(nrm), _p(mean), _p(sigma), k_pick, patch, min_count)
    n = lib().oracle_peaks(*args, 0, None)
    out = np.zeros(n, PEAK_DTYPE)
    lib().oracle_peaks(*args, n, _p(out))
    return out


def process_frames(det, W: Weights, frames, calib=None, norm=None, n_iter=5, k_clip=3.0, k_pick=3.0,
                   patch=3, min_count=3, threads=0):
    """Whole frames end to end: per-bin mean/sigma, kept count and peak count."""
    F = frames.shape[0]
    is_raw = frames.dtype == np.uint16
    fr = np.ascontiguousarray(frames)
    ped = gain = None
    if is_raw:
        ped = _c(calib[0], np.float32)
        gain = _c(calib[1], np.float32)
    mean = np.zeros((F, W.nbins))
    sigma = np.zeros((F, W.nbins))
    nk = np.zeros(F, np.int32)
    npk = np.zeros(F, np.int32)
    rc = lib().oracle_process_frames(det.rows, det.cols, W.pix.size, _p(W.pix), _p(W.bin), _p(W.c),
                                     _p(W.bin_of_pixel), W.nbins, F, int(is_raw), _p(fr), _p(ped), _p(gain),
                                     _p(_c(norm, np.float32)), n_iter, k_clip, k_pick, patch, min_count,
                                     _p(mean), _p(sigma), _p(nk), _p(npk), threads)
    assert rc == 0
    return mean, sigma, nk, npk


def max_threads() -> int:
    return lib().oracle_max_threads()
