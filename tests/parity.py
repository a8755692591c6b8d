"""GPU-vs-oracle comparison rules shared by the GPU tests.

Tolerances: per-bin mean and deviation within a relative 1e-5 (absolute
1e-6 * max(1, |mean|) when the deviation is 0); kept pixels and peak lists
identical except for pixels whose value lies within a relative 1e-5 of their
threshold; peak centroid and intensity within a relative 1e-4.

A local maximum between two pixels whose values are equal up to one FP32
rounding of signal / norm may be either pixel (the library compares the FP32
values, the oracle the FP64 quotients).

With thresholds interpolated between bin centres (``interp``, the oracle's
binary64 interpolation table) every pixel has its own threshold; the same
band applies to it.

A clip decision taken within a relative 1e-5 of a boundary ("banded" bin in
the oracle's log) may legitimately go either way in FP32 on the GPU and then
change the rest of that bin's trajectory. For such bins the GPU's own final
set (the interval [L, H] it reports) is re-evaluated in FP64 by the oracle
and the GPU's mean, deviation and count must match that.
"""
from __future__ import annotations

import numpy as np

import oracle

BAND = 1e-5
RTOL = 1e-5
PEAK_RTOL = 1e-4


# absolute floor of the mean's tolerance, in deviations: one FP32 rounding of
# the bin's spread. A mean near zero against its spread (|mu| ~ 1e-4 sigma)
# has no relative precision when the per-lane sums are plain FP32 (PLAIN,
# DWORD and FP64MERGE accumulate each lane's share in FP32 before their
# merge: the Chauvenet parity test meets such a bin, mean error 7.5e-9 sigma
# = 1.5e-5 relative in DWORD). KAHAN compensates the per-lane sums and is
# held to the relative tolerance alone (floor 0).
MEAN_FLOOR = 1e-7


def close(a, b, rtol=RTOL, sd=None, floor=MEAN_FLOOR):
    """|a - b| <= rtol |b|; where the bin's deviation sd is 0 the bound is
    1e-6 max(1, |b|); with a deviation, floor * sd is added (MEAN_FLOOR
    except for the KAHAN mode, see above)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    tol = rtol * np.abs(b)
    if sd is not None:
        sd = np.asarray(sd, np.float64)
        tol = np.where(sd == 0, 1e-6 * np.maximum(1.0, np.abs(b)), tol + floor * sd)
    return np.abs(a - b) <= tol + 1e-30


class Frame:
    """Oracle view of one frame: values, clip results, thresholds."""

    def __init__(self, W, signal, n_iter, k_clip, k_pick, norm=None, chauvenet=False, model=0, dark=0.0,
                 interp=None):
        self.W = W
        self.interp = interp
        self.model, self.dark = model, dark
        self.sig = np.ascontiguousarray(signal, np.float32).reshape(-1)
        self.norm = norm
        self.v = self.sig.astype(np.float64) / (1.0 if norm is None else norm.astype(np.float64))
        self.k_clip, self.k_pick, self.n_iter = k_clip, k_pick, n_iter
        self.ref = oracle.integrate_clip(W, self.sig, norm=norm, n_iter=n_iter, k=k_clip, chauvenet=chauvenet,
                                         model=model, dark=dark)
        self.order = np.argsort(W.bin, kind="stable")
        self.start = np.searchsorted(W.bin[self.order], np.arange(W.nbins + 1))

    def entries(self, b):
        e = self.order[self.start[b]:self.start[b + 1]]
        return self.W.pix[e], self.W.c[e]


def check_clip(fr: Frame, mean, sigma, count, bounds, floor=MEAN_FLOOR):
    """Returns (number of banded bins, list of bins whose GPU stats come from a
    different trajectory). Raises AssertionError on a mismatch. floor: the
    absolute floor of the mean's tolerance in deviations (see close)."""
    ref = fr.ref
    banded = ref["band"] < BAND
    ok = close(mean, ref["mean"], sd=ref["sigma"], floor=floor) & close(sigma, ref["sigma"], sd=ref["sigma"]) & \
        (count == ref["count"])
    bad = np.flatnonzero(~ok & ~banded)
    assert bad.size == 0, (f"{bad.size} unbanded bins differ, e.g. bin {bad[0]}: gpu "
                           f"({mean[bad[0]]}, {sigma[bad[0]]}, {count[bad[0]]}) oracle "
                           f"({ref['mean'][bad[0]]}, {ref['sigma'][bad[0]]}, {ref['count'][bad[0]]}) "
                           f"band {ref['band'][bad[0]]}")
    moved = []
    for b in np.flatnonzero(~ok & banded):
        pix, c = fr.entries(b)
        L, H = bounds[b]
        vv = fr.sig[pix]
        sel = (vv >= L) & (vv <= H)
        mu, sd, n = oracle.moments_subset(pix, c, sel.astype(np.uint8), fr.sig, fr.norm, model=fr.model, dark=fr.dark)
        assert close(mean[b], mu, sd=np.array(sd), floor=floor) and close(sigma[b], sd, sd=np.array(sd)) and \
            count[b] == n, (b, mean[b], mu, sigma[b], sd, count[b], n)
        moved.append((b, mu, sd))
    return int(banded.sum()), moved


def thresholds(fr: Frame, moved):
    """Per-pixel thresholds from the oracle's profile, and from the profile
    with the bins of another trajectory replaced by the GPU's own sets."""
    mean, sigma = fr.ref["mean"], fr.ref["sigma"]
    mean_alt, sigma_alt = mean.copy(), sigma.copy()
    for b, mu, sd in moved:
        mean_alt[b], sigma_alt[b] = mu, sd
    bop = fr.W.bin_of_pixel
    b = np.where(bop >= 0, bop, 0)
    if fr.interp is None:
        return (mean + fr.k_pick * sigma)[b], (mean_alt + fr.k_pick * sigma_alt)[b]
    nb = fr.W.nbins
    at = oracle.profile_at
    return (at(fr.interp, mean, nb) + fr.k_pick * at(fr.interp, sigma, nb),
            at(fr.interp, mean_alt, nb) + fr.k_pick * at(fr.interp, sigma_alt, nb))


def check_kept(fr: Frame, idx, val, n_kept, moved, capacity=None):
    """Kept pixels (ascending) against the oracle's; returns the set of excused pixels."""
    bop = fr.W.bin_of_pixel
    thr, thr_alt = thresholds(fr, moved)
    valid = bop >= 0
    v = fr.v
    want = np.flatnonzero(valid & (v > thr))
    want_alt = np.flatnonzero(valid & (v > thr_alt))
    n = int(n_kept)
    got = np.asarray(idx[: min(n, capacity if capacity is not None else n)])
    assert np.all(np.diff(got) > 0), "kept pixels not ascending"
    # values are the corrected pixel values, bit for bit
    want_val = fr.sig[got] if fr.norm is None else fr.sig[got] / fr.norm[got].astype(np.float32)
    assert np.array_equal(np.asarray(val[: got.size], np.float32), want_val.astype(np.float32))
    diff = np.setxor1d(got, want)
    near = np.abs(v[diff] - thr[diff]) <= BAND * np.abs(thr[diff])
    alt = np.isin(diff, want_alt) == np.isin(diff, got)
    excused = near | alt
    assert np.all(excused), (f"{(~excused).sum()} kept pixels differ beyond the band, e.g. pixel "
                             f"{diff[~excused][0]} v={v[diff[~excused][0]]} thr={thr[diff[~excused][0]]}")
    if capacity is None or n <= capacity:
        assert abs(n - want.size) <= diff.size
    return set(diff.tolist())


def check_peaks(det, fr: Frame, peaks, excused, patch=3, min_count=3, truncated=False):
    """Peak list against the oracle's, computed on the oracle's thresholds
    (truncated: the list filled its capacity, so it is compared up to its
    last pixel)."""
    ref = oracle.peaks(det, fr.W, fr.sig, fr.ref["mean"], fr.ref["sigma"], k_pick=fr.k_pick, patch=patch,
                       min_count=min_count, norm=fr.norm, interp=fr.interp)
    if truncated and len(peaks):
        ref = ref[ref["idx"] <= peaks["idx"][-1]]
    cols = det.cols
    h = patch // 2

    def touches(i):
        r0, c0 = divmod(int(i), cols)
        for r in range(r0 - h, r0 + h + 1):
            for c in range(c0 - h, c0 + h + 1):
                if 0 <= r < det.rows and 0 <= c < cols and (r * cols + c) in excused:
                    return True
        return False

    def near_tie(i):
        # with a norm, the local maximum between two values equal up to one
        # binary32 rounding of signal / norm (Eq. 1) may go either way: the
        # library compares the binary32 values, the oracle the FP64 quotients.
        # Without a norm both compare the same binary32 values: no excuse.
        if fr.norm is None:
            return False
        r0, c0 = divmod(int(i), cols)
        vi = fr.v[i]
        for r in range(r0 - h, r0 + h + 1):
            for c in range(c0 - h, c0 + h + 1):
                j = r * cols + c
                if (0 <= r < det.rows and 0 <= c < cols and j != i and fr.W.bin_of_pixel[j] >= 0
                        and abs(fr.v[j] - vi) <= 2.0 ** -23 * max(abs(vi), abs(fr.v[j]))):
                    return True
        return False

    gi = peaks["idx"].astype(np.int64)
    ri = ref["idx"].astype(np.int64)
    for i in np.setxor1d(gi, ri):
        assert touches(i) or near_tie(i), f"peak at pixel {i} differs and no excused pixel is in its patch"
    common, ia, ib = np.intersect1d(gi, ri, return_indices=True)
    g, r = peaks[ia], ref[ib]
    clean = np.array([not touches(i) for i in common], bool)
    g, r = g[clean], r[clean]
    assert np.array_equal(g["npix"], r["npix"])
    for k in ("y", "x", "I", "sigma"):
        assert np.all(close(g[k], r[k], rtol=PEAK_RTOL)), (k, g[k][:5], r[k][:5])
    return ref.size, int(clean.sum())


def check_frame(det, W, sig, o, f, n_iter=5, k_clip=3.0, k_pick=3.0, kcap=None, bounds=None, norm=None,
                chauvenet=False, model=0, dark=0.0, interp=None, floor=MEAN_FLOOR):
    """Frame f of a batch's outputs `o` (numpy arrays as returned by the
    library) against the oracle on the frame's signal. Returns (banded bins,
    bins on another trajectory, excused pixels)."""
    fr = Frame(W, sig, n_iter, k_clip, k_pick, norm=norm, chauvenet=chauvenet, model=model, dark=dark,
               interp=interp)
    if bounds is None:
        bounds = np.tile(np.array([-np.inf, np.inf], np.float32), (W.nbins, 1))
    nb, moved = check_clip(fr, o["mean"][f], o["sigma"][f], o["count"][f], bounds, floor=floor)
    excused = check_kept(fr, o["idx"][f], o["val"][f], o["n_kept"][f], moved, capacity=kcap)
    pcap = o["peaks"].shape[1]
    peaks = o["peaks"][f][: int(o["n_peaks"][f])].copy().view(np.dtype([("idx", "<i4"), ("y", "<f4"), ("x", "<f4"),
                                                                      ("I", "<f4"), ("sigma", "<f4"),
                                                                      ("npix", "<i4")])).reshape(-1)
    check_peaks(det, fr, peaks, excused, truncated=int(o["n_peaks"][f]) > pcap)
    return nb, len(moved), len(excused)
