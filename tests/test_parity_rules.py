"""The GPU-vs-oracle comparison rules themselves (tests/parity.py), on the
CPU: the oracle's own outputs, laid out as the library returns them, pass
them, for thresholds per bin and interpolated between bin centres; a kept
pixel dropped far from its threshold fails them; and the rules tell the two
threshold readings apart on a frame where they keep different pixels."""
import numpy as np
import pytest

import oracle
import synth
from parity import check_frame

PEAK_FIELDS = np.dtype([("idx", "<i4"), ("y", "<f4"), ("x", "<f4"), ("I", "<f4"), ("sigma", "<f4"), ("npix", "<i4")])


def _outputs(det, W, frames, interp=None, kcap=8192, pcap=512):
    """Oracle results in the library's output layout (float32 profiles,
    kept lists padded to kcap, 24-byte peak records padded to pcap)."""
    F = len(frames)
    o = {"mean": np.zeros((F, W.nbins), np.float32), "sigma": np.zeros((F, W.nbins), np.float32),
         "count": np.zeros((F, W.nbins), np.int32), "idx": np.full((F, kcap), -1, np.int32),
         "val": np.zeros((F, kcap), np.float32), "n_kept": np.zeros(F, np.int32),
         "peaks": np.zeros((F, pcap, 6), np.int32), "n_peaks": np.zeros(F, np.int32)}
    for f, sig in enumerate(frames):
        ref = oracle.integrate_clip(W, sig)
        o["mean"][f], o["sigma"][f], o["count"][f] = ref["mean"], ref["sigma"], ref["count"]
        idx, val = oracle.sparsify(W, sig, ref["mean"], ref["sigma"], 3.0, interp=interp)
        o["idx"][f, :idx.size], o["val"][f, :idx.size], o["n_kept"][f] = idx, val, idx.size
        pk = oracle.peaks(det, W, sig, ref["mean"], ref["sigma"], interp=interp)
        rec = np.zeros(pk.size, PEAK_FIELDS)
        for k in PEAK_FIELDS.names:
            rec[k] = pk[k]
        o["peaks"][f, :pk.size] = rec.view(np.int32).reshape(-1, 6)
        o["n_peaks"][f] = pk.size
    return o


@pytest.fixture(scope="module")
def config1():
    det = synth.det_config1()
    W = oracle.weights(det)
    frames = [synth.frames(det, synth.spec_config1(s), 0, 1)[0][0].astype(np.float32) for s in (0, 1)]
    return det, W, frames, oracle.interpolation(det, W, exact=True)


@pytest.mark.parametrize("use_interp", [False, True])
def test_oracle_outputs_pass_the_rules(config1, use_interp):
    det, W, frames, interp = config1
    ip = interp if use_interp else None
    o = _outputs(det, W, frames, interp=ip)
    for f, sig in enumerate(frames):
        check_frame(det, W, sig, o, f, kcap=8192, interp=ip)


def test_a_dropped_kept_pixel_fails(config1):
    det, W, frames, interp = config1
    o = _outputs(det, W, frames[:1])
    n = int(o["n_kept"][0])
    ref = oracle.integrate_clip(W, frames[0])
    thr = (ref["mean"] + 3.0 * ref["sigma"])[W.bin_of_pixel]
    idx = o["idx"][0, :n]
    far = np.argmax(frames[0][idx] - thr[idx])                # the kept pixel farthest above its threshold
    o["idx"][0, far:n - 1] = o["idx"][0, far + 1:n].copy()
    o["val"][0, far:n - 1] = o["val"][0, far + 1:n].copy()
    o["n_kept"][0] = n - 1
    with pytest.raises(AssertionError):
        check_frame(det, W, frames[0], o, 0, kcap=8192)


def test_the_rules_separate_the_two_threshold_readings(config1):
    det, W, frames, interp = config1
    o = _outputs(det, W, frames[:1], interp=interp)
    with pytest.raises(AssertionError):
        check_frame(det, W, frames[0], o, 0, kcap=8192)


def test_rules_on_masked_split_raw_frames():
    """The same on two raw Jungfrau-shaped frames with a mask and 2 x 2
    splitting, interpolated thresholds."""
    det = synth.det_small_jf(split=2, nbins=300)
    mask = det.mask()
    cal = synth.jf_calib(det.npix, seed=7)
    spec = synth.spec_jf_serial(11)
    spec.hit_rate = 0.5
    fr = synth.frames(det, spec, 0, 2, calib=cal, mask=mask)[0]
    W = oracle.weights(det, mask)
    ip = oracle.interpolation(det, W, exact=True)
    sigs = [oracle.jf_photons(fr[f], cal[0], cal[1]) for f in range(2)]
    kcap = det.npix // 4
    o = _outputs(det, W, sigs, interp=ip, kcap=kcap, pcap=20000)
    for f in range(2):
        check_frame(det, W, sigs[f], o, f, kcap=kcap, interp=ip)


def test_band_covers_a_binary32_interpolated_threshold(config1):
    """The arithmetic the header states for interpolated thresholds (binary32
    profile at the pixel from binary32 levels and weight, the sum rounded
    down to binary32), evaluated here in numpy on the oracle's levels, keeps
    a set the rules accept against the oracle's binary64 thresholds."""
    det, W, frames, interp = config1
    a, t = oracle.interpolation(det, W)                       # the library's binary32 table
    B = W.nbins
    for sig in frames:
        o = _outputs(det, W, [sig], interp=interp)
        m32, s32 = o["mean"][0], o["sigma"][0]

        def prof(p):
            up = np.where(a + 1 < B, p[np.minimum(a + 1, B - 1)], np.float32(0))
            return (np.float32(1) - t) * p[a] + t * up           # binary32 operations

        exact = prof(m32).astype(np.float64) + 3.0 * prof(s32).astype(np.float64)
        thr = exact.astype(np.float32)
        above = thr.astype(np.float64) > exact
        thr[above] = np.nextafter(thr[above], np.float32(-np.inf))
        idx = np.flatnonzero((W.bin_of_pixel >= 0) & (sig > thr)).astype(np.int32)
        o["idx"][0, :] = -1
        o["idx"][0, :idx.size], o["val"][0, :idx.size], o["n_kept"][0] = idx, sig[idx], idx.size
        check_frame(det, W, sig, o, 0, kcap=8192, interp=interp)
