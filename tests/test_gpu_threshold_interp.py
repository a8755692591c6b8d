"""Sparsification and peak picking against the background interpolated at
each pixel centre (Section 3's smooth profile; sep_params.interpolate = 1),
GPU through the C ABI against the oracle: float frames of the 256 x 256
detector with and without a norm, raw Jungfrau-shaped frames with 2 x 2
splitting and a mask; the standalone calls and the allocation-free
sparsification equal the batch bit for bit; a mixed batch equals its
detectors' own batches."""
import numpy as np
import pytest

import oracle
import synth
from parity import check_frame

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2411_09515_gb300 import Context, Separator, _binding as B, process_mixed  # noqa: E402


def _batch(sep, frames_np, kcap, pcap, use_graph=True):
    if frames_np.dtype == np.uint16:
        frames_np = frames_np.view(np.int16)
    fr = torch.from_numpy(np.ascontiguousarray(frames_np)).cuda()
    out = sep.process_batch(fr, kcap, pcap, use_graph=use_graph)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}, fr


@pytest.mark.parametrize("with_norm", [False, True])
def test_config1_interpolated_thresholds(with_norm):
    det = synth.det_config1()
    W = oracle.weights(det)
    interp = oracle.interpolation(det, W, exact=True)
    norm = np.random.default_rng(6).uniform(0.5, 2.0, det.npix).astype(np.float32) if with_norm else None
    fr = np.concatenate([synth.frames(det, synth.spec_config1(s), 0, 1)[0] for s in range(4)]).astype(np.float32)
    if with_norm:
        fr = (fr * norm).astype(np.float32)
    sep = Separator.from_detector(det, norm=norm)
    sep.set_params(interpolate=1)
    o, dfr = _batch(sep, fr, 8192, 512)
    bnd = sep.integrate_clip(dfr, bounds=True)["bounds"].cpu().numpy()
    for f in range(fr.shape[0]):
        check_frame(det, W, fr[f], o, f, kcap=8192, bounds=bnd[f], norm=norm, interp=interp)
    assert sep.device_status() == 0
    # the per-bin reading keeps other pixels on these frames
    sep.set_params(interpolate=0)
    o0, _ = _batch(sep, fr, 8192, 512)
    assert any(int(o0["n_kept"][f]) != int(o["n_kept"][f]) or
               not np.array_equal(o0["idx"][f, :o0["n_kept"][f]], o["idx"][f, :o["n_kept"][f]])
               for f in range(fr.shape[0]))


def test_jungfrau_raw_split_interpolated_thresholds():
    det = synth.det_small_jf(split=2, nbins=300)
    mask = det.mask()
    cal = synth.jf_calib(det.npix, seed=7)
    spec = synth.spec_jf_serial(11)
    spec.hit_rate = 0.5
    fr = synth.frames(det, spec, 0, 4, calib=cal, mask=mask)[0]
    W = oracle.weights(det, mask)
    interp = oracle.interpolation(det, W, exact=True)
    sep = Separator.from_detector(det, mask=mask, calib=cal)
    sep.set_params(interpolate=1)
    kcap = det.npix // 4
    o, dfr = _batch(sep, fr, kcap, 20000)
    bnd = sep.integrate_clip(dfr, bounds=True)["bounds"].cpu().numpy()
    for f in range(fr.shape[0]):
        sig = oracle.jf_photons(fr[f], cal[0], cal[1])
        check_frame(det, W, sig, o, f, kcap=kcap, bounds=bnd[f], interp=interp)
    assert sep.device_status() == 0


@pytest.mark.parametrize("raw", [False, True])
def test_standalone_calls_equal_the_batch(raw):
    if raw:
        det = synth.det_small_jf(split=2, nbins=200)
        mask = det.mask()
        cal = synth.jf_calib(det.npix, seed=3)
        spec = synth.spec_jf_serial(5)
        spec.hit_rate = 1.0
        fr = synth.frames(det, spec, 0, 3, calib=cal, mask=mask)[0]
        sep = Separator.from_detector(det, mask=mask, calib=cal)
    else:
        det = synth.det_config1()
        fr = np.concatenate([synth.frames(det, synth.spec_config1(s), 0, 1)[0] for s in (1, 2, 3)])
        sep = Separator.from_detector(det)
    sep.set_params(interpolate=1)
    kcap, pcap = det.npix // 8, 4000
    o, dfr = _batch(sep, fr, kcap, pcap, use_graph=False)
    ic = sep.integrate_clip(dfr)
    sp = sep.sparsify(dfr, ic["mean"], ic["sigma"], kcap)
    pk = sep.peakfind(dfr, ic["mean"], ic["sigma"], sp["idx"], sp["n_kept"], pcap)
    F = fr.shape[0]
    idx = torch.full((F, kcap), -7, dtype=torch.int32, device="cuda")
    val = torch.full((F, kcap), -7.0, dtype=torch.float32, device="cuda")
    nk = torch.full((F,), -7, dtype=torch.int32, device="cuda")
    B.sep_sparsify_noalloc(sep.ctx, sep.csr, sep.calib, dfr, sep._dtype(dfr), F, sep.params, ic["mean"],
                           ic["sigma"], idx, val, kcap, nk)
    torch.cuda.synchronize()
    # the same profiles and the same binary32 values: identical thresholds
    assert np.array_equal(ic["mean"].cpu().numpy(), o["mean"])
    for f in range(F):
        n = int(o["n_kept"][f])
        assert int(sp["n_kept"][f]) == n and int(nk[f]) == n
        for got_i, got_v in ((sp["idx"], sp["val"]), (idx, val)):
            assert np.array_equal(got_i[f, :n].cpu().numpy(), o["idx"][f, :n])
            assert np.array_equal(got_v[f, :n].cpu().numpy(), o["val"][f, :n])
        npk = int(o["n_peaks"][f])
        assert int(pk["n_peaks"][f]) == npk
        assert np.array_equal(pk["peaks"][f, :npk].cpu().numpy(), o["peaks"][f, :npk])
    assert sep.device_status() == 0


def test_mixed_batch_equals_per_detector_batches():
    ctx = Context(0)
    dets = [synth.det_config1(), synth.det_small_jf(split=2, nbins=150)]
    seps = [Separator.from_detector(d, mask=d.mask() if d.layout else None, context=ctx) for d in dets]
    for s in seps:
        s.set_params(interpolate=1)
    pattern = [0, 1, 0, 1, 1, 0]
    frames, per_det = [], {0: [], 1: []}
    for g, d in enumerate(pattern):
        spec = synth.spec_mixed(seed=70 + g, hit_rate=0.5) if d == 1 else synth.spec_config1(70 + g)
        fr = synth.frames(dets[d], spec, g, 1, mask=dets[d].mask() if dets[d].layout else None)[0]
        frames.append((d, torch.from_numpy(fr[0]).cuda()))
        per_det[d].append((g, fr[0]))
    kcap, pcap = 60000, 4000
    for use_graph in (True, False):
        out = process_mixed(seps, frames, kcap, pcap, use_graph=use_graph)
        torch.cuda.synchronize()
        rows = out["row_off"]
        for d, lst in per_det.items():
            batch = torch.from_numpy(np.stack([f for _, f in lst])).cuda()
            ref = seps[d].process_batch(batch, kcap, pcap, use_graph=False)
            torch.cuda.synchronize()
            for j, (g, _) in enumerate(lst):
                r0, r1 = rows[g], rows[g + 1]
                assert np.array_equal(out["mean"][r0:r1].cpu().numpy(), ref["mean"][j].cpu().numpy())
                nk = int(ref["n_kept"][j])
                assert int(out["n_kept"][g]) == nk
                assert np.array_equal(out["idx"][g, :nk].cpu().numpy(), ref["idx"][j, :nk].cpu().numpy())
                npk = int(ref["n_peaks"][j])
                assert int(out["n_peaks"][g]) == npk
                assert np.array_equal(out["peaks"][g, :npk].cpu().numpy(), ref["peaks"][j, :npk].cpu().numpy())
    assert seps[0].device_status() == 0
    for s in seps:
        s.close()
    ctx.close()


def test_interpolate_flag_is_validated():
    det = synth.det_config1()
    sep = Separator.from_detector(det)
    d = torch.zeros((1, det.npix), dtype=torch.float32, device="cuda")
    sep.set_params(interpolate=2)
    with pytest.raises(Exception):
        sep.process_batch(d, 16, 16)
