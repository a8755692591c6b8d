"""GPU path against the CPU oracle, element by element, through the C ABI.

Sizes: the 256 x 256 frame (ten seeds), a two-module Jungfrau-shaped detector
with raw words and 2 x 2 splitting (several hundred bins, a ragged last
tile), and the exhaustive correction table; edge cases below."""
import numpy as np
import pytest

import oracle
import synth
from parity import MEAN_FLOOR, Frame, check_clip, check_frame, check_kept, check_peaks

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2411_09515_gb300 import (SEP_CUTOFF_CHAUVENET, SEP_ERROR_HYBRID, SEP_ERROR_POISSON,  # noqa: E402
                                    SEP_PREC_DWORD, SEP_PREC_FP64MERGE, SEP_PREC_KAHAN, SEP_PREC_PLAIN, SepError,
                                    Separator, peaks_to_numpy)


def run_batch(sep, frames_np, kcap, pcap, use_graph=True):
    if frames_np.dtype == np.uint16:
        frames_np = frames_np.view(np.int16)   # raw words travel as 16-bit integers
    fr = torch.from_numpy(np.ascontiguousarray(frames_np)).cuda()
    out = sep.process_batch(fr, kcap, pcap, use_graph=use_graph)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}, fr


def test_config1_ten_seeds_batch():
    det = synth.det_config1()
    W = oracle.weights(det)
    fr = np.concatenate([synth.frames(det, synth.spec_config1(s), 0, 1)[0] for s in range(10)])
    sep = Separator.from_detector(det)
    o, dfr = run_batch(sep, fr, 8192, 512)
    # the bounds of the final sets come from the standalone call (same kernel)
    ic = sep.integrate_clip(dfr, bounds=True, iters=True)
    torch.cuda.synchronize()
    assert np.array_equal(ic["mean"].cpu().numpy(), o["mean"])
    assert np.array_equal(ic["count"].cpu().numpy(), o["count"])
    bnd = ic["bounds"].cpu().numpy()
    for f in range(10):
        check_frame(det, W, fr[f], o, f, kcap=8192, bounds=bnd[f])
    assert sep.device_status() == 0
    assert (o["n_peaks"] >= 11).all()


def test_standalone_calls_equal_the_batch():
    det = synth.det_config1()
    fr = np.concatenate([synth.frames(det, synth.spec_config1(s), 0, 1)[0] for s in range(3)])
    sep = Separator.from_detector(det)
    o, dfr = run_batch(sep, fr, 8192, 512, use_graph=False)
    ic = sep.integrate_clip(dfr)
    sp = sep.sparsify(dfr, ic["mean"], ic["sigma"], 8192)
    pk = sep.peakfind(dfr, ic["mean"], ic["sigma"], sp["idx"], sp["n_kept"], 512)
    torch.cuda.synchronize()
    assert np.array_equal(ic["mean"].cpu().numpy(), o["mean"])
    assert np.array_equal(ic["sigma"].cpu().numpy(), o["sigma"])
    # the standalone sparsify takes float32 profiles: its thresholds may differ
    # from the fused ones (rounded from the extended mean) by a rounding of
    # the mean, hence only at pixels within the band of their threshold
    W = oracle.weights(det)
    bop = W.bin_of_pixel
    mean, sigma = o["mean"], o["sigma"]
    sidx, snk = sp["idx"].cpu().numpy(), sp["n_kept"].cpu().numpy()
    pks = pk["peaks"].cpu().numpy()
    npk = pk["n_peaks"].cpu().numpy()
    for f in range(3):
        a = o["idx"][f][: o["n_kept"][f]]
        b = sidx[f][: snk[f]]
        diff = np.setxor1d(a, b)
        v = fr[f].reshape(-1).astype(np.float64)
        thr = (mean[f] + 3.0 * sigma[f]).astype(np.float64)[bop[diff]]
        assert np.all(np.abs(v[diff] - thr) <= 1e-5 * np.abs(thr)), (f, diff)
        # peaks differ only where a differing kept pixel lies in the patch
        ga = peaks_to_numpy(torch.from_numpy(o["peaks"][f]), o["n_peaks"][f])["idx"]
        gb = peaks_to_numpy(torch.from_numpy(pks[f]), npk[f])["idx"]
        near = set()
        for i in diff:
            r0, c0 = divmod(int(i), det.cols)
            near.update((r0 + dr) * det.cols + c0 + dc for dr in (-1, 0, 1) for dc in (-1, 0, 1))
        for i in np.setxor1d(ga, gb):
            assert int(i) in near, (f, i)


def test_graph_replay_is_deterministic():
    det = synth.det_config1()
    fr = synth.frames(det, synth.spec_config1(4), 0, 2)[0]
    sep = Separator.from_detector(det)
    d = torch.from_numpy(fr).cuda()
    out = sep.alloc_outputs(2, 4096, 256)
    res = []
    for _ in range(3):
        sep.process_batch(d, 4096, 256, out=out, use_graph=True)
        torch.cuda.synchronize()
        res.append({k: v.cpu().numpy().copy() for k, v in out.items()})
    for k in res[0]:
        assert np.array_equal(res[0][k], res[1][k]) and np.array_equal(res[0][k], res[2][k]), k


@pytest.fixture(scope="module")
def jf_small():
    det = synth.det_small_jf(split=2, nbins=300)
    mask = det.mask()
    cal = synth.jf_calib(det.npix, seed=7)
    spec = synth.spec_jf_serial(11)
    spec.hit_rate = 0.5
    fr, _, _ = synth.frames(det, spec, 0, 6, calib=cal, mask=mask)
    W = oracle.weights(det, mask)
    return det, mask, cal, fr, W


# the compensated mode (KAHAN) meets the relative tolerance without the
# mean's absolute floor; the modes with plain FP32 per-lane sums keep it
@pytest.mark.parametrize("precision,floor", [(SEP_PREC_DWORD, MEAN_FLOOR), (SEP_PREC_FP64MERGE, MEAN_FLOOR),
                                             (SEP_PREC_KAHAN, 0.0), (SEP_PREC_PLAIN, MEAN_FLOOR)])
def test_jungfrau_raw_split_parity(jf_small, precision, floor):
    det, mask, cal, fr, W = jf_small
    sep = Separator.from_detector(det, mask=mask, calib=cal, precision=precision)
    kcap = det.npix // 4
    o, dfr = run_batch(sep, fr, kcap, 20000)
    bnd = sep.integrate_clip(dfr, bounds=True)["bounds"].cpu().numpy()
    tot_band = 0
    for f in range(fr.shape[0]):
        sig = oracle.jf_photons(fr[f], cal[0], cal[1])
        nb, nm, ne = check_frame(det, W, sig, o, f, kcap=kcap, bounds=bnd[f], floor=floor)
        tot_band += nb
    assert sep.device_status() == 0


def test_correction_bit_exact_all_raw_codes():
    """Every 16-bit raw word through the GPU correction, against the oracle's
    binary32 definition, bit for bit (values come back as kept pixels with a
    threshold below everything)."""
    rows, cols = 256, 256
    det = synth.Detector("codes", rows, cols, dist_m=0.1, center_px=(128.3, 120.7), nbins=8, split=1)
    rng = np.random.default_rng(9)
    ped = np.stack([rng.normal(m, s, rows * cols) for m, s in ((1500, 50), (14000, 200), (15000, 200))]).astype(np.float32)
    gain = np.stack([40 * (1 + rng.uniform(-.02, .02, rows * cols)), -1.5 * (1 + rng.uniform(-.02, .02, rows * cols)),
                     -0.1 * (1 + rng.uniform(-.02, .02, rows * cols))]).astype(np.float32)
    raw = np.arange(rows * cols, dtype=np.uint32).astype(np.uint16)[None]
    sep = Separator.from_detector(det, calib=(ped, gain), k_pick=0.0)
    d = torch.from_numpy(raw.astype(np.int16)).cuda()
    mean = torch.full((1, 8), -1e30, dtype=torch.float32, device="cuda")
    sigma = torch.zeros((1, 8), dtype=torch.float32, device="cuda")
    sp = sep.sparsify(d, mean, sigma, rows * cols)
    torch.cuda.synchronize()
    assert int(sp["n_kept"][0]) == rows * cols
    got = sp["val"][0].cpu().numpy()
    want = oracle.jf_photons(raw[0], ped, gain)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def _adversarial_gains():
    """Level-0 gains where a division by a correctly rounded reciprocal plus
    one correction step is most exposed: significands of all ones and just
    above a power of two, exact powers of two, both signs, across exponents
    up to and beyond the range the shortcut accepts (2^-100 .. 2^100)."""
    one_less = np.nextafter(np.float32(2), np.float32(0))     # 1.11..1b
    one_more = np.nextafter(np.float32(1), np.float32(2))     # 1.00..01b
    g = []
    for e in (-101, -100, -60, -7, -1, 0, 1, 5, 40, 99, 100):
        for m in (np.float32(1), one_less, one_more, np.float32(1.5), np.float32(40) / np.float32(32)):
            v = np.ldexp(m, e).astype(np.float32)
            g += [v, -v]
    return np.array(g, np.float32)


def test_level0_division_adversarial_gains():
    """The level-0 quotient RN((adc - ped) / gain) of the staging kernel,
    bit for bit against the oracle's binary32 definition, on every 14-bit
    ADC value and adversarial gains and pedestals (integers, fractions close
    to the ADC values, tiny, zero)."""
    rows, cols = 128, 128
    n = rows * cols
    det = synth.Detector("adv", rows, cols, dist_m=0.1, center_px=(64.3, 60.7), nbins=8, split=2)
    raw = np.arange(n, dtype=np.uint32).astype(np.uint16)          # code 0: level 0, adc = 0 .. 16383
    adc = raw.astype(np.float32)
    rng = np.random.default_rng(5)
    peds = [np.float32(1500.25) + rng.normal(0, 50, n).astype(np.float32),
            np.round(rng.uniform(0, 16000, n)).astype(np.float32),
            adc - np.float32(2.0 ** -10),                          # tiny differences
            np.full(n, np.float32(1e-30)), np.zeros(n, np.float32)]
    lv = np.ones(n, np.float32)
    for gi, g0 in enumerate(_adversarial_gains()):
        ped0 = peds[gi % len(peds)]
        ped = np.stack([ped0, lv * 14000, lv * 15000]).astype(np.float32)
        gain = np.stack([np.full(n, g0, np.float32), lv * -1.5, lv * -0.1]).astype(np.float32)
        sep = Separator.from_detector(det, calib=(ped, gain))
        got = sep.correct(torch.from_numpy(raw.astype(np.int16)[None]).cuda()).cpu().numpy()[0]
        want = oracle.jf_photons(raw, ped, gain)
        staged = ~np.isnan(got)
        assert staged.sum() > 0.9 * n
        a, b = got[staged], want[staged]
        same = (a.view(np.uint32) == b.view(np.uint32)) | (np.isnan(a) & np.isnan(b))
        assert same.all(), (g0, np.flatnonzero(~same)[:5], a[~same][:5], b[~same][:5])
        sep.close()


def test_staged_correction_bit_exact_all_raw_codes():
    """Every 16-bit raw word through the staging kernel (the values the
    integration reads), against the oracle's binary32 definition, bit for
    bit, on four calibrations; masked pixels come back as NaN."""
    rows, cols = 256, 256
    det = synth.Detector("codes", rows, cols, dist_m=0.1, center_px=(128.3, 120.7), nbins=8, split=2)
    raw = np.arange(rows * cols, dtype=np.uint32).astype(np.uint16)
    frames = np.stack([raw, raw[::-1], np.roll(raw, 12345), np.roll(raw, -777)])
    mask = np.zeros(rows * cols, np.uint8)
    mask[::97] = 1
    for seed in range(4):
        rng = np.random.default_rng(100 + seed)
        ped = np.stack([rng.normal(m, s, rows * cols) for m, s in ((1500, 50), (14000, 200), (15000, 200))])
        gain = np.stack([40 * (1 + rng.uniform(-.02, .02, rows * cols)), -1.5 * (1 + rng.uniform(-.02, .02, rows * cols)),
                         -0.1 * (1 + rng.uniform(-.02, .02, rows * cols))])
        ped, gain = ped.astype(np.float32), gain.astype(np.float32)
        sep = Separator.from_detector(det, mask=mask, calib=(ped, gain))
        got = sep.correct(torch.from_numpy(frames.astype(np.int16)).cuda()).cpu().numpy()
        for f in range(frames.shape[0]):
            want = oracle.jf_photons(frames[f], ped, gain)
            ok = mask == 0
            assert np.array_equal(got[f][ok].view(np.uint32), want[ok].view(np.uint32))
            assert np.all(np.isnan(got[f][~ok]))


def test_staged_division_many_adc_values():
    """Level-0 words with 256 different ADC values per pixel (every ADC value
    reaches 1024 pixels): the staged quotient equals the oracle's binary32
    division everywhere."""
    rows, cols = 256, 256
    det = synth.Detector("adc", rows, cols, dist_m=0.1, center_px=(128.3, 120.7), nbins=8, split=1)
    rng = np.random.default_rng(55)
    ped = np.stack([rng.normal(m, s, rows * cols) for m, s in ((1500, 50), (14000, 200), (15000, 200))]).astype(np.float32)
    gain = np.stack([40 * (1 + rng.uniform(-.02, .02, rows * cols)), -1.5 * (1 + rng.uniform(-.02, .02, rows * cols)),
                     -0.1 * (1 + rng.uniform(-.02, .02, rows * cols))]).astype(np.float32)
    sep = Separator.from_detector(det, calib=(ped, gain))
    i = np.arange(rows * cols)
    for chunk in range(4):
        f = np.arange(64 * chunk, 64 * chunk + 64)[:, None]
        frames = ((i[None, :] * 7 + f * 64) % 16384).astype(np.uint16)   # gain code 0
        got = sep.correct(torch.from_numpy(frames.astype(np.int16)).cuda()).cpu().numpy()
        for k in range(frames.shape[0]):
            want = oracle.jf_photons(frames[k], ped, gain)
            assert np.array_equal(got[k].view(np.uint32), want.view(np.uint32)), (chunk, k)


def test_edge_cases():
    det = synth.Detector("e", 40, 50, dist_m=0.05, center_px=(20.3, 18.7), nbins=30, split=2, unit=synth.UNIT_R_MM)
    mask = np.zeros(det.npix, np.uint8)
    W0 = oracle.weights(det, mask)
    # mask every pixel of bin 5: an empty bin
    mask[np.unique(W0.pix[W0.bin == 5])] = 1
    sep = Separator.from_detector(det, mask=mask)
    W = oracle.weights(det, mask)
    # empty batch: nothing launched, nothing written
    out = sep.alloc_outputs(1, 16, 16)
    sep.process_batch(torch.zeros((0, det.npix), dtype=torch.float32, device="cuda"), 16, 16)
    # constant frame: mean = constant, sigma = 0, nothing rejected, nothing kept
    const = np.full((1, det.npix), 7.25, np.float32)
    o, _ = run_batch(sep, const, 16, 16)
    ref = oracle.integrate_clip(W, const[0])
    has = ref["count"] > 0
    assert np.allclose(o["mean"][0][has], 7.25, rtol=1e-6) and np.all(o["sigma"][0] <= 1e-5)
    assert np.array_equal(o["count"][0], ref["count"]) and o["count"][0][5] == 0
    assert o["mean"][0][5] == 0 and o["sigma"][0][5] == 0
    assert o["n_kept"][0] == 0 and o["n_peaks"][0] == 0
    # capacity overflow: true count reported, first `cap` entries written, flag raised
    rng = np.random.default_rng(1)
    fr = rng.normal(10, 1, (1, det.npix)).astype(np.float32)
    fr[0, ::7] += 40
    o, _ = run_batch(sep, fr, 16, 4)
    assert o["n_kept"][0] > 16
    assert sep.device_status() & 1
    full, _ = run_batch(sep, fr, det.npix, 1000)
    assert np.array_equal(o["idx"][0][:16], full["idx"][0][:16])
    assert sep.device_status() == 0
    # no clipping at all
    sep.set_params(n_iter=0)
    o, _ = run_batch(sep, fr, det.npix, 1000)
    check_frame(det, W, fr[0], o, 0, n_iter=0, kcap=det.npix)


def test_norm_weights():
    det = synth.det_config1()
    rng = np.random.default_rng(2)
    norm = rng.uniform(0.5, 2.0, det.npix).astype(np.float32)
    fr = synth.frames(det, synth.spec_config1(3), 0, 2)[0] * norm
    fr = fr.astype(np.float32)
    sep = Separator.from_detector(det, norm=norm)
    o, dfr = run_batch(sep, fr, 8192, 512)
    bnd = sep.integrate_clip(dfr, bounds=True)["bounds"].cpu().numpy()
    W = oracle.weights(det)
    for f in range(2):
        check_frame(det, W, fr[f], o, f, kcap=8192, bounds=bnd[f], norm=norm)


def test_invalid_arguments_raise_before_launch():
    from paper_2411_09515_gb300 import SepError
    det = synth.det_config1()
    sep = Separator.from_detector(det)
    d = torch.zeros((1, det.npix), dtype=torch.float32, device="cuda")
    sep.set_params(patch=4)
    with pytest.raises(SepError):
        sep.process_batch(d, 16, 16)
    sep.set_params(patch=3, k_clip=0.0)
    with pytest.raises(SepError):
        sep.integrate_clip(d)
    sep.set_params(k_clip=3.0)
    with pytest.raises(SepError):   # raw frames without a calibration
        sep.integrate_clip(torch.zeros((1, det.npix), dtype=torch.int16, device="cuda"))


@pytest.mark.parametrize("tpb,thr", [([64], []), ([128], []), ([256], []), ([64, 256], [2048]), ([128, 128, 256], [512, 4096])])
def test_clip_plans_keep_parity(jf_small, tpb, thr):
    """The clip kernel's schedule (size classes, threads per block, parallel
    branches) changes no result beyond the stated tolerances."""
    det, mask, cal, fr, W = jf_small
    sep = Separator.from_detector(det, mask=mask, calib=cal)
    sep.set_plan(tpb, thr)
    assert sep.get_plan() == {"tpb": tpb, "thresholds": thr}
    kcap = det.npix // 4
    o, dfr = run_batch(sep, fr[:3], kcap, 20000)
    bnd = sep.integrate_clip(dfr, bounds=True)["bounds"].cpu().numpy()
    for f in range(3):
        sig = oracle.jf_photons(fr[f], cal[0], cal[1])
        check_frame(det, W, sig, o, f, kcap=kcap, bounds=bnd[f])


def test_autotune_picks_a_plan_and_caches_it(jf_small, tmp_path):
    det, mask, cal, fr, W = jf_small
    sep = Separator.from_detector(det, mask=mask, calib=cal)
    d = torch.from_numpy(fr.view(np.int16)).cuda()
    cache = tmp_path / "plans.txt"
    ms = sep.autotune(d, cache_path=cache)
    assert ms > 0 and cache.exists()
    plan = sep.get_plan()
    sep2 = Separator.from_detector(det, mask=mask, calib=cal)
    ms2 = sep2.autotune(d, cache_path=cache)   # read back, no timing
    assert sep2.get_plan() == plan and ms2 == pytest.approx(ms, rel=1e-3)
    o, dfr = run_batch(sep2, fr[:2], det.npix // 4, 20000)
    sig = oracle.jf_photons(fr[0], cal[0], cal[1])
    bnd = sep2.integrate_clip(dfr, bounds=True)["bounds"].cpu().numpy()
    check_frame(det, W, sig, o, 0, kcap=det.npix // 4, bounds=bnd[0])


def test_process_host_pipeline_equals_device_batch(jf_small):
    """Host-to-host pipelined path (chunks of 1 and 4: slots reused, ragged
    last chunk; one chunk) returns exactly what the device batch returns."""
    det, mask, cal, fr, W = jf_small
    sep = Separator.from_detector(det, mask=mask, calib=cal)
    kcap, pcap = det.npix // 4, 20000
    frames = np.ascontiguousarray(fr)
    o_dev, _ = run_batch(sep, frames, kcap, pcap)
    host = torch.from_numpy(frames.view(np.int16)).pin_memory()
    ho = sep.alloc_host_outputs(frames.shape[0], kcap, pcap)
    for chunk in (1, 4, 64):
        for v in ho.values():
            v.zero_()
        sep.process_host(host, ho, kcap, pcap, chunk_frames=chunk)
        torch.cuda.synchronize()
        for k in ("mean", "sigma", "count", "n_kept", "n_peaks"):
            assert np.array_equal(ho[k].numpy(), o_dev[k]), (chunk, k)
        for f in range(frames.shape[0]):
            n = int(o_dev["n_kept"][f])
            assert np.array_equal(ho["idx"][f, :n].numpy(), o_dev["idx"][f, :n])
            assert np.array_equal(ho["val"][f, :n].numpy(), o_dev["val"][f, :n])
            p = int(o_dev["n_peaks"][f])
            assert np.array_equal(ho["peaks"][f, :p].numpy(), o_dev["peaks"][f, :p])
    # pageable (not pinned) host outputs: the same results
    pageable = {k: torch.zeros(v.shape, dtype=v.dtype) for k, v in ho.items()}
    assert not any(t.is_pinned() for t in pageable.values())
    sep.process_host(host, pageable, kcap, pcap, chunk_frames=4)
    torch.cuda.synchronize()
    for k in ("mean", "sigma", "count", "n_kept", "n_peaks"):
        assert np.array_equal(pageable[k].numpy(), o_dev[k]), k
    for f in range(frames.shape[0]):
        n, p = int(o_dev["n_kept"][f]), int(o_dev["n_peaks"][f])
        assert np.array_equal(pageable["idx"][f, :n].numpy(), o_dev["idx"][f, :n])
        assert np.array_equal(pageable["val"][f, :n].numpy(), o_dev["val"][f, :n])
        assert np.array_equal(pageable["peaks"][f, :p].numpy(), o_dev["peaks"][f, :p])
    assert sep.device_status() == 0


@pytest.mark.parametrize("precision", [SEP_PREC_DWORD, SEP_PREC_PLAIN])
def test_chauvenet_cutoff_parity(jf_small, precision):
    """Eq. 20's cut-off for each set's size, against the oracle: raw split
    frames (coefficient classes), float frames without splitting (unit
    weights) and with a norm (per-entry weights), several iteration limits."""
    det, mask, cal, fr, W = jf_small
    sep = Separator.from_detector(det, mask=mask, calib=cal, precision=precision)
    sep.set_params(cutoff=SEP_CUTOFF_CHAUVENET)
    kcap = det.npix // 4
    for n_iter in (1, 5, 30):
        sep.set_params(n_iter=n_iter)
        o, dfr = run_batch(sep, fr[:3], kcap, 20000)
        bnd = sep.integrate_clip(dfr, bounds=True)["bounds"].cpu().numpy()
        for f in range(3):
            sig = oracle.jf_photons(fr[f], cal[0], cal[1])
            check_frame(det, W, sig, o, f, n_iter=n_iter, kcap=kcap, bounds=bnd[f], chauvenet=True)
    det1 = synth.det_config1()
    W1 = oracle.weights(det1)
    fr1 = synth.frames(det1, synth.spec_config1(7), 0, 2)[0].astype(np.float32)
    rng = np.random.default_rng(8)
    norm = rng.uniform(0.5, 2.0, det1.npix).astype(np.float32)
    for nrm in (None, norm):
        sep1 = Separator.from_detector(det1, norm=nrm, precision=precision)
        sep1.set_params(cutoff=SEP_CUTOFF_CHAUVENET)
        x = fr1 if nrm is None else (fr1 * nrm).astype(np.float32)
        o, dfr = run_batch(sep1, x, 8192, 512)
        bnd = sep1.integrate_clip(dfr, bounds=True)["bounds"].cpu().numpy()
        for f in range(2):
            check_frame(det1, W1, x[f], o, f, kcap=8192, bounds=bnd[f], norm=nrm, chauvenet=True)
    sep.set_params(surrogate=1)
    with pytest.raises(Exception):   # the surrogate predicts fixed-cut-off clipping only
        sep.integrate_clip(torch.from_numpy(fr[:1].view(np.int16)).cuda())


@pytest.mark.parametrize("precision", [SEP_PREC_DWORD, SEP_PREC_FP64MERGE])
def test_poisson_and_hybrid_error_models_parity(jf_small, precision):
    """Section 2.4.1's Poisson and hybrid models (Eqs. 3-4) against the
    oracle: raw split frames and float frames with unit coefficients, with and
    without a dark variance, and with Chauvenet's cut-off."""
    det, mask, cal, fr, W = jf_small
    det1 = synth.det_config1()
    W1 = oracle.weights(det1)
    fr1 = synth.frames(det1, synth.spec_config1(5), 0, 2)[0].astype(np.float32)
    for model in (SEP_ERROR_POISSON, SEP_ERROR_HYBRID):
        for dark, chauv in ((0.0, False), (1.5, False), (0.0, True)):
            cut = SEP_CUTOFF_CHAUVENET if chauv else 0
            sep = Separator.from_detector(det, mask=mask, calib=cal, precision=precision)
            sep.set_params(error_model=model, dark_var=dark, cutoff=cut)
            kcap = det.npix // 2
            o, dfr = run_batch(sep, fr[:2], kcap, 100000)   # emptied bins keep every positive pixel
            bnd = sep.integrate_clip(dfr, bounds=True)["bounds"].cpu().numpy()
            for f in range(2):
                sig = oracle.jf_photons(fr[f], cal[0], cal[1])
                check_frame(det, W, sig, o, f, kcap=kcap, bounds=bnd[f], chauvenet=chauv, model=model, dark=dark)
            sep1 = Separator.from_detector(det1, precision=precision)
            sep1.set_params(error_model=model, dark_var=dark, cutoff=cut)
            o, dfr = run_batch(sep1, fr1, 16384, 512)
            bnd = sep1.integrate_clip(dfr, bounds=True)["bounds"].cpu().numpy()
            for f in range(2):
                check_frame(det1, W1, fr1[f], o, f, kcap=16384, bounds=bnd[f], chauvenet=chauv, model=model, dark=dark)
    # a norm is refused (the Poisson variance is defined on unnormalised frames)
    norm = np.full(det1.npix, 2.0, np.float32)
    sepn = Separator.from_detector(det1, norm=norm)
    sepn.set_params(error_model=SEP_ERROR_POISSON)
    with pytest.raises(SepError):
        sepn.integrate_clip(torch.from_numpy(fr1).cuda())


@pytest.mark.parametrize("precision", [SEP_PREC_DWORD, SEP_PREC_FP64MERGE])
def test_exact_area_coefficients_parity(precision):
    """Exact area fractions (split 0: per-entry weights) against the oracle's
    own fractions, plain clipping and the Poisson model, with a mask."""
    det = synth.Detector("exact", 96, 110, dist_m=0.05, center_px=(40.3, 50.7), nbins=40, split=0,
                         unit=synth.UNIT_2TH_DEG)
    mask = np.zeros(det.npix, np.uint8)
    mask[::29] = 1
    W = oracle.weights_exact(det, mask)
    fr = synth.frames(det, synth.spec_config1(9), 0, 3, mask=mask)[0].astype(np.float32)
    for model in (0, SEP_ERROR_POISSON):
        sep = Separator.from_detector(det, mask=mask, precision=precision)
        sep.set_params(error_model=model)
        o, dfr = run_batch(sep, fr, det.npix, 4000)
        bnd = sep.integrate_clip(dfr, bounds=True)["bounds"].cpu().numpy()
        for f in range(3):
            check_frame(det, W, fr[f], o, f, kcap=det.npix, bounds=bnd[f], model=model)
