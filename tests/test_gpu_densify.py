"""Densification on the GPU (Section 3, "Densification / Decompression")
against the oracle, bit for bit: noise-free and noisy backgrounds, the fill of
pixels without a bin, kept lists longer than their capacity, indices outside
the detector, and the round trip through the library's own sparsification."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2411_09515_gb300 import SepError, Separator  # noqa: E402


@pytest.fixture(scope="module")
def small():
    det = synth.det_small_jf(split=2, nbins=300)
    mask = det.mask()
    cal = synth.jf_calib(det.npix, seed=7)
    spec = synth.spec_jf_serial(11)
    spec.hit_rate = 0.5
    fr, _, _ = synth.frames(det, spec, 0, 4, calib=cal, mask=mask)
    return det, mask, cal, fr, oracle.weights(det, mask)


def test_round_trip_through_the_library(small):
    det, mask, cal, fr, W = small
    sep = Separator.from_detector(det, mask=mask, calib=cal)
    kcap = det.npix // 4
    d = torch.from_numpy(fr.view(np.int16)).cuda()
    o = sep.process_batch(d, kcap, 2000)
    z = torch.from_numpy(np.random.default_rng(3).standard_normal((fr.shape[0], det.npix)).astype(np.float32)).cuda()
    for noise in (None, z):
        for fill in (float("nan"), -3.5):
            out = sep.densify(o["mean"], o["sigma"], o["idx"], o["val"], o["n_kept"], noise=noise, fill=fill)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            for f in range(fr.shape[0]):
                n = int(o["n_kept"][f])
                idx = o["idx"][f, :n].cpu().numpy()
                val = o["val"][f, :n].cpu().numpy()
                want = oracle.densify(W, o["mean"][f].cpu().numpy(), o["sigma"][f].cpu().numpy(), idx, val,
                                      noise=None if noise is None else z[f].cpu().numpy(), fill=fill)
                assert np.array_equal(got[f].view(np.uint32), want.view(np.uint32)), (f, noise is None, fill)
                # the kept pixels are the frame's corrected values
                sig = oracle.jf_photons(fr[f], cal[0], cal[1])
                assert np.array_equal(got[f][idx], sig[idx])
    assert sep.device_status() == 0


def test_capacity_and_foreign_indices(small):
    det, mask, cal, fr, W = small
    sep = Separator.from_detector(det, mask=mask, calib=cal)
    rng = np.random.default_rng(9)
    F, cap = 3, 64
    mean = rng.uniform(1, 5, (F, W.nbins)).astype(np.float32)
    sigma = rng.uniform(0, 1, (F, W.nbins)).astype(np.float32)
    # distinct indices per frame (a repeated index has no single answer),
    # a few of them outside the detector
    idx = np.stack([rng.permutation(np.arange(-10, det.npix + 10))[:cap] for _ in range(F)]).astype(np.int32)
    idx[:, :3] = [-5, det.npix, det.npix + 7]
    val = rng.uniform(100, 200, (F, cap)).astype(np.float32)
    n_kept = np.array([cap + 50, 10, 0], np.int32)                        # above, below, none
    t = {k: torch.from_numpy(v).cuda() for k, v in (("mean", mean), ("sigma", sigma), ("idx", idx), ("val", val),
                                                    ("n", n_kept))}
    out = sep.densify(t["mean"], t["sigma"], t["idx"], t["val"], t["n"]).cpu().numpy()
    for f in range(F):
        k = min(int(n_kept[f]), cap)
        want = oracle.densify(W, mean[f], sigma[f], idx[f, :k], val[f, :k])
        assert np.array_equal(out[f].view(np.uint32), want.view(np.uint32)), f
    with pytest.raises(SepError):   # noise without deviations
        sep.densify(t["mean"], None, t["idx"], t["val"], t["n"], noise=torch.zeros((F, det.npix), device="cuda"))


def test_odd_pixel_count_takes_the_scalar_kernel():
    det = synth.Detector("odd", 37, 41, dist_m=0.05, center_px=(18.3, 20.1), nbins=12, split=2)
    mask = np.zeros(det.npix, np.uint8)
    mask[::11] = 1
    W = oracle.weights(det, mask)
    sep = Separator.from_detector(det, mask=mask)
    rng = np.random.default_rng(4)
    F, cap = 2, 40
    mean = rng.uniform(1, 5, (F, W.nbins)).astype(np.float32)
    sigma = rng.uniform(0, 1, (F, W.nbins)).astype(np.float32)
    idx = np.stack([np.sort(rng.permutation(det.npix)[:cap]) for _ in range(F)]).astype(np.int32)
    val = rng.uniform(100, 200, (F, cap)).astype(np.float32)
    n_kept = np.array([cap, 7], np.int32)
    z = rng.standard_normal((F, det.npix)).astype(np.float32)
    t = [torch.from_numpy(a).cuda() for a in (mean, sigma, idx, val, n_kept, z)]
    interp = oracle.interpolation(det, W)
    for smooth in (False, True):
        out = sep.densify(t[0], t[1], t[2], t[3], t[4], noise=t[5], fill=0.5, interpolate=smooth).cpu().numpy()
        for f in range(F):
            k = int(n_kept[f])
            want = oracle.densify(W, mean[f], sigma[f], idx[f, :k], val[f, :k], noise=z[f], fill=0.5,
                                  interp=interp if smooth else None)
            assert np.array_equal(out[f].view(np.uint32), want.view(np.uint32)), (f, smooth)


def test_interpolated_background_bit_exact(small):
    det, mask, cal, fr, W = small
    sep = Separator.from_detector(det, mask=mask, calib=cal)
    d = torch.from_numpy(fr.view(np.int16)).cuda()
    o = sep.process_batch(d, det.npix // 4, 2000)
    z = torch.from_numpy(np.random.default_rng(5).standard_normal((fr.shape[0], det.npix)).astype(np.float32)).cuda()
    interp = oracle.interpolation(det, W)
    for noise in (None, z):
        got = sep.densify(o["mean"], o["sigma"], o["idx"], o["val"], o["n_kept"], noise=noise,
                          interpolate=True).cpu().numpy()
        for f in range(fr.shape[0]):
            n = int(o["n_kept"][f])
            want = oracle.densify(W, o["mean"][f].cpu().numpy(), o["sigma"][f].cpu().numpy(),
                                  o["idx"][f, :n].cpu().numpy(), o["val"][f, :n].cpu().numpy(),
                                  noise=None if noise is None else z[f].cpu().numpy(), interp=interp)
            assert np.array_equal(got[f].view(np.uint32), want.view(np.uint32)), (f, noise is None)
