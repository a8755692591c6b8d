"""The clip surrogate on the GPU, through the C ABI.

* network kernels against the FP64 CPU reference (oracle/mlp.py): forward
  outputs and the backpropagated gradient of the loss, evaluated at the
  BF16-rounded weights the GPU stores;
* training lowers the loss on a teacher-student problem;
* recorded features and targets match their definitions on the oracle's
  per-bin values;
* predict + verify: every bin the surrogate settles is a fixed point of the
  clip map (Eq. 19) whose moments match the oracle's on that set, bins that
  fall back are bit-identical to the plain loop, and the kept-pixel sets agree
  with the plain method's outside the threshold band.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import mlp
from parity import BAND, Frame, close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2411_09515_gb300 import Separator, Surrogate  # noqa: E402
from paper_2411_09515_gb300 import _binding as B  # noqa: E402


def bf16(x):
    """Round float32 values to the nearest BF16 (ties to even), as float32."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


@pytest.fixture(scope="module")
def sur():
    sep = Separator.from_detector(synth.det_config1())
    s = Surrogate(sep.ctx, seed=3)
    yield sep, s
    s.close()
    sep.close()


def test_forward_matches_oracle(sur):
    _, s = sur
    rng = np.random.default_rng(0)
    theta = (mlp.init(5) * 0.8).astype(np.float32)
    theta[mlp.N_PARAMS - 2:] = [0.3, -0.7]
    s.params(theta)
    x = rng.normal(0, 1.5, (300, mlp.N_IN)).astype(np.float32)
    y = s.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    want, _ = mlp.forward(bf16(theta).astype(np.float64), x.astype(np.float64))
    assert np.allclose(y, want, rtol=1e-4, atol=1e-4 * np.abs(want).max())


def test_gradient_matches_oracle(sur):
    _, s = sur
    rng = np.random.default_rng(1)
    theta = (mlp.init(9) * 0.9).astype(np.float32)
    s.params(theta)
    n = 777   # several tiles of 64 and a ragged last one
    x = rng.normal(0, 1, (n, mlp.N_IN)).astype(np.float32)
    t = rng.normal(0, 1, (n, mlp.N_OUT)).astype(np.float32)
    loss, g = s.loss_grad(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    g = g.cpu().numpy().astype(np.float64)
    th = bf16(theta).astype(np.float64)
    want = mlp.grad(th, x.astype(np.float64), t.astype(np.float64))
    assert float(loss.item()) == pytest.approx(mlp.loss(th, x, t), rel=1e-4)
    rel = np.linalg.norm(g - want) / np.linalg.norm(want)
    assert rel < 1e-4, rel
    assert np.allclose(g, want, rtol=1e-3, atol=1e-4 * np.abs(want).max())


def test_training_lowers_the_loss(sur):
    _, s0 = sur
    # a teacher network defines the targets; the student starts elsewhere
    rng = np.random.default_rng(2)
    teacher = mlp.init(11) * 0.5
    x = rng.normal(0, 1, (20000, mlp.N_IN))
    t, _ = mlp.forward(teacher, x)
    t = (t - t.mean(0)) / t.std(0)
    s = Surrogate(s0.ctx, seed=4)
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    td = torch.from_numpy(t.astype(np.float32)).cuda()
    l0 = float(s.loss_grad(xd, td)[0].item())
    loss, nv = s.fit(xd, td, epochs=30, batch=256, lr=3e-3)
    assert nv == 20000
    # fit() normalised the data; measure on the same normalisation
    norm = s.norm()
    xn = (xd - torch.from_numpy(norm[:20]).cuda()) / torch.from_numpy(norm[20:40]).cuda()
    tn = (td - torch.from_numpy(norm[40:42]).cuda()) / torch.from_numpy(norm[42:44]).cuda()
    l1 = float(s.loss_grad(xn, tn)[0].item())
    assert l1 < 0.25 * l0 and l1 < 0.3, (l0, l1, loss)
    s.close()


def test_prepare_drops_nonfinite_rows_and_normalises(sur):
    sep, _ = sur
    rng = np.random.default_rng(5)
    f = rng.normal(2, 3, (5000, 20)).astype(np.float32)
    t = rng.normal(-1, 0.5, (5000, 2)).astype(np.float32)
    t[::7, 1] = np.nan
    f[3::11, 4] = np.inf
    keep = np.isfinite(t).all(1) & np.isfinite(f).all(1)
    x = torch.empty((5000, 20), dtype=torch.float32, device="cuda")
    y = torch.empty((5000, 2), dtype=torch.float32, device="cuda")
    norm, nv = B.sep_surrogate_prepare(sep.ctx, torch.from_numpy(f).cuda(), torch.from_numpy(t).cuda(), 5000, x, y)
    assert nv == keep.sum()
    fk, tk = f[keep].astype(np.float64), t[keep].astype(np.float64)
    assert np.allclose(norm[:20], fk.mean(0), rtol=1e-6, atol=1e-6)
    assert np.allclose(norm[20:40], fk.std(0), rtol=1e-5)
    assert np.allclose(norm[40:42], tk.mean(0), rtol=1e-6, atol=1e-6)
    assert np.allclose(norm[42:44], tk.std(0), rtol=1e-5)
    xn = x[:nv].cpu().numpy()
    assert np.allclose(xn, (fk - norm[:20]) / norm[20:40], atol=1e-5)   # order preserved


@pytest.fixture(scope="module")
def jf_train():
    det = synth.det_small_jf(split=2, nbins=300)
    mask = det.mask()
    cal = synth.jf_calib(det.npix, seed=7)
    spec = synth.spec_jf_serial(21)
    spec.hit_rate = 0.5
    fr, _, _ = synth.frames(det, spec, 0, 48, calib=cal, mask=mask)
    held, _, _ = synth.frames(det, spec, 1000, 4, calib=cal, mask=mask)
    return det, mask, cal, fr, held


def _dev(fr):
    return torch.from_numpy(np.ascontiguousarray(fr).view(np.int16)).cuda()


def test_record_features_and_targets(jf_train):
    det, mask, cal, fr, _ = jf_train
    sep = Separator.from_detector(det, mask=mask, calib=cal)
    rec = sep.record(_dev(fr[:1]))
    plain = sep.integrate_clip(_dev(fr[:1]))
    torch.cuda.synchronize()
    # the recording run is the plain clip
    for k in ("mean", "sigma", "count"):
        assert np.array_equal(rec[k].cpu().numpy(), plain[k].cpu().numpy()), k
    feat = rec["feat"].cpu().numpy()[0]
    tgt = rec["target"].cpu().numpy()[0]
    W = oracle.weights(det, mask)
    sig = oracle.jf_photons(fr[0], cal[0], cal[1])
    F = Frame(W, sig, 5, 3.0, 3.0)
    checked = 0
    for b in range(0, W.nbins, 7):
        pix, c = F.entries(b)
        live = c > 0
        if live.sum() < 16:
            continue
        v, w = F.v[pix[live]], c[live]
        n = live.sum()
        om = w.sum()
        m1 = (w * v).sum() / om
        s1 = math.sqrt((w * w * (v - m1) ** 2).sum() / (w * w).sum())   # Eq. 13 over the full set
        assert feat[b, 0] == pytest.approx(math.log(n) / 8, rel=1e-5)
        assert feat[b, 1] == pytest.approx(om / n, rel=1e-5)
        assert feat[b, 2] == pytest.approx(max(min(m1 / s1, 20), -20) / 4, rel=1e-3, abs=1e-4)
        z = (v - m1) / s1
        assert feat[b, 3] == pytest.approx((z >= 4).mean(), abs=2.0 / n)
        q = feat[b, 4:]
        assert np.all(np.diff(q) >= 0) and q[0] >= -4 and q[-1] <= 12
        # a quantile read off the 0.25-wide histogram lies within one bin of the exact one
        for j in (3, 8, 12):
            exact = np.quantile(z, (j + 0.5) / 16)
            if -4 < exact < 12:
                assert abs(q[j] - exact) <= 0.25 + 1e-3, (b, j, q[j], exact)
        mu, sd = F.ref["mean"][b], F.ref["sigma"][b]
        if F.ref["count"][b] >= 2 and sd > 0 and F.ref["band"][b] >= BAND:
            assert tgt[b, 0] == pytest.approx((mu - m1) / s1, rel=1e-3, abs=1e-3)
            assert tgt[b, 1] == pytest.approx(math.log(sd / s1), rel=1e-3, abs=1e-3)
        checked += 1
    assert checked > 20


def _check_settled(F, k, mean, sigma, count, bounds, iters):
    """Every settled bin (iters == -1) is a fixed point of the clip map with the
    oracle's moments on its set; returns the settled bins."""
    settled = np.flatnonzero(iters == -1)
    for b in settled:
        pix, c = F.entries(b)
        L, H = bounds[b]
        vv = F.sig[pix]
        live = c > 0
        sel = (vv >= L) & (vv <= H) & live
        mu, sd, n = oracle.moments_subset(pix, c, sel.astype(np.uint8), F.sig, F.norm)
        assert count[b] == n and close(mean[b], mu, sd=np.array(sd)) and close(sigma[b], sd, sd=np.array(sd)), \
            (b, mean[b], mu, sigma[b], sd, count[b], n)
        # fixed point: the next set {|v - mu| <= k sd} is the same set (up to the band)
        nxt = (np.abs(vv.astype(np.float64) - mu) <= k * sd) & live
        diff = nxt != sel
        if diff.any():
            edge = np.abs(np.abs(vv[diff] - mu) - k * sd) <= BAND * (abs(mu) + k * sd)
            assert edge.all(), (b, vv[diff], mu, sd)
    return settled


@pytest.fixture(scope="module")
def trained(jf_train):
    det, mask, cal, fr, _ = jf_train
    sep = Separator.from_detector(det, mask=mask, calib=cal)
    feats, tgts = [], []
    for i in range(0, fr.shape[0], 16):
        r = sep.record(_dev(fr[i:i + 16]))
        feats.append(r["feat"])
        tgts.append(r["target"])
    s = Surrogate(sep.ctx, seed=1)
    loss, nv = s.fit(torch.cat(feats), torch.cat(tgts), epochs=40, batch=256, lr=2e-3)
    assert nv > 0.9 * fr.shape[0] * det.nbins * 0.5
    return sep, s, loss


def test_predict_verify_settled_bins_are_fixed_points(jf_train, trained):
    det, mask, cal, _, held = jf_train
    sep, s, loss = trained
    W = oracle.weights(det, mask)
    sep.attach_surrogate(s, passes=2)
    sep.surrogate_stats(reset=True)
    d = _dev(held)
    out = sep.integrate_clip(d, bounds=True, iters=True)
    acc, fb = sep.surrogate_stats(reset=True)
    sep.attach_surrogate(None)
    plain = sep.integrate_clip(d, bounds=True, iters=True)
    torch.cuda.synchronize()
    o = {k: v.cpu().numpy() for k, v in out.items()}
    p = {k: v.cpu().numpy() for k, v in plain.items()}
    assert 0 < acc + fb <= held.shape[0] * det.nbins
    assert acc >= 0.1 * (acc + fb), (acc, fb, loss)   # the trained model settles a share of the bins
    n_same = 0
    for f in range(held.shape[0]):
        sig = oracle.jf_photons(held[f], cal[0], cal[1])
        F = Frame(W, sig, 5, 3.0, 3.0)
        settled = _check_settled(F, 3.0, o["mean"][f], o["sigma"][f], o["count"][f], o["bounds"][f], o["iters"][f])
        fell = np.flatnonzero(o["iters"][f] != -1)
        # bins that fell back ran the plain loop from the same start: bit-identical
        for k in ("mean", "sigma", "count", "bounds", "iters"):
            assert np.array_equal(o[k][f][fell], p[k][f][fell]), k
        # a settled bin is the converged clip; the plain loop reaches the same
        # set unless it stopped at n_iter or at another fixed point
        n_same += (o["count"][f][settled] == p["count"][f][settled]).sum()
    assert n_same >= 0.5 * acc


def test_untrained_model_is_still_exact(jf_train):
    det, mask, cal, _, held = jf_train
    sep = Separator.from_detector(det, mask=mask, calib=cal)
    s = Surrogate(sep.ctx, seed=99)   # random weights: predictions are poor
    sep.attach_surrogate(s, passes=1)
    d = _dev(held[:2])
    out = {k: v.cpu().numpy() for k, v in sep.integrate_clip(d, bounds=True, iters=True).items()}
    sep.attach_surrogate(None)
    ref = {k: v.cpu().numpy() for k, v in sep.integrate_clip(d, bounds=True, iters=True).items()}
    W = oracle.weights(det, mask)
    for f in range(2):
        F = Frame(W, oracle.jf_photons(held[f], cal[0], cal[1]), 5, 3.0, 3.0)
        _check_settled(F, 3.0, out["mean"][f], out["sigma"][f], out["count"][f], out["bounds"][f], out["iters"][f])
        fell = out["iters"][f] != -1
        assert np.array_equal(out["mean"][f][fell], ref["mean"][f][fell])
        assert np.array_equal(out["sigma"][f][fell], ref["sigma"][f][fell])
    s.close()


def test_surrogate_batch_kept_sets_agree_with_plain(jf_train, trained):
    det, mask, cal, _, held = jf_train
    sep, s, _ = trained
    d = _dev(held)
    kcap = det.npix // 4
    sep.attach_surrogate(None)
    plain = {k: v.cpu().numpy() for k, v in sep.process_batch(d, kcap, 20000).items()}
    sep.attach_surrogate(s, passes=2)
    sur_o = {k: v.cpu().numpy() for k, v in sep.process_batch(d, kcap, 20000).items()}
    sep.attach_surrogate(None)
    assert sep.device_status() == 0
    for f in range(held.shape[0]):
        a = plain["idx"][f][: plain["n_kept"][f]]
        b = sur_o["idx"][f][: sur_o["n_kept"][f]]
        diff = np.setxor1d(a, b)
        # differences only at pixels within the band of either threshold
        sig = oracle.jf_photons(held[f], cal[0], cal[1])
        bop = oracle.weights(det, mask).bin_of_pixel
        thr_p = plain["mean"][f] + 3.0 * plain["sigma"][f]
        thr_s = sur_o["mean"][f] + 3.0 * sur_o["sigma"][f]
        for i in diff:
            bb = bop[i]
            ok = abs(sig[i] - thr_p[bb]) <= BAND * abs(thr_p[bb]) or abs(sig[i] - thr_s[bb]) <= BAND * abs(thr_s[bb]) \
                or plain["count"][f][bb] != sur_o["count"][f][bb]
            assert ok, (f, i, sig[i], thr_p[bb], thr_s[bb])


def test_model_checkpoint_round_trip(sur, tmp_path):
    sep, s = sur
    theta = (mlp.init(2) * 0.5).astype(np.float32)
    s.params(theta)
    norm = np.linspace(0.5, 2.0, 44).astype(np.float32)
    s.norm(norm)
    path = str(tmp_path / "m.sep")
    s.save(path)
    s2 = Surrogate(sep.ctx, path=path)
    assert np.array_equal(s2.params(), theta)
    assert np.array_equal(s2.norm(), norm)
    s2.close()


def test_surrogate_needs_a_model_and_dword(sur):
    sep, _ = sur
    fr = synth.frames(synth.det_config1(), synth.spec_config1(0), 0, 1)[0]
    d = torch.from_numpy(fr).cuda()
    sep.set_params(surrogate=1)
    with pytest.raises(B.SepError):
        sep.integrate_clip(d)    # no model attached
    sep.set_params(surrogate=0)
