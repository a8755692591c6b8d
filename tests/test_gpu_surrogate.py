"""The clip surrogate on the GPU, through the C ABI.

* network kernels against the FP64 CPU reference (oracle/mlp.py): forward
  outputs and the backpropagated gradient of the loss, evaluated at the
  BF16-rounded weights the GPU stores;
* training lowers the loss on a teacher-student problem;
* recorded features (on the row sample) and targets match their
  definitions on the oracle's per-bin values, and recording is the plain clip;
* with a model attached (trained or not) every result is the plain method's:
  the same clip sets (counts, bounds, iterations), means and deviations up to
  the rounding of another summation order, kept-pixel sets identical outside
  the threshold band, and the oracle's parity rules hold;
* what the trained network gains: its predicted cores spare rescans of the
  row that the plain placement needs.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import mlp
from parity import BAND, Frame, check_clip, close

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


def _row_sample(ex, b, step_of):
    """Entries of row b in pass A's sample: every step-th group of 4 of each
    coefficient class (the carriers after the classes excluded)."""
    r0, r1 = int(ex["rowptr"][b]), int(ex["rowptr"][b + 1])
    col, coef = ex["col"][r0:r1], ex["coef"][r0:r1]
    ng = (r1 - r0) // 4
    step = step_of(ng)
    # a group's class: the coefficient of its first matrix entry; a group of
    # padding slots only (col -1) lies inside the class of the run before it
    gcls = np.zeros(ng, np.float32)
    for q in range(ng):
        real = np.flatnonzero(col[4 * q:4 * q + 4] >= 0)
        gcls[q] = coef[4 * q + real[0]] if real.size else (gcls[q - 1] if q else 0.0)
    keep = np.zeros(r1 - r0, bool)
    g = 0
    while g < ng:
        if gcls[g] == 0:                     # the weight-0 carriers close the row
            break
        h = g
        while h < ng and gcls[h] == gcls[g]:
            h += 1
        for q in range(g, h, step):
            keep[4 * q:4 * q + 4] = True
        g = h
    sel = keep & (col >= 0) & (coef > 0)
    return col[sel], coef[sel].astype(np.float64), step


def _sketch(ex, b, sig):
    """The feature sketch's values of row b: element s (0 .. 127) is entry s
    when the row's weighted groups G hold at most 128 entries, else entry
    4 floor(s G / 128) + s mod 4; kept where it is a finite value of weight
    > 0."""
    r0, r1 = int(ex["rowptr"][b]), int(ex["rowptr"][b + 1])
    col, coef = ex["col"][r0:r1], ex["coef"][r0:r1]
    ng = (r1 - r0) // 4
    G = ng
    cls = 1.0
    for q in range(ng):
        real = np.flatnonzero(col[4 * q:4 * q + 4] >= 0)
        if real.size:
            cls = coef[4 * q + real[0]]
        if cls == 0:                          # the weight-0 carriers close the weighted groups
            G = q
            break
    out = []
    for s_ in range(128):
        if 4 * G <= 128:
            e = s_ if s_ < 4 * G else -1
        else:
            e = 4 * ((s_ * G) >> 7) + (s_ & 3)
        if e >= 0 and col[e] >= 0 and coef[e] > 0 and np.isfinite(sig[col[e]]):
            out.append(sig[col[e]])
    return np.asarray(out, np.float64)


def test_record_features_and_targets(jf_train):
    det, mask, cal, fr, _ = jf_train
    sep = Separator.from_detector(det, mask=mask, calib=cal)
    rec = sep.record(_dev(fr[:1]))
    plain = sep.integrate_clip(_dev(fr[:1]))
    torch.cuda.synchronize()
    # the recording run is the plain clip, bit for bit
    for k in ("mean", "sigma", "count"):
        assert np.array_equal(rec[k].cpu().numpy(), plain[k].cpu().numpy()), k
    feat = rec["feat"].cpu().numpy()[0]
    tgt = rec["target"].cpu().numpy()[0]
    ex = B.sep_csr_export(sep.csr)
    sig = oracle.jf_photons(fr[0], cal[0], cal[1])
    W = oracle.weights(det, mask)
    F = Frame(W, sig, 5, 3.0, 3.0)
    step_of = lambda ng: 4 if ng >= 512 else (2 if ng >= 128 else 1)
    checked = 0
    for b in range(0, det.nbins, 5):
        pix, c, step = _row_sample(ex, b, step_of)
        v = sig[pix].astype(np.float64)
        fin = np.isfinite(v)
        v, c = v[fin], c[fin]
        n = v.size
        if n < 16:
            continue
        om = c.sum()
        m1 = (c * v).sum() / om
        s1 = math.sqrt((c * c * (v - m1) ** 2).sum() / (c * c).sum())   # Eq. 13 over the sample
        if s1 == 0:
            continue
        assert feat[b, 0] == pytest.approx(math.log(n * step) / 8, rel=1e-5)
        assert feat[b, 1] == pytest.approx(om / n, rel=1e-5)
        assert feat[b, 2] == pytest.approx(max(min(m1 / s1, 20), -20) / 4, rel=1e-3, abs=1e-4)
        # the sketch: at most 128 entries spread over the weighted groups,
        # sorted; its share above m1 + 4 s1 and 16 order statistics of z
        sk = np.sort(_sketch(ex, b, sig))
        nv = sk.size
        assert nv > 0
        assert feat[b, 3] == pytest.approx((sk >= m1 + 4 * s1).mean(), abs=1.0 / nv + 1e-6)
        q = feat[b, 4:]
        assert np.all(np.diff(q) >= 0) and q[0] >= -4 and q[-1] <= 12
        ranks = ((2 * np.arange(16) + 1) * nv) >> 5
        want = np.clip((sk[ranks] - m1) / s1, -4, 12)
        assert np.allclose(q, want, rtol=1e-4, atol=2e-3), (b, q, want)
        mu, sd = F.ref["mean"][b], F.ref["sigma"][b]
        if F.ref["count"][b] >= 2 and sd > 0 and F.ref["band"][b] >= BAND:
            assert tgt[b, 0] == pytest.approx((mu - m1) / s1, rel=1e-3, abs=1e-3)
            assert tgt[b, 1] == pytest.approx(math.log(sd / s1), rel=1e-3, abs=1e-3)
        checked += 1
    assert checked > 20


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


def _same_as_plain(det, mask, cal, frames, out, plain):
    """Results with a model attached are the plain loop's: the same sets
    (count, bounds, iterations) wherever no decision sits in the band, the
    means and deviations up to the rounding of another summation order, and
    the oracle's parity rules."""
    W = oracle.weights(det, mask)
    for f in range(frames.shape[0]):
        F = Frame(W, oracle.jf_photons(frames[f], cal[0], cal[1]), 5, 3.0, 3.0)
        clean = F.ref["band"] >= BAND
        for k in ("count", "iters"):
            assert np.array_equal(out[k][f][clean], plain[k][f][clean]), k
        # the same set, its interval's bounds from moments rounded in another order
        bo, bp = out["bounds"][f][clean], plain["bounds"][f][clean]
        span = np.abs(bp[:, 1] - bp[:, 0])[:, None]
        assert np.all(np.abs(bo - bp) <= 1e-6 * (np.abs(bp) + span) + 1e-30), "bounds"
        sd = plain["sigma"][f]
        assert np.all(close(out["mean"][f][clean], plain["mean"][f][clean], rtol=1e-6, sd=sd[clean]))
        assert np.all(close(out["sigma"][f][clean], plain["sigma"][f][clean], rtol=1e-6, sd=sd[clean]))
        check_clip(F, out["mean"][f], out["sigma"][f], out["count"][f], out["bounds"][f])


def test_trained_model_gives_the_plain_results(jf_train, trained):
    det, mask, cal, _, held = jf_train
    sep, s, loss = trained
    d = _dev(held)
    sep.attach_surrogate(s)
    sep.surrogate_stats(reset=True)
    out = {k: v.cpu().numpy() for k, v in sep.integrate_clip(d, bounds=True, iters=True).items()}
    acc, fb = sep.surrogate_stats(reset=True)
    sep.attach_surrogate(None)
    plain = {k: v.cpu().numpy() for k, v in sep.integrate_clip(d, bounds=True, iters=True).items()}
    assert acc + fb == held.shape[0] * det.nbins
    _same_as_plain(det, mask, cal, held, out, plain)


def test_untrained_model_gives_the_plain_results(jf_train):
    det, mask, cal, _, held = jf_train
    sep = Separator.from_detector(det, mask=mask, calib=cal)
    s = Surrogate(sep.ctx, seed=99)   # random weights: poor predictions, more rescans
    sep.attach_surrogate(s)
    d = _dev(held[:2])
    out = {k: v.cpu().numpy() for k, v in sep.integrate_clip(d, bounds=True, iters=True).items()}
    sep.attach_surrogate(None)
    plain = {k: v.cpu().numpy() for k, v in sep.integrate_clip(d, bounds=True, iters=True).items()}
    _same_as_plain(det, mask, cal, held[:2], out, plain)
    s.close()


def test_trained_model_spares_rescans(jf_train, trained):
    """What the network gains: from its predicted final intervals the replay
    keeps its first core more often than from the plain placement (inside the
    first interval), so fewer rows are scanned again."""
    det, mask, cal, _, held = jf_train
    sep, s, _ = trained
    d = _dev(held)

    def scans():
        sep.clip_stats(enable=1, read=False, reset=True)
        sep.integrate_clip(d)
        st = sep.clip_stats(enable=0, read=True, reset=True)
        return (st["core_scans"] + st["full_passes"]) / st["items"]

    sep.attach_surrogate(None)
    plain = scans()
    sep.attach_surrogate(s)
    with_model = scans()
    sep.attach_surrogate(None)
    print(f"row scans per bin: plain {plain:.4f}, with the trained model {with_model:.4f}")
    assert with_model < plain, (with_model, plain)


def test_surrogate_batch_kept_sets_agree_with_plain(jf_train, trained):
    det, mask, cal, _, held = jf_train
    sep, s, _ = trained
    d = _dev(held)
    kcap = det.npix // 4
    sep.attach_surrogate(None)
    plain = {k: v.cpu().numpy() for k, v in sep.process_batch(d, kcap, 20000).items()}
    sep.attach_surrogate(s)
    sur_o = {k: v.cpu().numpy() for k, v in sep.process_batch(d, kcap, 20000).items()}
    sep.attach_surrogate(None)
    assert sep.device_status() == 0
    bop = oracle.weights(det, mask).bin_of_pixel
    for f in range(held.shape[0]):
        a = plain["idx"][f][: plain["n_kept"][f]]
        b = sur_o["idx"][f][: sur_o["n_kept"][f]]
        sig = oracle.jf_photons(held[f], cal[0], cal[1])
        thr_p = plain["mean"][f] + 3.0 * plain["sigma"][f]
        thr_s = sur_o["mean"][f] + 3.0 * sur_o["sigma"][f]
        # identical kept sets, except a pixel within the band of its threshold
        for i in np.setxor1d(a, b):
            bb = bop[i]
            ok = abs(sig[i] - thr_p[bb]) <= BAND * abs(thr_p[bb]) or abs(sig[i] - thr_s[bb]) <= BAND * abs(thr_s[bb])
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
