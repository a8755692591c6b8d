"""Veto and frame-drop compaction on the GPU (Section 4, "Peak count as veto
algorithm") against the oracle: frame lists over several scan tiles with
counts at the threshold, rows of any width (word and vector copies), and
the per-frame outputs of a real batch."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2411_09515_gb300 import Separator  # noqa: E402


def test_veto_lists_and_compaction():
    det = synth.det_config1()
    sep = Separator.from_detector(det)
    rng = np.random.default_rng(12)
    F = 3000
    counts = rng.integers(0, 41, F).astype(np.int32)
    counts[::97] = 20                                   # exactly at the threshold
    dc = torch.from_numpy(counts).cuda()
    for thr in (0, 1, 20, 40, 41):
        lst, n = sep.veto(dc, thr)
        want = oracle.veto(counts.tolist(), thr)
        assert int(n.item()) == len(want)
        assert lst[: len(want)].cpu().numpy().tolist() == want
    lst, n = sep.veto(dc, 20)
    want = oracle.veto(counts.tolist(), 20)
    for width, dtype in ((37, torch.int32), (64, torch.float32), (3, torch.float32)):
        if dtype == torch.float32:
            src = torch.from_numpy(rng.standard_normal((F, width)).astype(np.float32)).cuda()
        else:
            src = torch.from_numpy(rng.integers(-9, 9, (F, width)).astype(np.int32)).cuda()
        out = torch.full_like(src, 7)
        sep.compact_frames(lst, n, src, out=out)
        got = out.cpu().numpy()
        ref = src.cpu().numpy()
        assert np.array_equal(got[: len(want)], ref[want])
        assert np.all(got[len(want):] == 7)                # rows past the count untouched


def test_veto_on_a_batch():
    det = synth.det_small_jf(split=2, nbins=200)
    mask = det.mask()
    cal = synth.jf_calib(det.npix, seed=3)
    spec = synth.spec_jf_serial(5)
    spec.hit_rate = 0.5
    fr, _, _ = synth.frames(det, spec, 0, 8, calib=cal, mask=mask)
    sep = Separator.from_detector(det, mask=mask, calib=cal)
    o = sep.process_batch(torch.from_numpy(fr.view(np.int16)).cuda(), det.npix // 4, 4096)
    npk = o["n_peaks"].cpu().numpy()
    thr = int(np.median(npk)) + 1
    lst, n = sep.veto(o["n_peaks"], thr)
    want = oracle.veto(npk.tolist(), thr)
    assert lst[: int(n.item())].cpu().numpy().tolist() == want
    for k in ("mean", "n_kept", "idx", "peaks"):
        out = sep.compact_frames(lst, n, o[k])
        assert np.array_equal(out[: len(want)].cpu().numpy(), o[k][want].cpu().numpy()), k
