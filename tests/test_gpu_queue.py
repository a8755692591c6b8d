"""The persistent clip launch against the one-CTA-per-unit launch.

A clip launch whose units (a bin and a group of frames) outnumber the CTAs
that stay resident runs those CTAs over a work-queue counter; a smaller
launch runs one CTA per unit. Every item is computed by one warp from its
own row, whatever CTA takes it, so both launches give the same bits, and
the queue must hand out every unit exactly once.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2411_09515_gb300 import Separator  # noqa: E402


def test_queue_covers_every_unit_once_and_matches_the_plain_grid():
    det = synth.det_config1()
    base = np.concatenate([synth.frames(det, synth.spec_config1(s), 0, 1)[0] for s in range(8)])
    sep = Separator.from_detector(det)
    small = torch.from_numpy(base).cuda()
    # 1024 frames of 64 bins: 16,384 units of four frames, far more than the
    # CTAs one GPU keeps resident; 8 frames: 512 units of one frame
    big = small.repeat(128, 1)
    F = big.shape[0]
    ref = sep.integrate_clip(small, bounds=True)
    sep.clip_stats(enable=1, read=False, reset=True)
    got = sep.integrate_clip(big, bounds=True)
    torch.cuda.synchronize()
    st = sep.clip_stats(enable=0, read=True, reset=True)
    assert st["items"] == F * det.nbins, st
    for k in ("mean", "sigma", "count", "bounds"):
        r = ref[k].cpu().numpy()
        g = got[k].cpu().numpy()
        for m in range(F // 8):
            assert np.array_equal(g[8 * m:8 * m + 8], r), (k, m)
    # the whole path on both launch shapes: the same kept pixels and peaks
    cap = det.npix // 4
    o_s = sep.process_batch(small, cap, 512)
    o_b = sep.process_batch(big, cap, 512)
    torch.cuda.synchronize()
    nk_s, nk_b = o_s["n_kept"].cpu().numpy(), o_b["n_kept"].cpu().numpy()
    np_s, np_b = o_s["n_peaks"].cpu().numpy(), o_b["n_peaks"].cpu().numpy()
    for f in range(F):
        j = f % 8
        assert nk_b[f] == nk_s[j] and np_b[f] == np_s[j], f
    for f in (0, 7, 8, 515, F - 1):
        j = f % 8
        n = int(nk_s[j])
        assert np.array_equal(o_b["idx"][f, :n].cpu().numpy(), o_s["idx"][j, :n].cpu().numpy()), f
        assert np.array_equal(o_b["val"][f, :n].cpu().numpy(), o_s["val"][j, :n].cpu().numpy()), f
    assert sep.device_status() == 0
