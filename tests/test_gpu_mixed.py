"""Mixed batches: frames of several detectors of different sizes in one call
(one captured graph), each frame's outputs equal to processing it alone."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2411_09515_gb300 import Context, Separator, process_mixed  # noqa: E402


def test_mixed_stream_equals_per_detector_batches():
    ctx = Context(0)
    dets = [synth.det_jf1m(nbins=600), synth.det_config1(), synth.det_small_jf(split=2, nbins=150)]
    seps = [Separator.from_detector(d, mask=d.mask() if d.layout else None, context=ctx) for d in dets]
    seps[0].set_plan([64, 128], [1024])      # schedules differ per detector
    pattern = [0, 1, 0, 2, 1, 0, 2, 0, 1]
    frames, per_det = [], {0: [], 1: [], 2: []}
    for g, d in enumerate(pattern):
        spec = synth.spec_mixed(seed=40 + g, hit_rate=0.5) if d != 1 else synth.spec_config1(40 + g)
        fr = synth.frames(dets[d], spec, g, 1, mask=dets[d].mask() if dets[d].layout else None)[0]
        t = torch.from_numpy(fr[0]).cuda()
        frames.append((d, t))
        per_det[d].append((g, fr[0]))
    kcap, pcap = 60000, 4000
    for use_graph in (True, True, False):   # capture, replay, eager
        out = process_mixed(seps, frames, kcap, pcap, use_graph=use_graph)
        torch.cuda.synchronize()
        rows = out["row_off"]
        assert rows[-1] == sum(seps[d].nbins for d in pattern)
        for d, lst in per_det.items():
            batch = torch.from_numpy(np.stack([f for _, f in lst])).cuda()
            ref = seps[d].process_batch(batch, kcap, pcap, use_graph=False)
            torch.cuda.synchronize()
            for j, (g, _) in enumerate(lst):
                r0, r1 = rows[g], rows[g + 1]
                for k in ("mean", "sigma", "count"):
                    assert np.array_equal(out[k][r0:r1].cpu().numpy(), ref[k][j].cpu().numpy()), (k, g)
                nk = int(ref["n_kept"][j])
                assert int(out["n_kept"][g]) == nk
                assert np.array_equal(out["idx"][g, :nk].cpu().numpy(), ref["idx"][j, :nk].cpu().numpy())
                assert np.array_equal(out["val"][g, :nk].cpu().numpy(), ref["val"][j, :nk].cpu().numpy())
                npk = int(ref["n_peaks"][j])
                assert int(out["n_peaks"][g]) == npk
                assert np.array_equal(out["peaks"][g, :npk].cpu().numpy(), ref["peaks"][j, :npk].cpu().numpy())
    assert seps[0].device_status() == 0
    for s in seps:
        s.close()
    ctx.close()


def test_mixed_stream_1m_16m_against_the_oracle():
    """One 1M and one 16M Jungfrau-shaped float32 frame (600 / 2000 bins, no
    splitting), with a 4M frame between them, in one mixed call: the 1M and
    16M frames' profiles, kept pixels and peaks against the FP64 oracle."""
    import oracle
    from parity import check_frame
    ctx = Context(0)
    dets = [synth.det_jf1m(nbins=600), synth.det_jf4m(split=1, nbins=1000), synth.det_jf16m(nbins=2000)]
    masks = [d.mask() for d in dets]
    seps = [Separator.from_detector(d, mask=m, context=ctx) for d, m in zip(dets, masks)]
    pattern = [0, 1, 2]
    frames, host = [], []
    for g, d in enumerate(pattern):
        fr = synth.frames(dets[d], synth.spec_mixed(seed=70 + g, hit_rate=1.0), g, 1, mask=masks[d])[0]
        host.append(fr)
        frames.append((d, torch.from_numpy(fr[0]).cuda()))
    kcap, pcap = 1 << 20, 1 << 15
    out = process_mixed(seps, frames, kcap, pcap)
    torch.cuda.synchronize()
    assert seps[0].device_status() == 0
    rows = out["row_off"]
    for g in (0, 2):
        d = pattern[g]
        r0, r1 = rows[g], rows[g + 1]
        o = {"mean": out["mean"][r0:r1].cpu().numpy()[None], "sigma": out["sigma"][r0:r1].cpu().numpy()[None],
             "count": out["count"][r0:r1].cpu().numpy()[None],
             "idx": out["idx"][g:g + 1].cpu().numpy(), "val": out["val"][g:g + 1].cpu().numpy(),
             "n_kept": out["n_kept"][g:g + 1].cpu().numpy(), "peaks": out["peaks"][g:g + 1].cpu().numpy(),
             "n_peaks": out["n_peaks"][g:g + 1].cpu().numpy()}
        # the final sets' bounds, from the same kernel on the frame alone
        bnd = seps[d].integrate_clip(frames[g][1][None], bounds=True)["bounds"].cpu().numpy()
        W = oracle.weights(dets[d], masks[d])
        check_frame(dets[d], W, host[g][0], o, 0, kcap=kcap, bounds=bnd[0])
    for s in seps:
        s.close()
    ctx.close()
