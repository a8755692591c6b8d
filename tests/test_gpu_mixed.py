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
