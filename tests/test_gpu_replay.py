"""The tail replay of the clip loop (Eq. 19 on a core plus the entries
outside it) against the oracle on the paths a benchmark frame rarely takes:
bins whose outliers overflow a lane's tail slots (the remaining steps run as
full passes) and bins whose later intervals cut into the first core (the
row is scanned again), with the replay counters that show each path ran.
"""
import numpy as np
import pytest

import oracle
import synth
from parity import check_frame

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2411_09515_gb300 import Separator  # noqa: E402


def _frames(det, n, frac, scale, seed):
    """Config-1 frames with a fraction of pixels raised by a large factor:
    heavy tails that fill the tail slots and pull the first interval wide."""
    fr = np.concatenate([synth.frames(det, synth.spec_config1(seed + s), 0, 1)[0] for s in range(n)])
    rng = np.random.default_rng(seed)
    hot = rng.random(fr.shape) < frac
    fr = fr.copy()
    fr[hot] = fr[hot] * scale + scale
    return fr


@pytest.mark.parametrize("frac,scale", [(0.3, 50.0), (0.08, 7.0)])
def test_replay_fallbacks_match_the_oracle(frac, scale):
    det = synth.det_config1()
    W = oracle.weights(det)
    fr = _frames(det, 6, frac, scale, 100)
    sep = Separator.from_detector(det)
    dfr = torch.from_numpy(fr).cuda()
    sep.clip_stats(enable=1, read=False, reset=True)
    ic = sep.integrate_clip(dfr, bounds=True)
    torch.cuda.synchronize()
    st = sep.clip_stats(enable=0, read=True, reset=True)
    assert st["items"] == fr.shape[0] * det.nbins
    # every item scanned its row at least once or ran full passes
    assert st["core_scans"] + st["full_passes"] >= st["items"]
    if frac > 0.2:
        assert st["overflows"] > 0 and st["full_passes"] > 0, st
    else:
        assert st["core_scans"] > st["items"], st   # re-scans after a cut core
    # the same results with the counters off, bit for bit
    ic2 = sep.integrate_clip(dfr, bounds=True)
    torch.cuda.synchronize()
    for k in ("mean", "sigma", "count", "bounds"):
        assert np.array_equal(ic[k].cpu().numpy(), ic2[k].cpu().numpy()), k
    out = sep.process_batch(dfr, det.npix, det.npix // 4)
    torch.cuda.synchronize()
    o = {k: v.cpu().numpy() for k, v in out.items()}
    assert np.array_equal(o["mean"], ic["mean"].cpu().numpy())
    bnd = ic["bounds"].cpu().numpy()
    for f in range(fr.shape[0]):
        check_frame(det, W, fr[f], o, f, kcap=det.npix, bounds=bnd[f])
    assert sep.device_status() == 0
