"""Limits the library checks on the host before any launch: frames per call
(SEP_MAX_FRAMES, one grid row per frame), and the Poisson / hybrid error
models refused for a detector with a norm in a mixed batch as in a
single-detector one."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2411_09515_gb300 import (SEP_ERROR_POISSON, Context, Separator, SepError,  # noqa: E402
                                    _binding as B, process_mixed)


def test_frames_per_call_limit():
    det = synth.Detector("e", 40, 50, dist_m=0.05, center_px=(20.3, 18.7), nbins=30, split=2, unit=synth.UNIT_R_MM)
    sep = Separator.from_detector(det)
    big = torch.zeros((B.SEP_MAX_FRAMES + 1, det.npix), dtype=torch.float32, device="cuda")
    with pytest.raises(SepError) as e:
        sep.process_batch(big, 4, 4)
    assert e.value.status == B.SEP_ERR_ARG
    with pytest.raises(SepError) as e:
        sep.integrate_clip(big)
    assert e.value.status == B.SEP_ERR_ARG
    del big
    # the refusals leave the context usable
    ok = torch.zeros((4, det.npix), dtype=torch.float32, device="cuda")
    sep.process_batch(ok, 4, 4)
    torch.cuda.synchronize()
    assert sep.device_status() == 0
    sep.close()


def test_mixed_batch_refuses_poisson_with_a_norm():
    ctx = Context(0)
    det = synth.det_config1()
    norm = np.full(det.npix, 2.0, np.float32)
    seps = [Separator.from_detector(det, context=ctx), Separator.from_detector(det, norm=norm, context=ctx)]
    seps[0].set_params(error_model=SEP_ERROR_POISSON)
    frames = [(0, torch.zeros(det.npix, dtype=torch.float32, device="cuda")),
              (1, torch.zeros(det.npix, dtype=torch.float32, device="cuda"))]
    with pytest.raises(SepError) as e:
        process_mixed(seps, frames, 16, 16)
    assert e.value.status == B.SEP_ERR_ARG
    for s in seps:
        s.close()
    ctx.close()
