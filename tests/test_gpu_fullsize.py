"""The Jungfrau-4M workload in the launch configuration the benchmark times:
512 distinct raw frames in one batch (2164 x 2068 pixels, 1000 bins, 2 x 2
splitting), the autotuned clip schedule, one captured graph, default DWORD
precision, the benchmark's capacities. Sampled frames of the batch are
checked against the oracle one by one (per-bin mean, deviation and count,
kept pixels, peaks), and properties that hold for every frame are checked on
all 512."""
import numpy as np
import pytest

import oracle
from parity import check_frame

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import bench  # noqa: E402  (the benchmark's workload generator)
from paper_2411_09515_gb300 import Separator  # noqa: E402

F, KCAP, PCAP = 512, 262144, 8192
SAMPLED = (0, 311, 511)


def test_jf4m_batch_of_512_in_the_benchmark_configuration():
    det, mask, cal, frames = bench.setup_workload(F, 0)
    sep = Separator.from_detector(det, mask=mask, calib=cal)
    dev = torch.from_numpy(frames.view(np.int16)).cuda()
    sep.autotune(dev[: min(F, 128)])
    stream = torch.cuda.Stream()
    out = sep.alloc_outputs(F, KCAP, PCAP)
    with torch.cuda.stream(stream):
        sep.process_batch(dev, KCAP, PCAP, out=out, use_graph=True, stream=stream)
        sep.process_batch(dev, KCAP, PCAP, out=out, use_graph=True, stream=stream)   # graph replay
    torch.cuda.synchronize()
    assert sep.device_status() == 0
    o = {k: v.cpu().numpy() for k, v in out.items()}
    # every frame: counts within the row sizes, kept lists ascending and
    # inside the detector, kept values above their bin's threshold band
    assert np.all(o["n_kept"] >= 0) and np.all(o["n_kept"] <= KCAP)
    assert np.all(o["n_peaks"] >= 0) and np.all(o["n_peaks"] <= PCAP)
    assert np.all(np.isfinite(o["mean"])) and np.all(o["sigma"] >= 0)
    W = oracle.weights(det, mask)
    bop = np.asarray(W.bin_of_pixel)
    for f in range(F):
        idx = o["idx"][f, : o["n_kept"][f]]
        assert np.all(np.diff(idx) > 0) and (idx.size == 0 or (idx[0] >= 0 and idx[-1] < det.npix))
        b = bop[idx]
        assert np.all(b >= 0)
        thr = o["mean"][f, b].astype(np.float64) + 3.0 * o["sigma"][f, b].astype(np.float64)
        assert np.all(o["val"][f, : o["n_kept"][f]] > thr - 1e-5 * np.abs(thr) - 1e-6)
        pk = o["peaks"][f, : o["n_peaks"][f], 0]
        assert np.all(np.isin(pk, idx))
    # sampled frames against the oracle, with the GPU's final intervals for
    # bins decided inside the rounding band
    for f in SAMPLED:
        bnd = sep.integrate_clip(dev[f:f + 1], bounds=True)["bounds"].cpu().numpy()[0]
        sig = oracle.jf_photons(frames[f], cal[0], cal[1])
        check_frame(det, W, sig, o, f, kcap=KCAP, bounds=bnd)
