"""Sanity of the seeded input generator (it holds no method arithmetic)."""
import numpy as np

import synth


def test_jungfrau_layouts():
    for det, nv in ((synth.det_jf4m(), 4194304), (synth.det_jf1m(), 1048576), (synth.det_jf16m(), 16777216)):
        m = det.mask()
        assert (m == 0).sum() == nv
    assert synth.det_jf4m().npix == 2164 * 2068 == 4475152


def test_frames_are_pure_functions_of_seed_and_index():
    d = synth.det_small_jf()
    m = d.mask()
    cal = synth.jf_calib(d.npix, seed=5)
    a, _, _ = synth.frames(d, synth.spec_jf_serial(3), 10, 3, calib=cal, mask=m)
    b, _, _ = synth.frames(d, synth.spec_jf_serial(3), 11, 1, calib=cal, mask=m)
    assert np.array_equal(a[1], b[0])
    c, _, _ = synth.frames(d, synth.spec_jf_serial(4), 10, 1, calib=cal, mask=m)
    assert not np.array_equal(a[0], c[0])
    assert np.all(a[:, m == 1] == 0)


def test_philox_uniformity():
    u = np.array([synth.philox([i, 0, 0, 0], [1, 2]) for i in range(4000)]).ravel() / 2.0 ** 32
    assert abs(u.mean() - 0.5) < 0.01 and abs(u.var() - 1 / 12) < 0.005
