"""The allocation-free sparsification entry point, through the C ABI.

sep_sparsify_noalloc serves callers that must not allocate device memory at
call time (real-time acquisition threads, fixed device-memory budgets): it
runs sep_sparsify's checks and kernels with scratch in a static device
array. This file is collected last on purpose, so that a stop-at-first-
failure run has already run every other test.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2411_09515_gb300 import Separator, SepError, _binding as B  # noqa: E402


def _frames(det, seeds, raw=False, cal=None, mask=None):
    if raw:
        spec = synth.spec_jf_serial(seeds[0])
        spec.hit_rate = 1.0
        fr = synth.frames(det, spec, 0, len(seeds), calib=cal, mask=mask)[0]
        return torch.from_numpy(fr.view(np.int16)).cuda()
    return torch.from_numpy(np.concatenate([synth.frames(det, synth.spec_config1(s), 0, 1)[0] for s in seeds])).cuda()


@pytest.mark.parametrize("raw", [False, True])
def test_noalloc_matches_sparsify_twice(raw):
    if raw:
        det = synth.det_small_jf(split=2, nbins=200)
        mask = det.mask()
        cal = synth.jf_calib(det.npix, seed=3)
        sep = Separator.from_detector(det, mask=mask, calib=cal)
        fr = _frames(det, [5, 6, 7], raw=True, cal=cal, mask=mask)
        dtype = B.SEP_DTYPE_U16_JF
    else:
        det = synth.det_config1()
        sep = Separator.from_detector(det)
        fr = _frames(det, [1, 2, 3, 4])
        dtype = B.SEP_DTYPE_F32
    F = fr.shape[0]
    cap = det.npix // 8
    ic = sep.integrate_clip(fr)
    ref = sep.sparsify(fr, ic["mean"], ic["sigma"], cap)
    torch.cuda.synchronize()
    want_n = ref["n_kept"].cpu().numpy()
    for call in range(2):
        idx = torch.full((F, cap), -7, dtype=torch.int32, device="cuda")
        val = torch.full((F, cap), -7.0, dtype=torch.float32, device="cuda")
        nk = torch.full((F,), -7, dtype=torch.int32, device="cuda")
        B.sep_sparsify_noalloc(sep.ctx, sep.csr, sep.calib, fr, dtype, F, sep.params, ic["mean"], ic["sigma"], idx,
                               val, cap, nk)
        torch.cuda.synchronize()
        got_n = nk.cpu().numpy()
        assert np.array_equal(got_n, want_n), call
        for f in range(F):
            n = int(want_n[f])
            assert np.array_equal(idx[f, :n].cpu().numpy(), ref["idx"][f, :n].cpu().numpy()), (call, f)
            # same kernels on the same inputs: values agree bit for bit
            assert np.array_equal(val[f, :n].cpu().numpy(), ref["val"][f, :n].cpu().numpy()), (call, f)
    assert sep.device_status() == 0


def test_noalloc_rejects_batches_beyond_the_static_scratch():
    det = synth.det_jf4m(split=1, nbins=100)
    mask = det.mask()
    sep = Separator.from_detector(det, mask=mask)
    F = 64   # 64 x 0.56 MB of bitmap alone exceeds 16 MiB
    fr = torch.zeros((F, det.npix), dtype=torch.float32, device="cuda")
    mean = torch.zeros((F, det.nbins), dtype=torch.float32, device="cuda")
    idx = torch.zeros((F, 16), dtype=torch.int32, device="cuda")
    val = torch.zeros((F, 16), dtype=torch.float32, device="cuda")
    nk = torch.zeros((F,), dtype=torch.int32, device="cuda")
    with pytest.raises(SepError) as e:
        B.sep_sparsify_noalloc(sep.ctx, sep.csr, None, fr, B.SEP_DTYPE_F32, F, sep.params, mean, mean, idx, val, 16,
                               nk)
    assert e.value.status == B.SEP_ERR_ARG and "static array" in str(e.value)


def test_noalloc_allocates_nothing_where_sparsify_grows_its_scratch():
    """Free device memory is unchanged across a call on a batch larger than
    any the context has seen; sep_sparsify on the same batch grows the
    context's scratch (so the measurement can see an allocation)."""
    det = synth.det_config1()
    sep = Separator.from_detector(det)
    small, big = _frames(det, [1]), _frames(det, [1, 2, 3, 4, 5, 6, 7, 8] * 8)
    cap = det.npix // 8

    def outputs(F):
        return (torch.empty((F, cap), dtype=torch.int32, device="cuda"),
                torch.empty((F, cap), dtype=torch.float32, device="cuda"),
                torch.empty((F,), dtype=torch.int32, device="cuda"))

    ic_s, ic_b = sep.integrate_clip(small), sep.integrate_clip(big)
    o_s, o_b = outputs(small.shape[0]), outputs(big.shape[0])
    # first call: the library's module and its static array are loaded
    B.sep_sparsify_noalloc(sep.ctx, sep.csr, None, small, B.SEP_DTYPE_F32, small.shape[0], sep.params,
                           ic_s["mean"], ic_s["sigma"], *o_s[:2], cap, o_s[2])
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    B.sep_sparsify_noalloc(sep.ctx, sep.csr, None, big, B.SEP_DTYPE_F32, big.shape[0], sep.params,
                           ic_b["mean"], ic_b["sigma"], *o_b[:2], cap, o_b[2])
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    # the measurement sees an allocation: sep_sparsify on a batch whose
    # scratch (8 MiB of bitmap) exceeds the driver's 2 MiB allocation granule
    huge = big.repeat(16, 1)
    ic_h = sep.integrate_clip(huge)
    o_h = outputs(huge.shape[0])
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    B.sep_sparsify(sep.ctx, sep.csr, None, huge, B.SEP_DTYPE_F32, huge.shape[0], sep.params, ic_h["mean"],
                   ic_h["sigma"], *o_h[:2], cap, o_h[2])
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] < free1
    assert sep.device_status() == 0


def test_noalloc_refuses_the_params_sparsify_refuses():
    det = synth.det_config1()
    sep = Separator.from_detector(det)
    fr = _frames(det, [1])
    ic = sep.integrate_clip(fr)
    idx = torch.zeros((1, 16), dtype=torch.int32, device="cuda")
    val = torch.zeros((1, 16), dtype=torch.float32, device="cuda")
    nk = torch.zeros((1,), dtype=torch.int32, device="cuda")
    for field, bad in (("n_iter", -1), ("k_clip", 0.0), ("patch", 4), ("precision", 99)):
        p = B.make_params(sep.params.n_iter, sep.params.k_clip, sep.params.k_pick, sep.params.patch,
                          sep.params.min_count, sep.params.precision)
        setattr(p, field, bad)
        for fn in (B.sep_sparsify, B.sep_sparsify_noalloc):
            with pytest.raises(SepError) as e:
                fn(sep.ctx, sep.csr, None, fr, B.SEP_DTYPE_F32, 1, p, ic["mean"], ic["sigma"], idx, val, 16, nk)
            assert e.value.status == B.SEP_ERR_ARG, (field, fn.__name__)
