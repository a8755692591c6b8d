"""ctypes binding of libsep (include/sep.h): argument marshalling only.

Every function here has the name of the C entry point it calls. Device
buffers are torch CUDA tensors (PyTorch provides memory and streams); their
pointers and the current stream are passed straight to the library. Nothing
here computes anything of the path: a missing library raises instead of
falling back.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsep.so")

SEP_OK, SEP_ERR_ARG, SEP_ERR_CUDA, SEP_ERR_OOM, SEP_ERR_CAPACITY, SEP_ERR_TIMEOUT, SEP_ERR_CSR, SEP_ERR_STATE = range(8)
SEP_DEV_CAPACITY, SEP_DEV_TIMEOUT = 0x1, 0x2
SEP_UNIT_2TH_DEG, SEP_UNIT_Q_NM, SEP_UNIT_R_MM = 0, 1, 2
SEP_DTYPE_F32, SEP_DTYPE_U16_JF = 0, 1
SEP_PREC_PLAIN, SEP_PREC_KAHAN, SEP_PREC_FP64MERGE, SEP_PREC_DWORD = 0, 1, 2, 3
SEP_CUTOFF_FIXED, SEP_CUTOFF_CHAUVENET = 0, 1
SEP_ERROR_AZIMUTHAL, SEP_ERROR_POISSON, SEP_ERROR_HYBRID = 0, 1, 2
SEP_MAX_PIXELS, SEP_MAX_BINS, SEP_MAX_FRAMES = 1 << 25, 32767, 65535

STATUS_NAMES = {0: "SEP_OK", 1: "SEP_ERR_ARG", 2: "SEP_ERR_CUDA", 3: "SEP_ERR_OOM", 4: "SEP_ERR_CAPACITY",
                5: "SEP_ERR_TIMEOUT", 6: "SEP_ERR_CSR", 7: "SEP_ERR_STATE"}

# every symbol include/sep.h declares
EXPORTS = ["sep_version", "sep_ctx_create", "sep_ctx_destroy", "sep_last_error", "sep_get_device_status",
           "sep_build_csr", "sep_csr_destroy", "sep_csr_info", "sep_csr_export", "sep_calib_create",
           "sep_calib_destroy", "sep_integrate_clip", "sep_sparsify", "sep_peakfind", "sep_process_batch",
           "sep_sparsify_noalloc", "sep_csr_set_plan", "sep_csr_get_plan", "sep_autotune", "sep_process_mixed",
           "sep_model_create", "sep_model_destroy", "sep_model_params", "sep_model_norm", "sep_mlp_forward",
           "sep_mlp_loss_grad", "sep_surrogate_train", "sep_model_save", "sep_model_load", "sep_csr_attach_model",
           "sep_surrogate_record", "sep_surrogate_prepare", "sep_surrogate_stats", "sep_csr_staging", "sep_correct",
           "sep_process_host", "sep_densify", "sep_veto", "sep_compact_frames", "sep_csr_interp", "sep_clip_stats",
           "sep_csr_validate", "sep_csr_check"]

SEP_MLP_IN, SEP_MLP_HIDDEN, SEP_MLP_OUT, SEP_MLP_PARAMS, SEP_MLP_NORM = 20, 64, 2, 5634, 44
SEP_CLIP_STATS = 8


class SepError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class sep_geometry(C.Structure):
    _fields_ = [("rows", C.c_int32), ("cols", C.c_int32), ("pixel_m", C.c_double * 2), ("dist_m", C.c_double),
                ("center_px", C.c_double * 2), ("wavelength_m", C.c_double), ("unit", C.c_int32),
                ("nbins", C.c_int32), ("split", C.c_int32), ("range", C.c_double * 2)]


class sep_params(C.Structure):
    _fields_ = [("n_iter", C.c_int32), ("k_clip", C.c_float), ("k_pick", C.c_float), ("patch", C.c_int32),
                ("min_count", C.c_int32), ("precision", C.c_int32), ("surrogate", C.c_int32),
                ("cutoff", C.c_int32), ("error_model", C.c_int32), ("dark_var", C.c_float),
                ("interpolate", C.c_int32)]


class sep_train_cfg(C.Structure):
    _fields_ = [("epochs", C.c_int32), ("batch", C.c_int32), ("lr", C.c_float), ("pad", C.c_int32),
                ("seed", C.c_uint64)]


class sep_frame_desc(C.Structure):
    _fields_ = [("det", C.c_int32), ("dtype", C.c_int32), ("frame_dev", C.c_void_p)]


PEAK_DTYPE = np.dtype([("idx", "<i4"), ("y", "<f4"), ("x", "<f4"), ("I", "<f4"), ("sigma", "<f4"), ("npix", "<i4")])
PEAK_BYTES = 24

_vp = C.c_void_p
_lib = None


def lib():
    """Load libsep.so (built in-tree by __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libsep.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    L.sep_version.restype = C.c_char_p
    L.sep_ctx_create.argtypes = [C.c_int32, C.POINTER(_vp)]
    L.sep_ctx_destroy.argtypes = [_vp]
    L.sep_ctx_destroy.restype = None
    L.sep_last_error.argtypes = [_vp]
    L.sep_last_error.restype = C.c_char_p
    L.sep_get_device_status.argtypes = [_vp, _vp, C.POINTER(C.c_int32)]
    L.sep_build_csr.argtypes = [_vp, C.POINTER(sep_geometry), _vp, _vp, C.POINTER(_vp)]
    L.sep_csr_destroy.argtypes = [_vp]
    L.sep_csr_destroy.restype = None
    L.sep_csr_info.argtypes = [_vp, C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.POINTER(C.c_int64),
                               C.POINTER(C.c_int32), C.POINTER(C.c_double)]
    L.sep_csr_export.argtypes = [_vp] * 6
    L.sep_csr_validate.argtypes = [_vp, _vp, _vp, _vp, C.c_int32, C.c_int64, C.c_int64, C.c_int64, C.c_char_p,
                                   C.c_int32]
    L.sep_csr_check.argtypes = [_vp, _vp]
    L.sep_calib_create.argtypes = [_vp, _vp, _vp, _vp, C.POINTER(_vp)]
    L.sep_calib_destroy.argtypes = [_vp]
    L.sep_calib_destroy.restype = None
    L.sep_integrate_clip.argtypes = [_vp, _vp, _vp, _vp, C.c_int32, C.c_int32, C.POINTER(sep_params), _vp, _vp, _vp,
                                     _vp, _vp, _vp]
    L.sep_sparsify.argtypes = [_vp, _vp, _vp, _vp, C.c_int32, C.c_int32, C.POINTER(sep_params), _vp, _vp, _vp, _vp,
                               C.c_int64, _vp, _vp]
    L.sep_sparsify_noalloc.argtypes = [_vp, _vp, _vp, _vp, C.c_int32, C.c_int32, C.POINTER(sep_params), _vp, _vp, _vp,
                                       _vp, C.c_int64, _vp, _vp]
    L.sep_csr_set_plan.argtypes = [_vp, _vp, C.c_int32, _vp, _vp]
    L.sep_csr_get_plan.argtypes = [_vp, _vp, _vp, _vp]
    L.sep_autotune.argtypes = [_vp, _vp, _vp, _vp, C.c_int32, C.c_int32, C.POINTER(sep_params), C.c_char_p,
                               C.POINTER(C.c_float), _vp]
    L.sep_process_mixed.argtypes = [_vp, C.c_int32, _vp, _vp, _vp, C.c_int32, C.POINTER(sep_params), _vp, _vp, _vp,
                                    _vp, _vp, _vp, C.c_int64, _vp, _vp, C.c_int64, _vp, C.c_int32, _vp]
    L.sep_peakfind.argtypes = [_vp, _vp, _vp, _vp, C.c_int32, C.c_int32, C.POINTER(sep_params), _vp, _vp, _vp, _vp,
                               C.c_int64, _vp, C.c_int64, _vp, _vp]
    L.sep_veto.argtypes = [_vp, C.c_int32, _vp, C.c_int32, _vp, _vp, _vp]
    L.sep_compact_frames.argtypes = [_vp, C.c_int32, _vp, _vp, C.c_int64, _vp, _vp, _vp]
    L.sep_densify.argtypes = [_vp, _vp, C.c_int32, _vp, _vp, _vp, _vp, C.c_int64, _vp, _vp, C.c_float, C.c_int32,
                              _vp, _vp]
    L.sep_process_batch.argtypes = [_vp, _vp, _vp, _vp, C.c_int32, C.c_int32, C.POINTER(sep_params), _vp, _vp, _vp,
                                    _vp, _vp, C.c_int64, _vp, _vp, C.c_int64, _vp, C.c_int32, _vp]
    L.sep_model_create.argtypes = [_vp, C.c_uint64, C.POINTER(_vp)]
    L.sep_model_destroy.argtypes = [_vp]
    L.sep_model_destroy.restype = None
    L.sep_model_params.argtypes = [_vp, _vp, _vp]
    L.sep_model_norm.argtypes = [_vp, _vp, _vp]
    L.sep_mlp_forward.argtypes = [_vp, _vp, C.c_int64, _vp, _vp]
    L.sep_mlp_loss_grad.argtypes = [_vp, _vp, _vp, C.c_int64, _vp, _vp, _vp]
    L.sep_surrogate_train.argtypes = [_vp, _vp, _vp, C.c_int64, C.POINTER(sep_train_cfg), C.POINTER(C.c_float), _vp]
    L.sep_model_save.argtypes = [_vp, C.c_char_p]
    L.sep_model_load.argtypes = [_vp, C.c_char_p, C.POINTER(_vp)]
    L.sep_csr_attach_model.argtypes = [_vp, _vp]
    L.sep_csr_staging.argtypes = [_vp, _vp, C.POINTER(C.c_int64)]
    L.sep_correct.argtypes = [_vp, _vp, _vp, _vp, C.c_int32, C.c_int32, _vp, _vp]
    L.sep_process_host.argtypes = [_vp, _vp, _vp, _vp, C.c_int32, C.c_int32, C.POINTER(sep_params), _vp, _vp, _vp,
                                   _vp, _vp, C.c_int64, _vp, _vp, C.c_int64, _vp, C.c_int32, _vp]
    L.sep_surrogate_record.argtypes = [_vp, _vp, _vp, _vp, C.c_int32, C.c_int32, C.POINTER(sep_params), _vp, _vp,
                                       _vp, _vp, _vp, _vp]
    L.sep_surrogate_prepare.argtypes = [_vp, _vp, _vp, C.c_int64, _vp, _vp, _vp, C.POINTER(C.c_int64), _vp]
    L.sep_surrogate_stats.argtypes = [_vp, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), C.c_int32, _vp]
    L.sep_clip_stats.argtypes = [_vp, C.c_int32, C.POINTER(C.c_uint64), C.c_int32, _vp]
    for name in EXPORTS:
        f = getattr(L, name)
        if name not in ("sep_version", "sep_last_error", "sep_ctx_destroy", "sep_csr_destroy", "sep_calib_destroy",
                        "sep_model_destroy"):
            f.restype = C.c_int32
    _lib = L
    return L


def _ptr(t):
    """Device (or host) address of a torch tensor / numpy array, or None."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(_vp)
    return _vp(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return _vp(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _check(ctx, st):
    if st != SEP_OK:
        msg = lib().sep_last_error(ctx).decode() if ctx else ""
        raise SepError(st, msg)


def sep_version() -> str:
    return lib().sep_version().decode()


def sep_ctx_create(device: int = 0):
    h = _vp()
    st = lib().sep_ctx_create(device, C.byref(h))
    if st != SEP_OK:
        raise SepError(st, f"cannot create a context on device {device}")
    return h


def sep_ctx_destroy(ctx):
    lib().sep_ctx_destroy(ctx)


def sep_last_error(ctx) -> str:
    return lib().sep_last_error(ctx).decode()


def sep_get_device_status(ctx, stream=None) -> int:
    v = C.c_int32(0)
    _check(ctx, lib().sep_get_device_status(ctx, _stream(stream), C.byref(v)))
    return v.value


def make_geometry(rows, cols, pixel_m, dist_m, center_px, wavelength_m, unit, nbins, split, rng):
    g = sep_geometry()
    g.rows, g.cols = rows, cols
    g.pixel_m[0], g.pixel_m[1] = pixel_m
    g.dist_m = dist_m
    g.center_px[0], g.center_px[1] = center_px
    g.wavelength_m = wavelength_m
    g.unit, g.nbins, g.split = unit, nbins, split
    g.range[0], g.range[1] = rng
    return g


def make_params(n_iter=5, k_clip=3.0, k_pick=3.0, patch=3, min_count=3, precision=SEP_PREC_DWORD, surrogate=0,
                cutoff=SEP_CUTOFF_FIXED, interpolate=0):
    p = sep_params()
    p.n_iter, p.k_clip, p.k_pick, p.patch, p.min_count, p.precision = n_iter, k_clip, k_pick, patch, min_count, precision
    p.surrogate = surrogate
    p.cutoff = cutoff
    p.interpolate = interpolate
    return p


def sep_build_csr(ctx, geom: sep_geometry, mask=None, norm=None):
    h = _vp()
    m = None if mask is None else np.ascontiguousarray(mask, np.uint8)
    n = None if norm is None else np.ascontiguousarray(norm, np.float32)
    _check(ctx, lib().sep_build_csr(ctx, C.byref(geom), _ptr(m), _ptr(n), C.byref(h)))
    return h


def sep_csr_destroy(csr):
    lib().sep_csr_destroy(csr)


def sep_csr_info(csr):
    npix, nnz = C.c_int64(), C.c_int64()
    nbins, max_row = C.c_int32(), C.c_int32()
    rng = (C.c_double * 2)()
    st = lib().sep_csr_info(csr, C.byref(npix), C.byref(nbins), C.byref(nnz), C.byref(max_row), rng)
    if st != SEP_OK:
        raise SepError(st, "sep_csr_info")
    return {"npix": npix.value, "nbins": nbins.value, "nnz": nnz.value, "max_row": max_row.value,
            "range": (rng[0], rng[1])}


def sep_csr_export(csr):
    info = sep_csr_info(csr)
    rowptr = np.zeros(info["nbins"] + 1, np.int32)
    col = np.zeros(info["nnz"], np.int32)
    coef = np.zeros(info["nnz"], np.float32)
    bop = np.zeros(info["npix"], np.int32)
    centers = np.zeros(info["nbins"], np.float32)
    st = lib().sep_csr_export(csr, _ptr(rowptr), _ptr(col), _ptr(coef), _ptr(bop), _ptr(centers))
    if st != SEP_OK:
        raise SepError(st, "sep_csr_export")
    return {"rowptr": rowptr, "col": col, "coef": coef, "bin_of_pixel": bop, "bin_centers": centers, **info}


def sep_csr_validate(rowptr, col, coef, bin_of_pixel, npix, calib_npix=-1):
    """Host-side check of a matrix in the export layout: (status, reason)."""
    rp = np.ascontiguousarray(rowptr, np.int32)
    cl = np.ascontiguousarray(col, np.int32)
    cf = np.ascontiguousarray(coef, np.float32)
    bp = None if bin_of_pixel is None else np.ascontiguousarray(bin_of_pixel, np.int32)
    if cl.size != cf.size:
        raise ValueError("col and coef differ in size")
    msg = C.create_string_buffer(256)
    st = lib().sep_csr_validate(_ptr(rp), _ptr(cl), _ptr(cf), _ptr(bp), rp.size - 1, cl.size, int(npix),
                                int(calib_npix), msg, len(msg))
    return st, msg.value.decode()


def sep_csr_check(csr, calib=None):
    """The matrix checks on a built handle (and the calibration's size)."""
    return lib().sep_csr_check(csr, calib)


def sep_calib_create(ctx, csr, ped, gain):
    h = _vp()
    p = np.ascontiguousarray(ped, np.float32)
    g = np.ascontiguousarray(gain, np.float32)
    _check(ctx, lib().sep_calib_create(ctx, csr, _ptr(p), _ptr(g), C.byref(h)))
    return h


def sep_calib_destroy(calib):
    lib().sep_calib_destroy(calib)


def sep_integrate_clip(ctx, csr, calib, frames, dtype, n_frames, params, mean, sigma, count, bounds=None, iters=None,
                       stream=None):
    _check(ctx, lib().sep_integrate_clip(ctx, csr, calib, _ptr(frames), dtype, n_frames, C.byref(params), _ptr(mean),
                                         _ptr(sigma), _ptr(count), _ptr(bounds), _ptr(iters), _stream(stream)))


def sep_sparsify(ctx, csr, calib, frames, dtype, n_frames, params, mean, sigma, idx, val, capacity, n_kept,
                 stream=None):
    _check(ctx, lib().sep_sparsify(ctx, csr, calib, _ptr(frames), dtype, n_frames, C.byref(params), _ptr(mean),
                                   _ptr(sigma), _ptr(idx), _ptr(val), capacity, _ptr(n_kept), _stream(stream)))


def sep_sparsify_noalloc(ctx, csr, calib, frames, dtype, n_frames, params, mean, sigma, idx, val, capacity, n_kept,
                         stream=None):
    _check(ctx, lib().sep_sparsify_noalloc(ctx, csr, calib, _ptr(frames), dtype, n_frames, C.byref(params),
                                           _ptr(mean), _ptr(sigma), _ptr(idx), _ptr(val), capacity, _ptr(n_kept),
                                           _stream(stream)))


def sep_csr_set_plan(ctx, csr, tpb, thresholds=()):
    t = np.ascontiguousarray(list(thresholds) + [0] * (4 - len(thresholds)), np.int32)
    b = np.ascontiguousarray(list(tpb) + [256] * (4 - len(tpb)), np.int32)
    _check(ctx, lib().sep_csr_set_plan(ctx, csr, len(tpb), _ptr(t), _ptr(b)))


def sep_csr_get_plan(csr):
    n = np.zeros(1, np.int32)
    t = np.zeros(4, np.int32)
    b = np.zeros(4, np.int32)
    st = lib().sep_csr_get_plan(csr, _ptr(n), _ptr(t), _ptr(b))
    if st != SEP_OK:
        raise SepError(st, "sep_csr_get_plan")
    k = int(n[0])
    return {"tpb": b[:k].tolist(), "thresholds": t[: k - 1].tolist()}


def sep_autotune(ctx, csr, calib, frames, dtype, n_frames, params, cache_path=None, stream=None):
    ms = C.c_float(0)
    _check(ctx, lib().sep_autotune(ctx, csr, calib, _ptr(frames), dtype, n_frames, C.byref(params),
                                   None if cache_path is None else str(cache_path).encode(), C.byref(ms),
                                   _stream(stream)))
    return ms.value


def sep_process_mixed(ctx, csrs, calibs, descs, params, mean, sigma, count, idx, val, kept_capacity, n_kept, peaks,
                      peak_capacity, n_peaks, use_graph=1, stream=None):
    """descs: list of (det, dtype, device tensor). Returns the row offsets (numpy int64)."""
    n = len(descs)
    D = (sep_frame_desc * max(n, 1))()
    for i, (d, dt, t) in enumerate(descs):
        D[i].det, D[i].dtype, D[i].frame_dev = d, dt, t.data_ptr()
    cs = (C.c_void_p * len(csrs))(*[c.value if hasattr(c, "value") else c for c in csrs])
    ks = (C.c_void_p * len(csrs))(*[(k.value if hasattr(k, "value") else k) if k is not None else None
                                    for k in calibs])
    rows = np.zeros(n + 1, np.int64)
    _check(ctx, lib().sep_process_mixed(ctx, len(csrs), cs, ks, D, n, C.byref(params), _ptr(mean), _ptr(sigma),
                                        _ptr(count), _ptr(rows), _ptr(idx), _ptr(val), kept_capacity, _ptr(n_kept),
                                        _ptr(peaks), peak_capacity, _ptr(n_peaks), int(use_graph), _stream(stream)))
    return rows


def sep_peakfind(ctx, csr, calib, frames, dtype, n_frames, params, mean, sigma, idx, n_kept, kept_capacity, peaks,
                 capacity, n_peaks, stream=None):
    _check(ctx, lib().sep_peakfind(ctx, csr, calib, _ptr(frames), dtype, n_frames, C.byref(params), _ptr(mean),
                                   _ptr(sigma), _ptr(idx), _ptr(n_kept), kept_capacity, _ptr(peaks), capacity,
                                   _ptr(n_peaks), _stream(stream)))


def sep_veto(ctx, n_frames, n_peaks, min_peaks, frame_list, n_pass, stream=None):
    _check(ctx, lib().sep_veto(ctx, n_frames, _ptr(n_peaks), int(min_peaks), _ptr(frame_list), _ptr(n_pass),
                               _stream(stream)))


def sep_compact_frames(ctx, n_frames, frame_list, n_pass, row_bytes, src, dst, stream=None):
    _check(ctx, lib().sep_compact_frames(ctx, n_frames, _ptr(frame_list), _ptr(n_pass), int(row_bytes), _ptr(src),
                                         _ptr(dst), _stream(stream)))


def sep_densify(ctx, csr, n_frames, mean, sigma, idx, val, kept_capacity, n_kept, noise, fill, out, interpolate=0,
                stream=None):
    _check(ctx, lib().sep_densify(ctx, csr, n_frames, _ptr(mean), _ptr(sigma), _ptr(idx), _ptr(val), kept_capacity,
                                  _ptr(n_kept), _ptr(noise), C.c_float(fill), int(interpolate), _ptr(out),
                                  _stream(stream)))


def sep_process_batch(ctx, csr, calib, frames, dtype, n_frames, params, mean, sigma, count, idx, val, kept_capacity,
                      n_kept, peaks, peak_capacity, n_peaks, use_graph=1, stream=None):
    _check(ctx, lib().sep_process_batch(ctx, csr, calib, _ptr(frames), dtype, n_frames, C.byref(params), _ptr(mean),
                                        _ptr(sigma), _ptr(count), _ptr(idx), _ptr(val), kept_capacity, _ptr(n_kept),
                                        _ptr(peaks), peak_capacity, _ptr(n_peaks), int(use_graph), _stream(stream)))


# ---- surrogate ----

def sep_model_create(ctx, seed=0):
    h = _vp()
    _check(ctx, lib().sep_model_create(ctx, seed, C.byref(h)))
    return h


def sep_model_destroy(model):
    lib().sep_model_destroy(model)


def sep_model_params(ctx, model, set_host=None):
    """Returns the parameters (float32 [5634]); sets them first if set_host is given."""
    out = np.zeros(SEP_MLP_PARAMS, np.float32)
    src = None if set_host is None else np.ascontiguousarray(set_host, np.float32)
    _check(ctx, lib().sep_model_params(model, _ptr(out), _ptr(src)))
    return out


def sep_model_norm(ctx, model, set_host=None):
    out = np.zeros(SEP_MLP_NORM, np.float32)
    src = None if set_host is None else np.ascontiguousarray(set_host, np.float32)
    _check(ctx, lib().sep_model_norm(model, _ptr(out), _ptr(src)))
    return out


def sep_mlp_forward(ctx, model, x, n, y, stream=None):
    _check(ctx, lib().sep_mlp_forward(model, _ptr(x), n, _ptr(y), _stream(stream)))


def sep_mlp_loss_grad(ctx, model, x, t, n, grad, loss, stream=None):
    _check(ctx, lib().sep_mlp_loss_grad(model, _ptr(x), _ptr(t), n, _ptr(grad), _ptr(loss), _stream(stream)))


def sep_surrogate_train(ctx, model, x, t, n, epochs=4, batch=4096, lr=2e-3, seed=0, stream=None):
    cfg = sep_train_cfg()
    cfg.epochs, cfg.batch, cfg.lr, cfg.seed = epochs, batch, lr, seed
    loss = C.c_float(0.0)
    _check(ctx, lib().sep_surrogate_train(model, _ptr(x), _ptr(t), n, C.byref(cfg), C.byref(loss), _stream(stream)))
    return loss.value


def sep_model_save(ctx, model, path):
    _check(ctx, lib().sep_model_save(model, os.fsencode(path)))


def sep_model_load(ctx, path):
    h = _vp()
    _check(ctx, lib().sep_model_load(ctx, os.fsencode(path), C.byref(h)))
    return h


def sep_csr_attach_model(ctx, csr, model):
    _check(ctx, lib().sep_csr_attach_model(csr, model))


def sep_surrogate_record(ctx, csr, calib, frames, dtype, n_frames, params, mean, sigma, count, feat, target,
                         stream=None):
    _check(ctx, lib().sep_surrogate_record(ctx, csr, calib, _ptr(frames), dtype, n_frames, C.byref(params),
                                           _ptr(mean), _ptr(sigma), _ptr(count), _ptr(feat), _ptr(target),
                                           _stream(stream)))


def sep_surrogate_prepare(ctx, feat, target, n, x, t, stream=None):
    """Returns (normalisation block float32 [44], number of kept rows)."""
    norm = np.zeros(SEP_MLP_NORM, np.float32)
    nv = C.c_int64(0)
    _check(ctx, lib().sep_surrogate_prepare(ctx, _ptr(feat), _ptr(target), n, _ptr(x), _ptr(t), _ptr(norm),
                                            C.byref(nv), _stream(stream)))
    return norm, nv.value


def sep_surrogate_stats(ctx, reset=False, stream=None):
    a, b = C.c_uint64(0), C.c_uint64(0)
    _check(ctx, lib().sep_surrogate_stats(ctx, C.byref(a), C.byref(b), int(reset), _stream(stream)))
    return a.value, b.value


CLIP_STATS_NAMES = ("items", "core_scans", "overflows", "replay_steps", "tail_entries", "tail_marked",
                    "full_passes", "reserved")


def sep_clip_stats(ctx, enable=-1, read=True, reset=False, stream=None):
    """Tail-replay counters of the clip kernel (a dict when read, else None);
    enable 1 / 0 switches collection for later calls, -1 leaves it."""
    buf = (C.c_uint64 * SEP_CLIP_STATS)()
    _check(ctx, lib().sep_clip_stats(ctx, int(enable), buf if read else None, int(reset), _stream(stream)))
    return dict(zip(CLIP_STATS_NAMES, (int(x) for x in buf))) if read else None


def sep_csr_staging(csr):
    """Pixel of every staging position (int32 [npos])."""
    n = C.c_int64(0)
    st = lib().sep_csr_staging(csr, None, C.byref(n))
    if st != SEP_OK:
        raise SepError(st, "sep_csr_staging")
    out = np.zeros(max(n.value, 1), np.int32)
    lib().sep_csr_staging(csr, _ptr(out), C.byref(n))
    return out[: n.value]


def sep_csr_interp(csr):
    """Interpolation table of the smooth background: lower bin (int32 [npix])
    and weight of the upper bin (float32 [npix])."""
    npix = C.c_int64()
    st = lib().sep_csr_info(csr, C.byref(npix), None, None, None, None)
    if st != SEP_OK:
        raise SepError(st, "sep_csr_info")
    a = np.zeros(npix.value, np.int32)
    t = np.zeros(npix.value, np.float32)
    st = lib().sep_csr_interp(csr, _ptr(a), _ptr(t))
    if st != SEP_OK:
        raise SepError(st, "sep_csr_interp")
    return a, t


def sep_correct(ctx, csr, calib, frames, dtype, n_frames, out, stream=None):
    _check(ctx, lib().sep_correct(ctx, csr, calib, _ptr(frames), dtype, n_frames, _ptr(out), _stream(stream)))


def sep_process_host(ctx, csr, calib, frames_host, dtype, n_frames, params, mean, sigma, count, idx, val,
                     kept_capacity, n_kept, peaks, peak_capacity, n_peaks, chunk_frames=0, stream=None):
    _check(ctx, lib().sep_process_host(ctx, csr, calib, _ptr(frames_host), dtype, n_frames, C.byref(params),
                                       _ptr(mean), _ptr(sigma), _ptr(count), _ptr(idx), _ptr(val), kept_capacity,
                                       _ptr(n_kept), _ptr(peaks), peak_capacity, _ptr(n_peaks), int(chunk_frames),
                                       _stream(stream)))
