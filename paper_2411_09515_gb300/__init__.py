"""GB300-native signal separation for diffraction frames (arXiv 2411.09515).

The compute path lives in ``libsep.so`` (hand-written CUDA for sm_103a behind
the C ABI of ``include/sep.h``); this package is the thin Python face of it:
``_binding`` marshals arguments to the C entry points, and :class:`Separator`
owns the handles and allocates output tensors with PyTorch.

Per frame (Kieffer et al., Sections 2-4): Jungfrau correction, CSR
azimuthal integration with weighted moments, iterative sigma-clipping,
sparsification and peak picking.
"""
from __future__ import annotations

import numpy as np

from . import _binding as B
from ._binding import (PEAK_DTYPE, SEP_CUTOFF_CHAUVENET, SEP_CUTOFF_FIXED, SEP_DTYPE_F32, SEP_DTYPE_U16_JF,
                       SEP_ERROR_AZIMUTHAL, SEP_ERROR_HYBRID, SEP_ERROR_POISSON,
                       SEP_PREC_DWORD, SEP_PREC_FP64MERGE, SEP_PREC_KAHAN, SEP_PREC_PLAIN, SEP_UNIT_2TH_DEG,
                       SEP_UNIT_Q_NM, SEP_UNIT_R_MM, SepError)

__all__ = ["Context", "Separator", "Surrogate", "process_mixed", "SepError", "PEAK_DTYPE", "peaks_to_numpy", "SEP_DTYPE_F32", "SEP_DTYPE_U16_JF",
           "SEP_PREC_PLAIN", "SEP_PREC_KAHAN", "SEP_PREC_FP64MERGE", "SEP_PREC_DWORD", "SEP_UNIT_2TH_DEG", "SEP_UNIT_Q_NM",
           "SEP_UNIT_R_MM", "SEP_CUTOFF_FIXED", "SEP_CUTOFF_CHAUVENET", "SEP_ERROR_AZIMUTHAL", "SEP_ERROR_POISSON",
           "SEP_ERROR_HYBRID"]


def peaks_to_numpy(peaks, n):
    """Peak records of one frame (an int32 tensor [cap, 6]) as a structured array of the first n."""
    a = peaks[: int(n)].contiguous().cpu().numpy()
    return a.view(PEAK_DTYPE).reshape(-1)


class Context:
    """A library context on one GPU; several Separators may share it (and
    must, to be processed together by :func:`process_mixed`)."""

    def __init__(self, device: int = 0):
        self.device = device
        self.ctx = B.sep_ctx_create(device)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            B.sep_ctx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Separator:
    """One detector on one GPU: integration matrix, optional calibration, parameters.

    geometry: dict with rows, cols, pixel_m (y, x), dist_m, center_px (x, y),
    wavelength_m, unit, nbins, split, range (lo, hi; NaN = automatic).
    """

    def __init__(self, geometry: dict, mask=None, norm=None, calib=None, device: int = 0, n_iter=5, k_clip=3.0,
                 k_pick=3.0, patch=3, min_count=3, precision=SEP_PREC_DWORD, context: Context | None = None):
        import torch  # device memory and streams
        self.torch = torch
        self.context = context
        self.device = context.device if context is not None else device
        self.ctx = context.ctx if context is not None else B.sep_ctx_create(device)
        g = geometry
        self.geom = B.make_geometry(g["rows"], g["cols"], g["pixel_m"], g["dist_m"], g["center_px"],
                                    g["wavelength_m"], g["unit"], g["nbins"], g["split"], g["range"])
        self.csr = B.sep_build_csr(self.ctx, self.geom, mask, norm)
        self.info = B.sep_csr_info(self.csr)
        self.rows, self.cols = g["rows"], g["cols"]
        self.npix = self.info["npix"]
        self.nbins = self.info["nbins"]
        self.calib = None
        if calib is not None:
            self.calib = B.sep_calib_create(self.ctx, self.csr, calib[0], calib[1])
        self.params = B.make_params(n_iter, k_clip, k_pick, patch, min_count, precision)
        self._outs = {}
        self.surrogate = None

    @classmethod
    def from_detector(cls, det, mask=None, **kw):
        """From a ``synth.Detector``-like object (rows, cols, pixel_m, ...)."""
        g = dict(rows=det.rows, cols=det.cols, pixel_m=det.pixel_m, dist_m=det.dist_m, center_px=det.center_px,
                 wavelength_m=det.wavelength_m, unit=det.unit, nbins=det.nbins, split=det.split, range=det.range)
        return cls(g, mask=mask, **kw)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            B.sep_calib_destroy(self.calib)
            B.sep_csr_destroy(self.csr)
            if self.context is None:
                B.sep_ctx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_plan(self, tpb, thresholds=()):
        """Clip-kernel schedule: size classes of bins and threads per block."""
        B.sep_csr_set_plan(self.ctx, self.csr, tpb, thresholds)

    def get_plan(self):
        return B.sep_csr_get_plan(self.csr)

    def autotune(self, frames, cache_path=None, stream=None):
        """Time candidate schedules on a sample batch and keep the fastest."""
        F = self._check_frames(frames)
        return B.sep_autotune(self.ctx, self.csr, self.calib, frames, self._dtype(frames), F, self.params,
                              cache_path, stream)

    def set_params(self, **kw):
        for k, v in kw.items():
            setattr(self.params, k, v)

    # ---- learned surrogate of the clip loop ----
    def attach_surrogate(self, model: "Surrogate | None"):
        """Place every bin's first replay core from the model's prediction of
        its final clip interval (the results stay the plain loop's); None
        detaches."""
        B.sep_csr_attach_model(self.ctx, self.csr, model.model if model is not None else None)
        self.surrogate = model
        self.params.surrogate = 1 if model is not None else 0

    def record(self, frames, stream=None):
        """Plain clip that also returns the surrogate's features [F][B][20]
        and training targets [F][B][2] per bin."""
        t = self.torch
        F = self._check_frames(frames)
        dev = frames.device
        mean = t.empty((F, self.nbins), dtype=t.float32, device=dev)
        sigma = t.empty_like(mean)
        count = t.empty((F, self.nbins), dtype=t.int32, device=dev)
        feat = t.empty((F, self.nbins, B.SEP_MLP_IN), dtype=t.float32, device=dev)
        target = t.empty((F, self.nbins, B.SEP_MLP_OUT), dtype=t.float32, device=dev)
        p = B.make_params(self.params.n_iter, self.params.k_clip, self.params.k_pick, self.params.patch,
                          self.params.min_count, SEP_PREC_DWORD)
        B.sep_surrogate_record(self.ctx, self.csr, self.calib, frames, self._dtype(frames), F, p, mean, sigma, count,
                               feat, target, stream)
        return {"mean": mean, "sigma": sigma, "count": count, "feat": feat, "target": target}

    def surrogate_stats(self, reset=False, stream=None):
        """(bins settled by the surrogate, bins that fell back) since the last reset."""
        return B.sep_surrogate_stats(self.ctx, reset, stream)

    # ------------------------------------------------------------------
    def _dtype(self, frames):
        t = self.torch
        if frames.dtype == t.uint16 or frames.dtype == t.int16:
            return SEP_DTYPE_U16_JF
        if frames.dtype == t.float32:
            return SEP_DTYPE_F32
        raise TypeError(f"frames must be uint16 (raw Jungfrau) or float32, not {frames.dtype}")

    def _check_frames(self, frames):
        if not frames.is_cuda or not frames.is_contiguous():
            raise ValueError("frames must be a contiguous CUDA tensor")
        if frames.numel() % self.npix:
            raise ValueError("frames size is not a multiple of the detector's pixel count")
        return frames.numel() // self.npix

    def export_csr(self):
        return B.sep_csr_export(self.csr)

    def correct(self, frames, stream=None):
        """Corrected frames (float32 [F][npix]; NaN where the matrix uses no pixel)."""
        t = self.torch
        F = self._check_frames(frames)
        out = t.empty((F, self.npix), dtype=t.float32, device=frames.device)
        B.sep_correct(self.ctx, self.csr, self.calib, frames, self._dtype(frames), F, out, stream)
        return out

    def integrate_clip(self, frames, bounds=False, iters=False, stream=None):
        t = self.torch
        F = self._check_frames(frames)
        dev = frames.device
        mean = t.empty((F, self.nbins), dtype=t.float32, device=dev)
        sigma = t.empty_like(mean)
        count = t.empty((F, self.nbins), dtype=t.int32, device=dev)
        bnd = t.empty((F, self.nbins, 2), dtype=t.float32, device=dev) if bounds else None
        its = t.empty((F, self.nbins), dtype=t.int32, device=dev) if iters else None
        B.sep_integrate_clip(self.ctx, self.csr, self.calib, frames, self._dtype(frames), F, self.params, mean, sigma,
                             count, bnd, its, stream)
        out = {"mean": mean, "sigma": sigma, "count": count}
        if bounds:
            out["bounds"] = bnd
        if iters:
            out["iters"] = its
        return out

    def sparsify(self, frames, mean, sigma, capacity, stream=None):
        t = self.torch
        F = self._check_frames(frames)
        dev = frames.device
        idx = t.empty((F, capacity), dtype=t.int32, device=dev)
        val = t.empty((F, capacity), dtype=t.float32, device=dev)
        n_kept = t.empty(F, dtype=t.int32, device=dev)
        B.sep_sparsify(self.ctx, self.csr, self.calib, frames, self._dtype(frames), F, self.params, mean, sigma, idx,
                       val, capacity, n_kept, stream)
        return {"idx": idx, "val": val, "n_kept": n_kept}

    def peakfind(self, frames, mean, sigma, idx, n_kept, capacity, stream=None):
        t = self.torch
        F = self._check_frames(frames)
        dev = frames.device
        peaks = t.empty((F, capacity, 6), dtype=t.int32, device=dev)
        n_peaks = t.empty(F, dtype=t.int32, device=dev)
        B.sep_peakfind(self.ctx, self.csr, self.calib, frames, self._dtype(frames), F, self.params, mean, sigma, idx,
                       n_kept, idx.shape[1], peaks, capacity, n_peaks, stream)
        return {"peaks": peaks, "n_peaks": n_peaks}

    def densify(self, mean, sigma, idx, val, n_kept, noise=None, fill=float("nan"), out=None, interpolate=False,
                stream=None):
        """Dense frames from their sparse form (Section 3): each binned pixel
        gets its bin's mean (or, with ``interpolate``, the profile linearly
        interpolated at the pixel's radial value), plus sigma * noise with
        caller-drawn standard normal deviates; kept pixels their recorded
        values; pixels without a bin `fill`."""
        t = self.torch
        F = mean.shape[0]
        if out is None:
            out = t.empty((F, self.npix), dtype=t.float32, device=mean.device)
        kcap = idx.shape[1] if idx is not None else 0
        B.sep_densify(self.ctx, self.csr, F, mean, sigma, idx, val, kcap, n_kept, noise, fill, out, int(interpolate),
                      stream)
        return out

    def veto(self, n_peaks, min_peaks, stream=None):
        """Frames with at least ``min_peaks`` peaks (Section 4's veto):
        (ascending frame list [F], count [1]) on the device."""
        t = self.torch
        F = int(n_peaks.shape[0])
        frame_list = t.empty(F, dtype=t.int32, device=n_peaks.device)
        n_pass = t.empty(1, dtype=t.int32, device=n_peaks.device)
        B.sep_veto(self.ctx, F, n_peaks, min_peaks, frame_list, n_pass, stream)
        return frame_list, n_pass

    def compact_frames(self, frame_list, n_pass, src, out=None, stream=None):
        """Rows of the passing frames of a per-frame output, moved to the
        front (row j = row frame_list[j]); rows past the count are untouched."""
        if out is None:
            out = self.torch.empty_like(src)
        F = int(src.shape[0])
        B.sep_compact_frames(self.ctx, F, frame_list, n_pass, src[0].numel() * src.element_size(), src, out, stream)
        return out

    def alloc_outputs(self, F, kept_capacity, peak_capacity, device=None):
        t = self.torch
        dev = device if device is not None else t.device("cuda", self.device)
        return {"mean": t.empty((F, self.nbins), dtype=t.float32, device=dev),
                "sigma": t.empty((F, self.nbins), dtype=t.float32, device=dev),
                "count": t.empty((F, self.nbins), dtype=t.int32, device=dev),
                "idx": t.empty((F, kept_capacity), dtype=t.int32, device=dev),
                "val": t.empty((F, kept_capacity), dtype=t.float32, device=dev),
                "n_kept": t.empty(F, dtype=t.int32, device=dev),
                "peaks": t.empty((F, peak_capacity, 6), dtype=t.int32, device=dev),
                "n_peaks": t.empty(F, dtype=t.int32, device=dev)}

    def process_batch(self, frames, kept_capacity, peak_capacity, out=None, use_graph=True, stream=None):
        """The whole path (integrate + clip, sparsify, peaks) on a device batch."""
        F = self._check_frames(frames)
        o = out if out is not None else self.alloc_outputs(F, kept_capacity, peak_capacity, frames.device)
        B.sep_process_batch(self.ctx, self.csr, self.calib, frames, self._dtype(frames), F, self.params, o["mean"],
                            o["sigma"], o["count"], o["idx"], o["val"], kept_capacity, o["n_kept"], o["peaks"],
                            peak_capacity, o["n_peaks"], int(use_graph), stream)
        return o

    def alloc_host_outputs(self, F, kept_capacity, peak_capacity):
        """Pinned host tensors for process_host."""
        t = self.torch
        kw = dict(pin_memory=True)
        return {"mean": t.empty((F, self.nbins), dtype=t.float32, **kw),
                "sigma": t.empty((F, self.nbins), dtype=t.float32, **kw),
                "count": t.empty((F, self.nbins), dtype=t.int32, **kw),
                "idx": t.empty((F, kept_capacity), dtype=t.int32, **kw),
                "val": t.empty((F, kept_capacity), dtype=t.float32, **kw),
                "n_kept": t.empty(F, dtype=t.int32, **kw),
                "peaks": t.empty((F, peak_capacity, 6), dtype=t.int32, **kw),
                "n_peaks": t.empty(F, dtype=t.int32, **kw)}

    def process_host(self, frames_host, host_out, kept_capacity, peak_capacity, chunk_frames=0, stream=None):
        """End to end from (pinned) host memory to host memory: the library
        copies chunks in, runs the path and copies results out, overlapping
        the copies with compute. Results are complete once `stream` (default:
        the current stream) has been synchronised."""
        if frames_host.is_cuda or not frames_host.is_contiguous():
            raise ValueError("frames_host must be a contiguous host tensor")
        if frames_host.numel() % self.npix:
            raise ValueError("frames size is not a multiple of the detector's pixel count")
        F = frames_host.numel() // self.npix
        o = host_out
        B.sep_process_host(self.ctx, self.csr, self.calib, frames_host, self._dtype(frames_host), F, self.params,
                           o["mean"], o["sigma"], o["count"], o["idx"], o["val"], kept_capacity, o["n_kept"],
                           o["peaks"], peak_capacity, o["n_peaks"], chunk_frames, stream)
        return o

    def device_status(self, stream=None):
        return B.sep_get_device_status(self.ctx, stream)

    def clip_stats(self, enable=-1, read=True, reset=False, stream=None):
        """Tail-replay counters of the clip kernel (see sep_clip_stats)."""
        return B.sep_clip_stats(self.ctx, enable, read, reset, stream)


class Surrogate:
    """The clip surrogate's network (20 -> 64 -> 64 -> 2, GELU), trained on
    the GPU by the library's own forward / backward / Adam kernels."""

    def __init__(self, context, seed=0, path=None):
        self.ctx = context.ctx if isinstance(context, Context) else context
        self._context = context
        self.model = B.sep_model_load(self.ctx, path) if path else B.sep_model_create(self.ctx, seed)

    def close(self):
        if getattr(self, "model", None) is not None:
            B.sep_model_destroy(self.model)
            self.model = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self, set_host=None):
        return B.sep_model_params(self.ctx, self.model, set_host)

    def norm(self, set_host=None):
        return B.sep_model_norm(self.ctx, self.model, set_host)

    def save(self, path):
        B.sep_model_save(self.ctx, self.model, path)

    def forward(self, x, stream=None):
        import torch
        y = torch.empty((x.shape[0], B.SEP_MLP_OUT), dtype=torch.float32, device=x.device)
        B.sep_mlp_forward(self.ctx, self.model, x, x.shape[0], y, stream)
        return y

    def loss_grad(self, x, t, stream=None):
        import torch
        g = torch.empty(B.SEP_MLP_PARAMS, dtype=torch.float32, device=x.device)
        l = torch.empty(1, dtype=torch.float32, device=x.device)
        B.sep_mlp_loss_grad(self.ctx, self.model, x, t, x.shape[0], g, l, stream)
        return l, g

    def fit(self, feat, target, epochs=4, batch=4096, lr=2e-3, seed=0, stream=None):
        """Train on recorded rows (feat [n][20], target [n][2], device):
        keeps the finite rows, sets the normalisation, runs Adam. Returns
        (last epoch's mean loss, rows used)."""
        import torch
        f = feat.reshape(-1, B.SEP_MLP_IN).contiguous()
        t = target.reshape(-1, B.SEP_MLP_OUT).contiguous()
        n = f.shape[0]
        x = torch.empty_like(f)
        y = torch.empty_like(t)
        norm, nv = B.sep_surrogate_prepare(self.ctx, f, t, n, x, y, stream)
        if nv == 0:
            raise ValueError("no usable training rows")
        self.norm(norm)
        loss = B.sep_surrogate_train(self.ctx, self.model, x, y, nv, epochs, batch, lr, seed, stream)
        return loss, nv


def process_mixed(seps, frames, kept_capacity, peak_capacity, use_graph=True, stream=None):
    """The whole path on a stream of frames from several detectors at once.

    seps: Separators sharing one :class:`Context`; frames: list of
    (detector index, contiguous CUDA tensor of one frame). Returns the output
    tensors and the per-frame row offsets into the flat mean/sigma/count."""
    import torch
    ctx = seps[0].ctx
    if any(s.ctx is not ctx for s in seps):
        raise ValueError("process_mixed needs Separators that share one Context")
    dev = frames[0][1].device
    total_bins = sum(seps[d].nbins for d, _ in frames)
    n = len(frames)
    out = {"mean": torch.empty(total_bins, dtype=torch.float32, device=dev),
           "sigma": torch.empty(total_bins, dtype=torch.float32, device=dev),
           "count": torch.empty(total_bins, dtype=torch.int32, device=dev),
           "idx": torch.empty((n, kept_capacity), dtype=torch.int32, device=dev),
           "val": torch.empty((n, kept_capacity), dtype=torch.float32, device=dev),
           "n_kept": torch.empty(n, dtype=torch.int32, device=dev),
           "peaks": torch.empty((n, peak_capacity, 6), dtype=torch.int32, device=dev),
           "n_peaks": torch.empty(n, dtype=torch.int32, device=dev)}
    descs = []
    for d, t in frames:
        if not t.is_contiguous() or t.numel() != seps[d].npix:
            raise ValueError("each frame must be one contiguous detector image")
        descs.append((d, seps[d]._dtype(t), t))
    rows = B.sep_process_mixed(ctx, [s.csr for s in seps], [s.calib for s in seps], descs, seps[0].params,
                               out["mean"], out["sigma"], out["count"], out["idx"], out["val"], kept_capacity,
                               out["n_kept"], out["peaks"], peak_capacity, out["n_peaks"], use_graph, stream)
    out["row_off"] = rows
    return out
