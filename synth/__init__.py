"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This package makes inputs only: detector descriptions (geometry + mask),
Jungfrau-like calibration planes and diffraction-like frames. It contains none
of the signal-separation arithmetic. The frames follow the workloads the paper
measures on (Jungfrau 4M serial-crystallography frames, Section 1.2 and
Section 3.4; Pilatus-like photon-counting frames, Section 2.3), which are not
available here, so seeded synthetic stand-ins of the same shape are used.

The C implementation (synth.c) is compiled into ``synth/_build/libsynth.so``
by :func:`build` (or by ``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from dataclasses import dataclass, field, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libsynth.so")
_lib = None


def build_cmd():
    return ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-ffp-contract=off", "-Wall",
            os.path.join(_HERE, "synth.c"), "-lm", "-o", _SO]


_SO_GPU = os.path.join(_HERE, "_build", "libsynth_gpu.so")
_lib_gpu = None


def build_gpu_cmd():
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-shared", "-Xcompiler", "-fPIC",
            "-fmad=false", os.path.join(_HERE, "synth_gpu.cu"), "-o", _SO_GPU]


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    src = os.path.join(_HERE, "synth.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.run(build_cmd(), check=True)
    src = os.path.join(_HERE, "synth_gpu.cu")
    if force or not os.path.exists(_SO_GPU) or os.path.getmtime(_SO_GPU) < os.path.getmtime(src):
        subprocess.run(build_gpu_cmd(), check=True)
    return _SO


class _Spec(C.Structure):
    _fields_ = [
        ("rows", C.c_int32), ("cols", C.c_int32),
        ("cx", C.c_double), ("cy", C.c_double),
        ("bg_kind", C.c_int32),
        ("bg_scale_lo", C.c_double), ("bg_scale_hi", C.c_double),
        ("bg_clip_lo", C.c_double), ("bg_clip_hi", C.c_double),
        ("hit_rate", C.c_double),
        ("spots_min", C.c_int32), ("spots_max", C.c_int32),
        ("amp_lo", C.c_double), ("amp_hi", C.c_double),
        ("amp_log", C.c_int32),
        ("sig_lo", C.c_double), ("sig_hi", C.c_double),
        ("out_raw", C.c_int32),
        ("read_noise_adu", C.c_double),
        ("seed", C.c_uint64),
    ]


class _Spot(C.Structure):
    _fields_ = [("x", C.c_float), ("y", C.c_float), ("amp", C.c_float), ("sigma", C.c_float)]


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(_SO):
            build()
        L = C.CDLL(_SO)
        L.synth_jf_mask.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_void_p]
        L.synth_jf_mask.restype = C.c_int
        L.synth_calib.argtypes = [C.c_uint64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_double, C.c_void_p, C.c_void_p]
        L.synth_calib.restype = None
        L.synth_frames.argtypes = [C.POINTER(_Spec), C.c_int64, C.c_int32, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]
        L.synth_frames.restype = C.c_int
        L.synth_philox4x32_10.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.synth_max_threads.restype = C.c_int
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# --------------------------------------------------------------------------
# Detector descriptions
# --------------------------------------------------------------------------
UNIT_2TH_DEG, UNIT_Q_NM, UNIT_R_MM = 0, 1, 2


@dataclass
class Detector:
    """A flat detector normal to the beam and its azimuthal-integration setup."""
    name: str
    rows: int
    cols: int
    pixel_m: tuple = (75e-6, 75e-6)      # (y, x)
    dist_m: float = 0.1
    center_px: tuple = (128.3, 120.7)    # (x = column, y = row), pixel centres at idx + 0.5
    wavelength_m: float = 1.0e-10
    unit: int = UNIT_2TH_DEG
    nbins: int = 64
    split: int = 1
    range: tuple = (float("nan"), float("nan"))
    layout: tuple | None = None          # Jungfrau module grid (n_mr, n_mc) or None = no mask

    @property
    def npix(self) -> int:
        return self.rows * self.cols

    def mask(self) -> np.ndarray:
        m = np.zeros(self.rows * self.cols, np.uint8)
        if self.layout is not None:
            rc = lib().synth_jf_mask(self.rows, self.cols, self.layout[0], self.layout[1], _p(m))
            if rc != 0:
                raise ValueError(f"layout {self.layout} does not fit {self.rows}x{self.cols}")
        return m


def det_config1() -> Detector:
    """256 x 256 float32 frame, 75 um pixels, 100 mm, centre (128.3, 120.7),
    no splitting, 64 bins in 2theta (degrees)."""
    return Detector("256x256", 256, 256, dist_m=0.100, center_px=(128.3, 120.7),
                    unit=UNIT_2TH_DEG, nbins=64, split=1)


def det_jf(rows, cols, layout, nbins, split, name, unit=UNIT_Q_NM, center=None):
    if center is None:
        center = (cols / 2 + 0.3, rows / 2 + 0.7)
    return Detector(name, rows, cols, dist_m=0.150, center_px=center, unit=unit,
                    nbins=nbins, split=split, layout=layout)


def det_jf4m(split=2, nbins=1000) -> Detector:
    """Jungfrau 4M: 2164 x 2068 px, 4 x 2 modules, 150 mm, centre (1040.3, 1090.7),
    q bins (nm^-1), 2 x 2 sub-pixel splitting by default."""
    return det_jf(2164, 2068, (4, 2), nbins, split, "JF4M", center=(1040.3, 1090.7))


def det_jf1m(split=1, nbins=600) -> Detector:
    return det_jf(1064, 1030, (2, 1), nbins, split, "JF1M")


def det_jf16m(split=1, nbins=2000) -> Detector:
    return det_jf(4362, 4148, (8, 4), nbins, split, "JF16M")


def det_small_jf(split=2, nbins=96, rows=514 * 2 + 36, cols=1030) -> Detector:
    """A reduced Jungfrau-like detector (2 x 1 modules) for parity tests."""
    return det_jf(rows, cols, (2, 1), nbins, split, "JF-2mod", center=(cols * 0.43, rows * 0.61))


# --------------------------------------------------------------------------
# Calibration and frames
# --------------------------------------------------------------------------
PED_MEAN = (1500.0, 14000.0, 15000.0)
PED_STD = (50.0, 200.0, 200.0)
# Gains of levels 1 and 2 are stored negative: the ADC falls as charge rises
# in the low-gain stages, so 5e4 photons still fit in 14 bits.
GAIN_NOM = (40.0, -1.5, -0.1)


def jf_calib(npix: int, seed: int = 1234):
    ped = np.empty((3, npix), np.float32)
    gain = np.empty((3, npix), np.float32)
    pm = np.array(PED_MEAN, np.float64)
    ps = np.array(PED_STD, np.float64)
    gn = np.array(GAIN_NOM, np.float64)
    lib().synth_calib(seed, npix, _p(pm), _p(ps), _p(gn), 0.02, _p(ped), _p(gain))
    return ped, gain


@dataclass
class FrameSpec:
    bg_kind: int = 0
    bg_scale: tuple = (1.0, 1.0)
    bg_clip: tuple = (0.0, 1e30)
    hit_rate: float = 1.0
    spots: tuple = (12, 12)
    amp: tuple = (200.0, 2000.0)
    amp_log: bool = False
    sigma: tuple = (1.2, 1.2)
    out_raw: bool = False
    read_noise_adu: float = 10.0
    seed: int = 0


def spec_config1(seed=0) -> FrameSpec:
    """50 exp(-r/80) + water ring (r = 90 px, amplitude 30, width 6) + 12 spots
    (sigma 1.2 px, 200-2000 photons), Poisson noise, float32 photons."""
    return FrameSpec(seed=seed)


def spec_jf_serial(seed=0, raw=True) -> FrameSpec:
    """Solvent rings + exponential fall-off clipped to 0.05-5 photons/px; 30 %
    hits with 20-300 spots of 10-1e4 photons (log-uniform), sigma 0.8-1.5 px."""
    return FrameSpec(bg_kind=1, bg_scale=(0.5, 3.0), bg_clip=(0.05, 5.0), hit_rate=0.3,
                     spots=(20, 300), amp=(10.0, 1e4), amp_log=True, sigma=(0.8, 1.5),
                     out_raw=raw, seed=seed)


def spec_jf_hdr(seed=0) -> FrameSpec:
    """High dynamic range: background 0.01-50 photons/px, spots up to 5e4
    photons, so all three gain levels occur."""
    return FrameSpec(bg_kind=1, bg_scale=(0.02, 30.0), bg_clip=(0.01, 50.0), hit_rate=0.5,
                     spots=(20, 300), amp=(10.0, 5e4), amp_log=True, sigma=(0.8, 1.5),
                     out_raw=True, seed=seed)


def spec_mixed(seed=0, hit_rate=0.3) -> FrameSpec:
    """Float32 photon frames for the mixed-detector stream: 5-500 spots per hit."""
    return FrameSpec(bg_kind=1, bg_scale=(0.5, 3.0), bg_clip=(0.05, 5.0), hit_rate=hit_rate,
                     spots=(5, 500), amp=(10.0, 1e4), amp_log=True, sigma=(0.8, 1.5),
                     out_raw=False, seed=seed)


def frames(det: Detector, spec: FrameSpec, frame0: int, n: int, calib=None, mask=None,
           max_spots: int = 0, out=None):
    """Generate ``n`` frames starting at frame index ``frame0``.

    Returns ``(frames, spots, n_spots)`` where frames is float32 or uint16
    ``[n][rows*cols]`` and spots is a structured array ``[n][max_spots]`` with
    fields x, y, amp, sigma (x = column, y = row, in px; None if max_spots = 0).
    """
    s = _Spec(det.rows, det.cols, det.center_px[0], det.center_px[1], spec.bg_kind,
              spec.bg_scale[0], spec.bg_scale[1], spec.bg_clip[0], spec.bg_clip[1],
              spec.hit_rate, spec.spots[0], spec.spots[1], spec.amp[0], spec.amp[1],
              int(spec.amp_log), spec.sigma[0], spec.sigma[1], int(spec.out_raw),
              spec.read_noise_adu, spec.seed)
    dt = np.uint16 if spec.out_raw else np.float32
    if out is None:
        out = np.empty((n, det.npix), dt)
    assert out.dtype == dt and out.shape == (n, det.npix) and out.flags.c_contiguous
    ped = gain = None
    if spec.out_raw:
        if calib is None:
            raise ValueError("raw frames need calibration planes")
        ped, gain = calib
    if mask is None and det.layout is not None:
        mask = det.mask()
    spots = nsp = None
    if max_spots > 0:
        spots = np.zeros((n, max_spots), dtype=[("x", "<f4"), ("y", "<f4"), ("amp", "<f4"), ("sigma", "<f4")])
        nsp = np.zeros(n, np.int32)
    rc = lib().synth_frames(C.byref(s), frame0, n, _p(ped), _p(gain), _p(mask), _p(out),
                            _p(spots), max_spots, _p(nsp))
    if rc != 0:
        raise RuntimeError(f"synth_frames failed ({rc})")
    return out, spots, nsp


def philox(ctr, key):
    c = np.asarray(ctr, np.uint32)
    k = np.asarray(key, np.uint32)
    o = np.zeros(4, np.uint32)
    lib().synth_philox4x32_10(_p(c), _p(k), _p(o))
    return o


def lib_gpu():
    global _lib_gpu
    if _lib_gpu is None:
        if not os.path.exists(_SO_GPU):
            build()
        L = C.CDLL(_SO_GPU)
        L.synth_gpu_scratch_bytes.argtypes = [C.POINTER(_Spec), C.c_int32]
        L.synth_gpu_scratch_bytes.restype = C.c_size_t
        L.synth_gpu_frames.argtypes = [C.POINTER(_Spec), C.c_int64, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]
        L.synth_gpu_frames.restype = C.c_int
        _lib_gpu = L
    return _lib_gpu


def _spec_struct(det, spec):
    return _Spec(det.rows, det.cols, det.center_px[0], det.center_px[1], spec.bg_kind,
                 spec.bg_scale[0], spec.bg_scale[1], spec.bg_clip[0], spec.bg_clip[1],
                 spec.hit_rate, spec.spots[0], spec.spots[1], spec.amp[0], spec.amp[1],
                 int(spec.amp_log), spec.sigma[0], spec.sigma[1], int(spec.out_raw),
                 spec.read_noise_adu, spec.seed)


def frames_gpu(det: Detector, spec: FrameSpec, frame0: int, n: int, out, calib_dev=None, mask_dev=None,
               scratch=None, stream=None):
    """The frames of :func:`frames` generated on the GPU (same model, same
    Philox streams; a rare pixel may differ by one count, see synth_gpu.cu).
    ``out``: a device tensor of n * npix uint16 (raw) or float32 words;
    ``calib_dev``: device (ped, gain) planes [3 * npix] for raw frames;
    ``mask_dev``: device uint8 [npix] or None; ``scratch``: a device uint8
    tensor of at least :func:`gpu_scratch_bytes` bytes (allocated when None);
    ``stream``: a torch CUDA stream (default: the current one)."""
    import torch
    s = _spec_struct(det, spec)
    need = lib_gpu().synth_gpu_scratch_bytes(C.byref(s), n)
    if scratch is None:
        scratch = torch.empty(need, dtype=torch.uint8, device=out.device)
    if scratch.numel() < need:
        raise ValueError("scratch too small")
    if stream is None:
        stream = torch.cuda.current_stream(out.device)
    ped = gain = None
    if spec.out_raw:
        if calib_dev is None:
            raise ValueError("raw frames need calibration planes on the device")
        ped, gain = (C.c_void_p(calib_dev[0].data_ptr()), C.c_void_p(calib_dev[1].data_ptr()))
    rc = lib_gpu().synth_gpu_frames(C.byref(s), frame0, n, ped, gain,
                                    None if mask_dev is None else C.c_void_p(mask_dev.data_ptr()),
                                    C.c_void_p(out.data_ptr()), C.c_void_p(scratch.data_ptr()), scratch.numel(),
                                    C.c_void_p(stream.cuda_stream))
    if rc != 0:
        raise RuntimeError(f"synth_gpu_frames failed ({rc})")
    return out


def gpu_scratch_bytes(det: Detector, spec: FrameSpec, n: int) -> int:
    s = _spec_struct(det, spec)
    return int(lib_gpu().synth_gpu_scratch_bytes(C.byref(s), n))
