"""Benchmark: Jungfrau-4M frames/s through the whole per-frame path
(correction + integration + sigma-clipping + sparsification + peak picking).

Workload: a batch of 512 synthetic raw Jungfrau-4M frames (2164 x 2068 uint16,
4 x 2 modules, gaps masked), 1000 q bins with 2 x 2 sub-pixel splitting,
5 clip iterations at k = 3, sparsification at k = 3, 3 x 3 peaks with at
least 3 kept pixels; per-pixel pedestal[3] / gain[3] calibration.

One step = one call of sep_process_batch on the whole batch (a replayed CUDA
graph). The batch (4.58 GB of raw frames) is larger than L2, so no flush is
needed between steps. Multi-GPU: each rank processes its own batch of
distinct frames (replicas, no collective on the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--frames F] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Jungfrau-4M frames/s (clip+sparsify+peaks), % HBM roofline; surrogate vs plain"
UNIT = "frames/s"
WORKLOAD = "JF4M raw uint16 2164x2068, 1000 q bins, 2x2 split, n_iter 5 k 3, k_pick 3, 3x3 peaks min 3"


def peaks_file():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x, device="cpu"):
    """The largest value of x over the ranks of the process group (x itself
    with one process): the job's time is its slowest rank's."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(frames_per_rank, steps, world, ms):
    """Frames per second of the whole job: every rank processes its own
    frames_per_rank frames per step (weak scaling), in ms for all steps."""
    return frames_per_rank * steps * world / (ms * 1e-3)


def setup_workload(F, rank, seed=2024):
    import synth
    det = synth.det_jf4m(split=2, nbins=1000)
    mask = det.mask()
    cal = synth.jf_calib(det.npix, seed=seed)
    spec = synth.spec_jf_serial(seed)
    frames, _, _ = synth.frames(det, spec, rank * F, F, calib=cal, mask=mask)
    return det, mask, cal, frames


def algorithmic_bytes_clip(F, npix, nvalid, nnz, nbins):
    """Minimum DRAM bytes of one staged integrate + clip of F raw frames
    (k_stage_ring + k_clip_warp): every raw word once (2 B/pixel/frame), the
    calibration planes and the matrix once per launch, the per-bin outputs
    (mean, sigma, count, threshold). The staged copy of the values that the
    two kernels exchange is an implementation choice and is not charged."""
    return 2 * npix * F + 24 * npix + 4 * nnz + 4 * (nbins + 1) + 16 * nbins * F


def algorithmic_bytes_path(F, npix, nnz, nbins, kept_per_frame, peaks_per_frame):
    """Minimum DRAM bytes per frame of the whole path at batch F: the raw
    frame (2 B/pixel), the calibration planes (24 B/pixel), the matrix and
    the bin map (4 B/pixel) shared by the batch, and the outputs: mean,
    sigma, count (12 B/bin), the kept list (8 B/pixel kept) and the peak
    records (24 B/peak) with their counts."""
    shared = 24 * npix + 4 * nnz + 4 * (nbins + 1) + 4 * npix
    out = 12 * nbins + 8 * kept_per_frame + 24 * peaks_per_frame + 8
    return 2 * npix + shared / F + out


NOMINAL_HBM_GBS = 7900.0   # GB300 HBM3e, nominal


CLIP_SOURCES = ["k_stage.cu", "k_clip.cu", "sep_internal.h", "sep_device.cuh"]


def strip_comments(src: str) -> str:
    """C++ source without its comments, runs of white space made one space
    (string and character literals kept as written)."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c == "/" and src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif c == "/" and src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        elif c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def source_fingerprint(names=CLIP_SOURCES):
    """SHA-256 of the staging and clip kernel sources without comments: the
    code the traffic capture measured."""
    import hashlib
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_2411_09515_gb300", "csrc", name), encoding="utf-8") as f:
            h.update(strip_comments(f.read()).encode())
        h.update(b"\0")
    return h.hexdigest()


def measured_traffic(F):
    """DRAM bytes (read + write) of k_stage_ring + k_clip_warp per launch of F
    frames, from the ncu capture recorded in profiles/roofline_traffic.json,
    scaled from its frame count; None when absent or when the kernels' code
    changed since the capture."""
    p = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f)
    if rec.get("sources_sha256") != source_fingerprint():
        return None
    return int(rec["bytes_per_frame"] * F)


def leg_status(sep, out=None, kcap=None, pcap=None):
    """The device status word of the leg just run (read and cleared by the
    library), with its largest kept-pixel and peak counts against the
    capacities; a leg whose outputs overflowed is marked void."""
    st = {"device_status": int(sep.device_status())}
    if out is not None:
        st["max_kept"] = int(out["n_kept"].max().item())
        st["max_peaks"] = int(out["n_peaks"].max().item())
        if kcap is not None:
            st["kept_capacity"] = kcap
            st["peak_capacity"] = pcap
    if st["device_status"] != 0:
        st["void"] = "capacity overflow: outputs truncated, this leg's number is not a valid measurement"
    return st


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2411_09515_gb300 import Separator, _binding as B

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    F = args.frames
    t0 = time.time()
    det, mask, cal, frames_np = setup_workload(F, rank)
    t_gen = time.time() - t0
    prec = {"plain": B.SEP_PREC_PLAIN, "kahan": B.SEP_PREC_KAHAN, "fp64merge": B.SEP_PREC_FP64MERGE,
            "dword": B.SEP_PREC_DWORD}[args.precision]
    sep = Separator.from_detector(det, mask=mask, calib=cal, device=local, precision=prec)
    info = sep.info
    kcap, pcap = args.kept_capacity, args.peak_capacity
    host = torch.from_numpy(frames_np.view(np.int16)).pin_memory()
    dev = host.to(f"cuda:{local}", non_blocking=False)
    out = sep.alloc_outputs(F, kcap, pcap)
    stream = torch.cuda.current_stream()
    tune_ms = None
    if args.clip_plan:
        # a fixed clip schedule "T1,T2:W1,W2,W3" (size-class thresholds in
        # entries : threads per block of each class), for reproducible profiles
        thr, tpb = args.clip_plan.split(":")
        sep.set_plan([int(x) for x in tpb.split(",")], [int(x) for x in thr.split(",") if x])
    elif not args.no_autotune:
        # the library's autotuner picks the clip schedule on a sample of the batch
        tune_ms = sep.autotune(dev[: min(F, 256)], stream=stream)
    plan = sep.get_plan()
    # launches of our kernels per step: staging, one clip launch per size
    # class of the schedule (it also marks the kept pixels), two for the
    # compaction, two for the peaks
    launches_per_step = max(len(plan["tpb"]), 1) + 5

    def step():
        sep.process_batch(dev, kcap, pcap, out=out, use_graph=True, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sep.device_status()   # clear the status word before the timed region
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    # one event between consecutive steps: the total and each step's time
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    with Clocks(local) as clk:
        evs[0].record(stream)
        for i in range(args.steps):
            step()
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ms = max_over_ranks(evs[0].elapsed_time(evs[-1]), device=f"cuda:{local}")
    per_step = sorted(evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps))
    main_leg = leg_status(sep, out, kcap, pcap)
    status = main_leg["device_status"]
    n_kept = out["n_kept"].cpu().numpy()
    n_peaks = out["n_peaks"].cpu().numpy()

    # dominant kernel alone (same kernel, same launch shape, no marking),
    # timed with events on the launching stream
    ic_mean = torch.empty((F, sep.nbins), dtype=torch.float32, device=dev.device)
    ic_sig = torch.empty_like(ic_mean)
    ic_cnt = torch.empty((F, sep.nbins), dtype=torch.int32, device=dev.device)
    for _ in range(2):
        B.sep_integrate_clip(sep.ctx, sep.csr, sep.calib, dev, B.SEP_DTYPE_U16_JF, F, sep.params, ic_mean, ic_sig,
                             ic_cnt, None, None, stream)
    torch.cuda.synchronize()
    k0 = torch.cuda.Event(enable_timing=True)
    k1 = torch.cuda.Event(enable_timing=True)
    k0.record(stream)
    for _ in range(args.steps):
        B.sep_integrate_clip(sep.ctx, sep.csr, sep.calib, dev, B.SEP_DTYPE_U16_JF, F, sep.params, ic_mean, ic_sig,
                             ic_cnt, None, None, stream)
    k1.record(stream)
    torch.cuda.synchronize()
    k_ms = k0.elapsed_time(k1) / args.steps
    clip_leg = leg_status(sep)

    # end to end through the public API from pinned host memory to pinned
    # host memory (the library pipelines copies and compute by chunks)
    host_out = sep.alloc_host_outputs(F, kcap, pcap)
    h2d = host.numel() * host.element_size()
    d2h = sum(v.numel() * v.element_size() for v in host_out.values())
    for _ in range(2):
        sep.process_host(host, host_out, kcap, pcap, chunk_frames=args.chunk_frames, stream=stream)
    torch.cuda.synchronize()
    sep.device_status()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        sep.process_host(host, host_out, kcap, pcap, chunk_frames=args.chunk_frames, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), device=f"cuda:{local}")
    e2e_leg = leg_status(sep)
    e2e_leg["max_kept"] = int(host_out["n_kept"].max())
    e2e_leg["max_peaks"] = int(host_out["n_peaks"].max())

    # densification (Section 3) of the batch's sparse output, timed alone
    sep.device_status()
    dens = densify_eval(sep, out, F, stream, args)
    dens.update(leg_status(sep))
    # the clip variants of Section 2.4 on the same batch, and the veto
    variants = variants_eval(sep, dev, out, kcap, pcap, stream, args)

    # the learned surrogate against the plain loop on the same batch
    sur = None
    if args.surrogate_train_frames > 0:
        sep.device_status()
        sur = surrogate_eval(sep, det, mask, cal, kcap, pcap, stream, args)

    # oracle on the host cores, rank 0 at N = 1 only, with the precision
    # modes' errors against it on the same frames
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        nc = max(1, min(args.cpu_frames, F))
        modes = {}
        for name, pv in (("plain", B.SEP_PREC_PLAIN), ("kahan", B.SEP_PREC_KAHAN),
                         ("fp64merge", B.SEP_PREC_FP64MERGE), ("dword", B.SEP_PREC_DWORD)):
            sep.set_params(precision=pv)
            r = sep.integrate_clip(dev[:nc])
            modes[name] = (r["mean"].double().cpu().numpy(), r["sigma"].double().cpu().numpy())
        sep.set_params(precision=prec)
        cpu = cpu_baseline(det, mask, cal, frames_np, args.cpu_frames, modes)

    # uneven batching (1M / 4M / 16M frames in one graph)
    mixed = None
    if world == 1 and args.mixed_frames > 0:
        mixed = mixed_eval(args.mixed_frames, 3, 2, args.kept_capacity, args.peak_capacity)

    # thresholds from the smooth background, last (it overwrites the outputs)
    interp = interp_eval(sep, dev, out, kcap, pcap, stream)

    if rank == 0:
        peaks, src = peaks_file()
        nvalid = int((mask == 0).sum())
        alg = algorithmic_bytes_clip(F, det.npix, nvalid, info["nnz"], info["nbins"])
        achieved = alg / (k_ms * 1e-3) / 1e9
        value = whole_job_rate(F, args.steps, world, ms)
        path_bytes = algorithmic_bytes_path(F, det.npix, info["nnz"], info["nbins"], float(n_kept.mean()),
                                            float(n_peaks.mean()))
        path_roof = peaks.get("hbm_gbs") * 1e9 / path_bytes
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True,
            "step_ms": ({"median": round(per_step[len(per_step) // 2], 4), "min": round(per_step[0], 4),
                         "max": round(per_step[-1], 4)} if per_step else None),
            "scaling": "weak", "vs_baseline": None, "dtype": "u16->f32",
            "data": "synthetic (seeded Jungfrau-4M-shaped raw frames; no dataset)",
            "config": {"workload": WORKLOAD, "frames_per_gpu": F, "nnz": info["nnz"], "max_row": info["max_row"],
                       "l2": "inputs larger than L2 (4.58 GB/batch), no flush", "parallelism": f"replicas x{world}",
                       "kept_capacity": kcap, "peak_capacity": pcap, "precision": args.precision,
                       "clip_schedule": plan, "autotune_sample_ms": tune_ms},
            "roofline": {"bound": "hbm", "kernel": "k_stage_ring + k_clip_warp", "achieved": round(achieved, 1),
                         "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                         "frac": round(achieved / peaks.get("hbm_gbs"), 4), "traffic": measured_traffic(F),
                         "peak_source": src, "kernel_ms": round(k_ms, 4), "kernel_leg": clip_leg,
                         "algorithmic_bytes_per_launch": alg,
                         "frac_of_nominal": round(achieved / NOMINAL_HBM_GBS, 4),
                         "whole_path": {"bytes_per_frame": round(path_bytes, 1),
                                        "frames_s_at_peak": round(path_roof, 1),
                                        "frac": round(value / world / path_roof, 4)}},
            "e2e": {"value": round(whole_job_rate(F, args.steps, world, e2e_ms), 2), "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "chunk_frames": args.chunk_frames,
                    **e2e_leg},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clk.summary(),
            "cpu_baseline": {k: v for k, v in cpu.items() if k != "precision"} if cpu else None,
            # each precision mode's error against the FP64 oracle on the same frames
            "precision": cpu.get("precision") if cpu else None,
            "surrogate": sur,
            "densify": dens,
            "variants": variants,
            "interpolated_thresholds": interp,
            "mixed": mixed,
            "device_status": status, "main_leg": main_leg,
            "mean_kept_per_frame": float(n_kept.mean()), "mean_peaks_per_frame": float(n_peaks.mean()),
            "setup_s": round(t_gen, 1),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def variants_eval(sep, dev, out, kcap, pcap, stream, args):
    """Whole-path frames/s with Chauvenet's cut-off (Eq. 20) and with the
    Poisson and hybrid error models (Section 2.4.1) on the benchmark batch,
    and the time of the veto (Section 4) with the compaction of the kept lists
    and peak records of the passing frames."""
    import torch
    from paper_2411_09515_gb300 import SEP_CUTOFF_CHAUVENET, SEP_ERROR_HYBRID, SEP_ERROR_POISSON
    F = dev.shape[0]

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    res = {}
    base = (sep.params.cutoff, sep.params.error_model)
    # the Poisson deviation of these low-count frames is below the azimuthal
    # one: those models keep several times more pixels and peaks, so the
    # variants write into outputs sized for them
    vk, vp = max(kcap, 1 << 21), max(pcap, 1 << 18)
    vout = sep.alloc_outputs(F, vk, vp)
    for name, kw in (("chauvenet", {"cutoff": SEP_CUTOFF_CHAUVENET}), ("poisson", {"error_model": SEP_ERROR_POISSON}),
                     ("hybrid", {"error_model": SEP_ERROR_HYBRID})):
        sep.set_params(**kw)
        sep.device_status()
        ms = timed(lambda: sep.process_batch(dev, vk, vp, out=vout, use_graph=True, stream=stream), 3)
        res[name] = {"frames_s": round(F / (ms * 1e-3), 1), "ms_per_step": round(ms, 3),
                     **leg_status(sep, vout, vk, vp)}
        sep.set_params(cutoff=base[0], error_model=base[1])
    del vout
    sep.process_batch(dev, kcap, pcap, out=out, use_graph=True, stream=stream)   # the plain outputs again
    dst = {k: torch.empty_like(out[k]) for k in ("idx", "val", "peaks", "n_kept", "n_peaks")}
    thr = 20

    def veto_step():
        lst, n = sep.veto(out["n_peaks"], thr, stream=stream)
        for k in dst:
            sep.compact_frames(lst, n, out[k], out=dst[k], stream=stream)
        return n

    sep.device_status()
    ms = timed(veto_step, 5)
    n = int(veto_step().item())
    res["veto"] = {"min_peaks": thr, "frames_passed": n, "frames": F, "ms": round(ms, 3), **leg_status(sep)}
    return res


def interp_eval(sep, dev, out, kcap, pcap, stream):
    """Whole-path frames/s with the sparsification and peak thresholds taken
    from the per-bin profile interpolated at each pixel centre (Section 3's
    smooth background): the clip kernel then marks nothing and a marking pass
    over the staged values follows it. An error is reported in the result
    instead of ending the run."""
    import torch
    F = dev.shape[0]
    try:
        sep.set_params(interpolate=1)
        run = lambda: sep.process_batch(dev, kcap, pcap, out=out, use_graph=True, stream=stream)
        run()
        torch.cuda.synchronize()
        sep.device_status()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            run()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 3
        return {"frames_s": round(F / (ms * 1e-3), 1), "ms_per_step": round(ms, 3),
                "mean_kept_per_frame": float(out["n_kept"].float().mean().item()),
                "mean_peaks_per_frame": float(out["n_peaks"].float().mean().item()),
                **leg_status(sep, out, kcap, pcap)}
    except Exception as e:   # reported, not hidden: the line still carries the other measurements
        return {"error": f"{type(e).__name__}: {e}"}
    finally:
        sep.set_params(interpolate=0)


def densify_eval(sep, out, F, stream, args):
    """Dense frames rebuilt from the batch's per-bin levels and kept lists,
    without and with a noisy background (normal deviates drawn once, outside
    the timed region), and with the radially interpolated profile.
    Algorithmic bytes per frame: the dense frame written (4N), the kept list
    read (8 per kept pixel), mean and sigma (8B), and the deviates read (4N)
    with noise; the interpolation table (8N) once per launch."""
    import torch
    N = sep.npix
    dense = torch.empty((F, N), dtype=torch.float32, device=out["mean"].device)
    z = torch.randn((F, N), dtype=torch.float32, device=out["mean"].device)
    kept = int(out["n_kept"].clamp(max=out["idx"].shape[1]).sum().item())
    res = {}
    for name, noise, smooth in (("plain", None, False), ("noise", z, False), ("smooth_noise", z, True)):
        run = lambda: sep.densify(out["mean"], out["sigma"], out["idx"], out["val"], out["n_kept"], noise=noise,
                                  out=dense, interpolate=smooth, stream=stream)
        for _ in range(2):
            run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            run()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        nbytes = 4 * N * F + 8 * kept + 8 * sep.nbins * F + (4 * N * F if noise is not None else 0) + \
            (8 * N if smooth else 0)
        gbs = nbytes / (ms * 1e-3) / 1e9
        res[name] = {"frames_s": round(F / (ms * 1e-3), 1), "ms": round(ms, 3), "achieved_gbs": round(gbs, 1),
                     "frac_of_hbm": round(gbs / peaks_file()[0]["hbm_gbs"], 4), "peak_source": peaks_file()[1]}
    del dense, z
    return res


def surrogate_eval(sep, det, mask, cal, kcap, pcap, stream, args):
    """Train the clip surrogate on JF4M frames generated on the GPU from
    another seed range (recorded by the plain clip, trained by the library's
    kernels), then run held-out frames of a third seed range with and
    without it: frames/s, how often the predicted core held (else the
    replay placed it again), row scans per bin and kept-set agreement."""
    import torch
    import synth
    from paper_2411_09515_gb300 import Surrogate, _binding as B
    spec = synth.spec_jf_serial(7777)
    device = torch.device("cuda", torch.cuda.current_device())
    cal_d = (torch.from_numpy(np.ascontiguousarray(cal[0])).to(device),
             torch.from_numpy(np.ascontiguousarray(cal[1])).to(device))
    mask_d = torch.from_numpy(np.ascontiguousarray(mask, np.uint8)).to(device)
    chunk = 512
    gen = torch.empty((chunk, det.npix), dtype=torch.int16, device=device)
    scratch = torch.empty(synth.gpu_scratch_bytes(det, spec, chunk), dtype=torch.uint8, device=device)
    ntr = args.surrogate_train_frames
    t0 = time.time()
    feats, tgts = [], []
    for i in range(0, ntr, chunk):
        n = min(chunk, ntr - i)
        synth.frames_gpu(det, spec, 1_000_000 + i, n, gen[:n], calib_dev=cal_d, mask_dev=mask_d, scratch=scratch,
                         stream=stream)
        r = sep.record(gen[:n], stream=stream)
        feats.append(r["feat"])
        tgts.append(r["target"])
    torch.cuda.synchronize()
    t_rec = time.time() - t0
    model = Surrogate(sep.ctx, seed=1)
    # about 2.5e8 row visits in all (24 epochs of a small set, 2 of 1e5 frames)
    nrows = ntr * sep.nbins
    epochs = int(min(24, max(2, round(2.5e8 / max(nrows, 1)))))
    feat_all, tgt_all = torch.cat(feats), torch.cat(tgts)
    del feats, tgts
    loss, rows = model.fit(feat_all, tgt_all, epochs=epochs, batch=1024, lr=2e-3, stream=stream)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    del feat_all, tgt_all

    # held-out frames of another seed range, generated on the GPU
    nh = args.surrogate_eval_frames
    held = torch.empty((nh, det.npix), dtype=torch.int16, device=device)
    for i in range(0, nh, chunk):
        n = min(chunk, nh - i)
        synth.frames_gpu(det, spec, 5_000_000 + i, n, held[i:i + n], calib_dev=cal_d, mask_dev=mask_d,
                         scratch=scratch, stream=stream)
    del gen, scratch
    out = sep.alloc_outputs(nh, kcap, pcap)

    def timed(steps):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            sep.process_batch(held, kcap, pcap, out=out, use_graph=True, stream=stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / steps

    def scans_per_item():
        # core scans (passes over the whole row) per bin and frame, one step
        sep.clip_stats(enable=1, read=False, reset=True, stream=stream)
        sep.process_batch(held, kcap, pcap, out=out, use_graph=True, stream=stream)
        st = sep.clip_stats(enable=0, read=True, reset=True, stream=stream)
        return round((st["core_scans"] + st["full_passes"]) / max(st["items"], 1), 4)

    steps = max(2, args.steps // 2)
    sep.attach_surrogate(None)
    timed(2)
    plain_ms = timed(steps)
    plain = {k: out[k].clone() for k in ("idx", "val", "n_kept", "count", "mean", "sigma")}
    res = {"train_frames": ntr, "train_frames_generated_on": "gpu", "train_rows": rows, "epochs": epochs,
           "train_loss": round(loss, 5), "record_s": round(t_rec, 1), "train_s": round(t_train, 1),
           "eval_frames": nh, "plain_fps": round(nh / (plain_ms * 1e-3), 2),
           "plain_row_scans_per_bin": scans_per_item()}
    sep.attach_surrogate(model)
    timed(2)
    sep.surrogate_stats(reset=True, stream=stream)
    ms = timed(steps)
    acc, fb = sep.surrogate_stats(reset=True, stream=stream)
    # kept sets against the plain path's: identical, or differing only in
    # pixels whose value lies within 1e-5 relative of the plain threshold
    # (the two paths sum the same sets in another order)
    bop = torch.from_numpy(B.sep_csr_export(sep.csr)["bin_of_pixel"]).to(device).long()
    k_pick = float(sep.params.k_pick)
    same = same_band = 0
    for f in range(nh):
        n, m = int(plain["n_kept"][f]), int(out["n_kept"][f])
        a_idx, b_idx = plain["idx"][f, :n].long(), out["idx"][f, :m].long()
        if n == m and torch.equal(a_idx, b_idx):
            same += 1
            same_band += 1
            continue
        vals = torch.cat([plain["val"][f, :n], out["val"][f, :m]])
        idx = torch.cat([a_idx, b_idx])
        u, inv, cnt = torch.unique(idx, return_inverse=True, return_counts=True)
        diff = cnt[inv] == 1
        px, v = idx[diff], vals[diff].double()
        b = bop[px]
        thr = plain["mean"][f, b].double() + k_pick * plain["sigma"][f, b].double()
        if bool(torch.all((v - thr).abs() <= 1e-5 * thr.abs())):
            same_band += 1
    res["surrogate"] = {
        "fps": round(nh / (ms * 1e-3), 2), "speedup_vs_plain": round(plain_ms / ms, 4),
        "predicted_core_held_frac": round(acc / max(acc + fb, 1), 4),
        "fallback_frac": round(fb / max(acc + fb, 1), 4),
        "row_scans_per_bin": scans_per_item(),
        "bins_same_count_frac": round(float((out["count"] == plain["count"]).float().mean().item()), 6),
        # bins whose final set differs: a clip decision within rounding of an
        # interval bound (the same sets summed in another order move mu and
        # sigma by a few units in the last place)
        "bins_other_count": int((out["count"] != plain["count"]).sum().item()),
        "frames_identical_kept": round(same / nh, 4),
        "frames_identical_kept_outside_band": round(same_band / nh, 4)}
    res.update(leg_status(sep, out, kcap, pcap))
    sep.attach_surrogate(None)
    model.close()
    del held, out
    return res


def cpu_baseline(det, mask, cal, frames_np, n, gpu_modes=None):
    """The oracle as it stands on a bounded sample of the same frames, all
    host cores; with gpu_modes (name -> (mean, sigma) of the library on those
    frames in each precision mode) also the modes' errors against the
    oracle's per-bin results."""
    import oracle
    W = oracle.weights(det, mask)
    threads = oracle.max_threads()
    n = max(1, min(n, frames_np.shape[0]))
    t0 = time.time()
    mean, sigma, _, _ = oracle.process_frames(det, W, frames_np[:n], calib=cal, threads=threads)
    dt = time.time() - t0
    res = {"value": round(n / dt, 3), "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"{n} of the batch's JF4M raw frames through oracle.process_frames (FP64), weights excluded"}
    if gpu_modes:
        prec = {"frames": n, "note": "per-bin relative error against the oracle over every bin with a "
                                     "nonzero deviation (a bin whose clip decision sits in the 1e-5 band "
                                     "may follow another trajectory; the GPU tests replay those)"}
        ok = sigma > 0
        for name, (gm, gs) in gpu_modes.items():
            em = np.abs(gm[:n] - mean) / np.maximum(np.abs(mean), 1e-2 * sigma)
            es = np.abs(gs[:n] - sigma) / np.maximum(sigma, 1e-30)
            em, es = em[ok], es[ok]
            within = (np.abs(gm[:n] - mean) <= 1e-5 * np.abs(mean) + 1e-7 * sigma) & \
                     (np.abs(gs[:n] - sigma) <= 1e-5 * sigma)
            prec[name] = {"mean_rel_err_median": float(np.median(em)), "mean_rel_err_p999": float(np.quantile(em, 0.999)),
                          "mean_rel_err_max": float(em.max()), "sigma_rel_err_median": float(np.median(es)),
                          "sigma_rel_err_p999": float(np.quantile(es, 0.999)), "sigma_rel_err_max": float(es.max()),
                          "bins_within_1e-5": float(within[ok].mean()), "bins": int(ok.sum())}
        res["precision"] = prec
    return res


def mixed_eval(n_frames, steps, warmup, kcap, pcap):
    """Uneven batching: a stream of float32 photon frames from 1M, 4M and 16M
    Jungfrau-shaped detectors (3:2:1, 600 / 1000 / 2000 bins, no splitting)
    in one call and one captured graph, schedules autotuned per detector.
    Returns aggregate frames/s and GB/s, and frames/s per detector size."""
    import torch
    import synth
    from paper_2411_09515_gb300 import Context, Separator, process_mixed
    rng = np.random.default_rng(7)
    dets = [synth.det_jf1m(nbins=600), synth.det_jf4m(split=1, nbins=1000), synth.det_jf16m(nbins=2000)]
    masks = [d.mask() for d in dets]
    groups = max(1, n_frames // 6)
    pattern = []
    for _ in range(groups):
        grp = [0, 1, 0, 2, 1, 0]
        rng.shuffle(grp)
        pattern += grp
    ctx = Context(0)
    seps = [Separator.from_detector(d, mask=m, context=ctx) for d, m in zip(dets, masks)]
    frames = []
    per = {0: [], 1: [], 2: []}
    # frames generated on the GPU (the host generator's model and streams)
    masks_d = [torch.from_numpy(np.ascontiguousarray(m, np.uint8)).cuda() for m in masks]
    for g, d in enumerate(pattern):
        spec = synth.spec_mixed(seed=1000 + g, hit_rate=float(rng.uniform(0.1, 0.5)))
        t = torch.empty(dets[d].npix, dtype=torch.float32, device="cuda")
        synth.frames_gpu(dets[d], spec, g, 1, t, mask_dev=masks_d[d])
        frames.append((d, t))
        per[d].append(t)
    torch.cuda.synchronize()
    tuned = {}
    for d in range(3):
        sample = torch.stack(per[d][:8])
        tuned[d] = {"ms": seps[d].autotune(sample), **seps[d].get_plan()}
    # 16M frames keep ~0.7 M pixels and carry up to a few thousand peaks
    kcap, pcap = max(kcap, 1 << 20), max(pcap, 1 << 15)
    for _ in range(warmup):
        out = process_mixed(seps, frames, kcap, pcap)
    torch.cuda.synchronize()
    seps[0].device_status()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        out = process_mixed(seps, frames, kcap, pcap)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    status = leg_status(seps[0], out, kcap, pcap)
    n = len(frames)
    byts = sum(4 * dets[d].npix for d in pattern)
    per_size = {}
    for d, name in enumerate(["1M", "4M", "16M"]):
        batch = torch.stack(per[d])
        o = seps[d].alloc_outputs(batch.shape[0], kcap, pcap)
        for _ in range(2):
            seps[d].process_batch(batch, kcap, pcap, out=o)
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record()
        for _ in range(steps):
            seps[d].process_batch(batch, kcap, pcap, out=o)
        a1.record()
        torch.cuda.synchronize()
        per_size[name] = round(batch.shape[0] / (a0.elapsed_time(a1) / steps) * 1e3, 1)
    res = {"frames_s": round(n / ms * 1e3, 2), "ms_per_step": round(ms, 3), "frames_per_step": n,
           "sizes": {"1M": len(per[0]), "4M": len(per[1]), "16M": len(per[2])},
           "gbs_input": round(byts / (ms * 1e-3) / 1e9, 1), "per_size_frames_s": per_size, "plans": tuned,
           **status}
    for sp in seps:
        sp.close()
    ctx.close()
    return res


def run_mixed(args):
    r = mixed_eval(args.frames, args.steps, args.warmup, args.kept_capacity, args.peak_capacity)
    line = {"metric": "mixed 1M/4M/16M frames/s (clip+sparsify+peaks), one graph", "value": r["frames_s"],
            "unit": "frames/s", "ms_per_step": r["ms_per_step"], "steps": args.steps, "warmup": args.warmup,
            "dtype": "f32", "data": "synthetic", **r,
            "config": {"workload": "mixed f32 1M:4M:16M = 3:2:1, 600/1000/2000 bins, no split"}}
    print(json.dumps(line), flush=True)


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    F = args.frames
    n = max(1, min(args.cpu_frames, F))
    det, mask, cal, frames_np = setup_workload(n, 0)
    W = oracle.weights(det, mask)
    threads = oracle.max_threads()
    for _ in range(min(args.warmup, 1)):
        oracle.process_frames(det, W, frames_np[:1], calib=cal, threads=threads)
    t0 = time.time()
    for _ in range(args.steps):
        oracle.process_frames(det, W, frames_np, calib=cal, threads=threads)
    dt = time.time() - t0
    value = n * args.steps / dt
    line = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * dt / args.steps, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "frames_per_step": n}, "impl": "reference",
            "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{n} JF4M raw frames per step (bounded sample of the batch)"},
            "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--frames", type=int, default=512)
    ap.add_argument("--kept-capacity", type=int, default=262144)  # mixed: raised to fit 16M frames
    ap.add_argument("--peak-capacity", type=int, default=8192)
    ap.add_argument("--cpu-frames", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--clip-plan", default="", help="fixed clip schedule 'T1,T2:W1,W2,W3' instead of the autotuner")
    ap.add_argument("--chunk-frames", type=int, default=64)
    ap.add_argument("--surrogate-train-frames", type=int, default=100000)
    ap.add_argument("--surrogate-eval-frames", type=int, default=1024)
    ap.add_argument("--mixed-frames", type=int, default=96)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["plain", "kahan", "fp64merge", "dword"], default="dword")
    ap.add_argument("--workload", choices=["jf4m", "mixed"], default="jf4m")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "mixed":
        run_mixed(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
