#!/usr/bin/env python3
"""Throughput of the anisotropic-diffusion hot path on GB300.

Workload (one "step"): the 512 x 512 x 256 float32 H I cube (four inclined
rotating disks and one faint tail in unit Gaussian noise, seed 0), resident in
HBM:
  a1  noise rms of the input (FP64 reduction) -> K = 1.0 * sigma
  a3-a6  50 per-face Perona-Malik iterations, rational conductance,
         dt = 1/8, zero-flux faces, out of place (the input stays intact)
  a8  FP64 sum of the result (conservation check)
Metric: Gvoxel-iterations per second = voxels * iterations / time.

Multi-GPU (torchrun): every rank filters its own cube (independent problems,
no collective on the data path; weak scaling); timing is the max over ranks.

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("Gvoxel-iter/s and % of HBM roofline (FP32 vs FP16-stored) at stated error; "
          "p50/p99 latency")
UNIT = "Gvoxel-iter/s"
N_ITER, DT, K_SIGMA, COND = 50, 1.0 / 8, 1.0, "rational"
SHAPE = (256, 512, 512)
WORKLOAD = ("cube512: 512x512x256 float32 (x, y, velocity), noise sigma=1, 4 disks "
            "(i = 20/45/70/85 deg) + 1 faint tail, seed 0; rational g, K = 1.0 sigma "
            "(GPU FP64 noise rms), dt = 1/8, 50 iterations, zero-flux faces")
FALLBACK_HBM_GBS = 6800.0
PROFILE = os.path.join(ROOT, "profiles", "pm_step_stream_cube512.md")
KERNEL_SOURCES = ["paper_1609_03782_gb300/csrc/pm_stream.cu",
                  "paper_1609_03782_gb300/csrc/afd_math.cuh",
                  "paper_1609_03782_gb300/csrc/afd_ptx.cuh"]


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__,
                                 formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["afd", "reference"], default="afd")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--lines",
                    default="paper,diagnostics,smoothing,precision,slabs,batch,serving",
                    help="extra lines measured after the headline (N=1 only): any of "
                         "paper, diagnostics, smoothing, precision, slabs, batch, serving, or "
                         "'none'")
    ap.add_argument("--serve-seconds", type=float, default=4.0,
                    help="arrival window per request rate of the serving line")
    return ap.parse_args()


# ----------------------------------------------------------------------------
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source (else None)."""
    try:
        text = open(PROFILE).read()
    except OSError:
        return None
    m = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]{16})", text)
    t = re.search(r"dram_bytes_per_launch_full_size:\s*([0-9.eE+]+)", text)
    if not m or not t or m.group(1) != kernel_source_hash():
        return None
    return float(t.group(1))


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_uuid: str | None):
        self.rows, self.proc, self.thread = [], None, None
        self.uuid = device_uuid

    def start(self):
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
               "-lms", "100"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        rows = [r for r in self.rows if len(r) == 8]
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(rows), "reasons": sorted(reasons)}


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ----------------------------------------------------------------------------
def oracle_rate(cube, K, shape, repeats=1):
    """Time the FP64 oracle (single thread) on the corner sub-cube `shape`."""
    import oracle
    nz, ny, nx = shape
    sub = cube[:nz, :ny, :nx].copy()
    oracle.build()
    t0 = time.perf_counter()
    for _ in range(repeats):
        oracle.pm_filter(sub, K, DT, N_ITER, COND)
    dt = time.perf_counter() - t0
    return sub.size * N_ITER * repeats / dt / 1e9, dt


def run_reference(args):
    """The oracle as it stands, on host cores, on a bounded sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    import synth
    cube = synth.cube512()
    K = K_SIGMA * oracle.noise_rms(cube)
    shape = (16, 64, 64)   # one step: 65,536 voxels x 50 iterations
    for _ in range(args.warmup):
        oracle_rate(cube, K, shape)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_rate(cube, K, shape)
    el = time.perf_counter() - t0
    n_vox = shape[0] * shape[1] * shape[2]
    value = n_vox * N_ITER * args.steps / el / 1e9
    sample = ("corner sub-cube %dx%dx%d of the 512x512x256 cube, 50 rational iterations "
              "per step, FP64 single-threaded C oracle" % (shape[2], shape[1], shape[0]))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0



# ----------------------------------------------------------------------------
# Extra lines (1 GPU): precision, batching, serving.
def _events_ms(fn, reps):
    import torch
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def pow2_near(v: float) -> float:
    """The power of two nearest v (log2 rounded half up): a cube's scale."""
    return 2.0 ** math.floor(math.log2(v) + 0.5) if v > 0 and math.isfinite(v) else 1.0


# Thread-instructions per voxel-iteration of the precision line's kernels
# (ncu, full size; profiles/precision_instructions_cube512.md), keyed by
# (storage, T); with the issue rate of the GPU they give each row's issue
# ceiling beside its HBM ceiling.
INSTR_PER_VOXEL_ITER = {("f32", 1): 29.9,
                        ("f16", 1): 30.86, ("f16", 2): 44.30, ("f16", 4): 41.14,
                        ("bf16", 1): 30.86, ("bf16", 2): 44.30, ("bf16", 4): 41.14,
                        ("i16", 1): 39.42, ("i16", 2): 47.89, ("i16", 4): 43.00}
ISSUE_THREAD_INSTR_PER_S = 152 * 4 * 32 * 2.07e9   # SMs x schedulers x lanes x clock


def ceilings(storage: str, T: int, value: float, peak_gbs: float):
    """HBM and issue ceilings (Gvox-it/s) of a pass, the one that binds, and
    the fraction of it reached."""
    b = 4.0 if storage == "f32" else 2.0
    hbm = peak_gbs / (2.0 * b / T)
    ins = INSTR_PER_VOXEL_ITER.get((storage, T))
    issue = ISSUE_THREAD_INSTR_PER_S / ins / 1e9 if ins else None
    bound = "issue" if issue is not None and issue < hbm else "hbm"
    lim = issue if bound == "issue" else hbm
    return {"hbm_ceiling": hbm, "issue_ceiling": issue, "thread_instr_per_voxel_iter": ins,
            "bound": bound, "frac_of_bound": value / lim}


def line_precision(afd, ctx, cube, d_in, ref32, sig):
    """2-byte storage (per-cube power-of-two scale) x temporal depth on the
    benchmark cube; error against the float32 GPU result over the whole cube
    (the float32 path itself is within 1e-4 sigma of the FP64 oracle, which the
    test-suite checks), in units of sigma."""
    import numpy as np
    import torch
    n_vox = cube.size
    K = K_SIGMA * sig
    scale = pow2_near(sig)
    dt = {"f16": torch.float16, "bf16": torch.bfloat16, "i16": torch.int16}
    ref = ref32.cpu().numpy()
    faint = np.abs(ref) < 3.0 * sig
    rows = []
    for st in ("f16", "bf16", "i16"):
        q = torch.empty(cube.shape, dtype=dt[st], device=d_in.device)
        o = torch.empty_like(q)
        back = torch.empty_like(d_in)
        afd.afd_quantize(ctx, d_in, q, st, scale)
        for T in (1, 2, 4):
            run = lambda: afd.afd_filter_ex(ctx, q, o, st, scale, K, DT, N_ITER, COND, None, T)
            run()
            ms = _events_ms(run, 5)
            afd.afd_dequantize(ctx, o, back, st, scale)
            afd.afd_sync(ctx)
            got = back.cpu().numpy()
            err = np.abs(got - ref)
            value = n_vox * N_ITER / (ms / 1e3) / 1e9
            rows.append({"storage": st, "t_block": T, "ms": ms, "value": value,
                         "bytes_per_voxel_iter": 4.0 / T,
                         **ceilings(st, T, value, measured_peaks()[0]),
                         "err_vs_f32_max_sigma": float(err.max()) / sig,
                         "err_vs_f32_rms_sigma": float(np.sqrt(np.mean(err ** 2))) / sig,
                         "err_faint_max_sigma": float(err[faint].max()) / sig,
                         "err_faint_rms_sigma": float(np.sqrt(np.mean(err[faint] ** 2))) / sig})
    best = max(rows, key=lambda r: r["value"])
    return {"unit": UNIT, "scale": scale, "workload": "the headline cube, K = 1.0 sigma, "
            "dt = 1/8, 50 rational iterations, stored in 2 bytes with a power-of-two scale; "
            "t_block iterations per pass over HBM; errors against the float32 result over "
            "the whole cube, in units of sigma (faint: |I| < 3 sigma); per row the HBM "
            "ceiling (measured copy GB/s over 2 b / T bytes) and the issue ceiling (152 SMs x "
            "4 x 32 lanes x 2.07 GHz over the ncu thread-instructions per voxel-iteration), "
            "and which binds",
            "best": {"storage": best["storage"], "t_block": best["t_block"],
                     "value": best["value"]}, "rows": rows}


def line_paper_form(afd, ctx):
    """The paper's own benchmark: its intensity-driven filter with its defaults
    (K = 1.5, tau = 0.0325, n = 20, C = 5) on a cube of the size of its
    benchmark cube (N = 1.4e8 voxels); device-only and with the host <->
    device copies the paper includes in its GPU timing."""
    import torch
    import synth
    shape = (536, 512, 512)  # 1.405e8 voxels
    cube = synth.galaxy_cube(shape, 0, 8, 2)
    n_vox = cube.size
    d_in = torch.from_numpy(cube).cuda()
    d_out = torch.empty_like(d_in)
    rms = afd.afd_noise_rms(ctx, d_in)
    C = (5.0, 5.0, 5.0)
    run = lambda: afd.afd_filter_intensity(ctx, d_in, d_out, 1.5, rms, 0.0325, 20, C)
    run()
    ms = _events_ms(run, 10)
    h_in = torch.from_numpy(cube).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()

    def e2e():
        d_in.copy_(h_in, non_blocking=True)
        afd.afd_filter_intensity(ctx, d_in, d_out, 1.5, rms, 0.0325, 20, C)
        h_out.copy_(d_out, non_blocking=True)
        torch.cuda.current_stream().synchronize()

    e2e()
    t0 = time.perf_counter()
    for _ in range(5):
        e2e()
    e_ms = (time.perf_counter() - t0) / 5 * 1e3
    return {"unit": UNIT, "workload": "intensity-driven form, K = 1.5 (units of the GPU noise "
            "rms), tau = 0.0325, n = 20, C = 5 (the paper's defaults), on a 512x512x536 "
            "synthetic cube (1.41e8 voxels, the size of the paper's benchmark cube)",
            "value": n_vox * 20 / (ms / 1e3) / 1e9, "ms": ms,
            "e2e_value": n_vox * 20 / (e_ms / 1e3) / 1e9, "e2e_ms": e_ms,
            "paper_context": {"gtx860m_opengl_incl_io_gvox_it_s": 0.90,
                              "i7_8core_openmp_gvox_it_s": "0.036-0.050",
                              "note": "other hardware, other data (NGC 2841); context only"}}


def line_diagnostics(afd, ctx, d_in, d_out):
    """F / F_M diagnostics (Sec. 4, Sec. 5): throughput of the one-pass masked
    sums on the benchmark cube (original + filtered, 8 B per voxel), and the
    paper's Tab. 3 parameter grid for the intensity form (C = 5) on the
    ModelB stand-in, F +- sigma_F and F_M over the faint tail's ROI."""
    import torch
    import synth
    n_vox = d_in.numel()
    rms_o = afd.afd_noise_rms(ctx, d_in)
    rms_f = afd.afd_noise_rms(ctx, d_out)
    call = lambda: afd.afd_f_diagnostic(ctx, d_in, d_out, rms_o=rms_o, rms_f=rms_f)
    for _ in range(3):
        call()
    reps = 30
    t0 = time.perf_counter()
    for _ in range(reps):
        r = call()
    us = (time.perf_counter() - t0) / reps * 1e6
    peak, peak_kind = measured_peaks()
    gbs = 8.0 * n_vox / us / 1e3
    cube, model, roi = synth.model_b()
    d_o = torch.from_numpy(cube).to(d_in.device)
    d_m = torch.from_numpy(model).to(d_in.device)
    d_f = torch.empty_like(d_o)
    rms = afd.afd_noise_rms(ctx, d_o)
    grid = [(0.5, 0.0325, 20), (0.5, 0.0625, 20), (0.5, 0.0325, 30), (0.5, 0.0625, 30),
            (1.0, 0.0325, 20), (1.0, 0.0325, 30), (1.5, 0.0325, 20), (1.5, 0.0325, 30),
            (2.0, 0.0325, 20), (2.0, 0.0325, 30)]
    rows = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for K, tau, n in grid:
        afd.afd_filter_intensity(ctx, d_o, d_f, K, rms, tau, n, (5.0, 5.0, 5.0))
        q = afd.afd_f_diagnostic(ctx, d_o, d_f, d_m, roi=roi)
        rows.append({"K": K, "tau": tau, "n": n, "F": q["F"], "sigma_F": q["sigma_F"],
                     "F_M": q["F_M"]})
    sweep_ms = (time.perf_counter() - t0) * 1e3
    return {"fdiag": {"workload": "masked F sums over the benchmark cube and its 50-iteration "
                                  "result (268 MB each), rms given, synchronous call",
                      "us_per_call": us, "algorithmic_GBs": gbs, "peak_GBs": peak,
                      "frac": gbs / peak, "peak_kind": peak_kind, "F": r["F"],
                      "N_o": r["N_o"], "N_f": r["N_f"]},
            "tab3_sweep": {"workload": "intensity form, C = 5, the (K, tau, n) grid of the "
                                       "paper's Tab. 3, on the ModelB stand-in (104x104x64, "
                                       "disk of peak SNR 32 + a 0.75-sigma tail, unit noise, "
                                       "seed 0); F, sigma_F and F_M over the tail's ROI "
                                       + str(roi),
                           "runs": rows, "ms_total": sweep_ms}}


def line_smoothing(afd, ctx):
    """Box and Gaussian smoothing (Sec. 3.1, 3.2) on a cube of the paper's
    benchmark size (512x512x536): one fused separable pass for the box and
    the axis-aligned Gaussian, the direct 3-D correlation for a rotated
    Gaussian.  Algorithmic bytes: 8 per voxel (read + write once)."""
    import numpy as np
    import torch
    import synth
    cube = synth.galaxy_cube((536, 512, 512), 0, 8, 2)
    d_in = torch.from_numpy(cube).cuda()
    d_out = torch.empty_like(d_in)
    n_vox = cube.size
    peak, peak_kind = measured_peaks()
    runs = {"box 3x5x3 (Tab. 1 ModelB)": lambda: afd.afd_smooth_box(ctx, d_in, d_out, (3, 5, 3)),
            "box 9x9x9": lambda: afd.afd_smooth_box(ctx, d_in, d_out, (9, 9, 9)),
            "gauss FWHM 3,5,3 (Tab. 1 ModelB)":
                lambda: afd.afd_smooth_gauss(ctx, d_in, d_out, (3.0, 5.0, 3.0)),
            "gauss FWHM 3,3,3 (isotropic)":
                lambda: afd.afd_smooth_gauss(ctx, d_in, d_out, (3.0, 3.0, 3.0)),
            "gauss FWHM 3,5,3 rotated 0,0,30 deg (direct 3-D)":
                lambda: afd.afd_smooth_gauss(ctx, d_in, d_out, (3.0, 5.0, 3.0), (0.0, 0.0, 30.0))}
    # taps per voxel of the rotated kernel (the direct pass is bound by its
    # FP32 multiply-adds, not by HBM): radius ceil(3 sqrt(Sigma_aa)) per axis
    sig = np.array([3.0, 5.0, 3.0]) / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    th = math.radians(30.0)
    Rz = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    cov = Rz @ np.diag(sig ** 2) @ Rz.T
    taps = int(np.prod([2 * math.ceil(3.0 * math.sqrt(cov[a, a]) - 1e-12) + 1 for a in range(3)]))
    fma_peak = 152 * 128 * 2.07e9   # FP32 lanes x clock: one FMA per lane per cycle
    rows = []
    for name, fn in runs.items():
        fn()
        ms = _events_ms(fn, 5)
        gbs = 8.0 * n_vox / (ms / 1e3) / 1e9
        row = {"filter": name, "ms": ms, "gvox_s": n_vox / (ms / 1e3) / 1e9}
        if "direct" in name:
            fma_s = taps * n_vox / (ms / 1e3)
            row.update({"bound": "alu", "taps_per_voxel": taps, "fma_per_s": fma_s,
                        "peak_fma_per_s": fma_peak, "frac": fma_s / fma_peak,
                        "peak_note": "152 SMs x 128 FP32 lanes x 2.07 GHz"})
        else:
            row.update({"bound": "hbm", "algorithmic_GBs": gbs, "frac": gbs / peak})
        rows.append(row)
    return {"workload": "512x512x536 float32 synthetic cube (8 disks + 2 tails, seed 0), "
                        "normalised correlation, out of place", "peak_GBs": peak,
            "peak_kind": peak_kind, "rows": rows,
            "paper_context": {"gtx860m_gauss_iso_s": 1.8, "gtx860m_gauss_aniso_s": 3.5,
                              "note": "N = 1.4e8, other hardware; context only"}}


def line_slabs(afd, ctx, cube, sig):
    """A cube filtered out of host memory through a small device budget
    (afd_filter_slabs): z-slabs with halo planes, rounds of `halo`
    iterations, copies overlapped with the passes.  The cube is the headline
    cube stacked four times along z (512 x 512 x 1024, 1 GiB); host to host,
    pinned buffers.  Context: the same cube through afd_filter_host (whole
    cube on the device)."""
    import numpy as np
    import torch
    big = np.ascontiguousarray(np.tile(cube, (4, 1, 1)))
    nz, ny, nx = big.shape
    plane = nx * ny * 4
    n_vox = big.size
    K = K_SIGMA * sig
    h_in = torch.from_numpy(big).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    h_tmp = torch.empty_like(h_in).pin_memory()
    rows = []
    for slab_nz, halo in ((64, 10), (64, 25), (128, 25), (128, 50)):
        run = lambda: afd.afd_filter_slabs(ctx, h_in, h_out, K, DT, N_ITER, COND, None,
                                           slab_nz, halo, h_tmp)
        run()
        secs = []
        for _ in range(5):   # median of 5: the host link is shared with the host's other work
            t0 = time.perf_counter()
            run()
            secs.append(time.perf_counter() - t0)
        sec = statistics.median(secs)
        rounds = -(-N_ITER // halo)
        slabs = -(-nz // slab_nz)
        # planes copied in per round: every slab with its ghost planes
        planes_in = sum(min(nz, z0 + slab_nz + halo) - max(0, z0 - halo)
                        for z0 in range(0, nz, slab_nz))
        moved = rounds * (planes_in + nz) * plane
        rows.append({"slab_nz": slab_nz, "halo": halo, "rounds": rounds, "slabs": slabs,
                     "device_bytes": 4 * min(nz, slab_nz + 2 * halo) * plane,
                     "s": sec, "samples_s": secs, "value": n_vox * N_ITER / sec / 1e9,
                     "host_link_GBs": moved / sec / 1e9})
    t0 = time.perf_counter()
    afd.afd_filter_host(ctx, h_in, h_out, K, DT, N_ITER, COND)
    whole = time.perf_counter() - t0
    best = max(rows, key=lambda r: r["value"])
    return {"unit": UNIT, "workload": "the headline cube stacked 4x along z (512x512x1024 "
            "float32, 1 GiB) in pinned host memory, K = 1.0 sigma, dt = 1/8, 50 rational "
            "iterations, host to host; device_bytes: the two staging slots (in + out) at "
            "the largest slab, besides a pass scratch of one slab",
            "best": {"slab_nz": best["slab_nz"], "halo": best["halo"], "value": best["value"]},
            "rows": rows,
            "whole_cube_host": {"s": whole, "value": n_vox * N_ITER / whole / 1e9,
                                "device_bytes": 3 * n_vox * 4}}


def line_batch(afd, ctx):
    """300 galaxy cutouts of uneven size, K_i = 1.5 sigma_i (GPU FP64 noise
    estimate), 20 iterations, one CUDA-graph launch per call; z-chunk picked
    by the autotuner."""
    import torch
    import synth
    from paper_1609_03782_gb300 import tune
    shapes = synth.cutout_shapes(0, 300)
    nvox = sum(a * b * c for a, b, c in shapes)
    tuner = tune.Tuner(cache_path=None, reps=3)
    out = {"unit": UNIT, "cubes": len(shapes), "voxels": nvox,
           "workload": "300 cutouts, nx, ny ~ U{32..256}, nz ~ U{32..128}, one disk each in "
                       "unit noise (seed 0); K_i = 1.5 sigma_i from the GPU FP64 noise rms; "
                       "rational g, dt = 1/8, 20 iterations; one graph launch per call "
                       "(statistics + coefficients + 20 batched passes)"}
    for st in ("f32", "f16"):
        b = afd.afd_batch_create(ctx, shapes, st, 1.0)
        for i, s in enumerate(shapes):
            t = torch.from_numpy(synth.cutout(s, 0 * 100003 + 1 + i)).cuda()
            if st == "f16":
                q = torch.empty(s, dtype=torch.float16, device="cuda")
                afd.afd_quantize(ctx, t, q, "f16", 1.0)
                t = q
            afd.afd_batch_set(b, i, t)
        K = [-1.5] * len(shapes)
        zc = tuner.tune_batch(afd, b, K, DT, 20, COND)
        run = lambda: afd.afd_batch_filter(b, K, DT, 20, COND)
        run()
        ms = _events_ms(run, 10)
        out[st] = {"ms_per_call": ms, "value": nvox * 20 / (ms / 1e3) / 1e9, "zchunk": zc,
                   "tuning_ms": tuner.cache[tune.batch_key(shapes, st, COND, 20)]["ms"]}
        b.close()
        torch.cuda.synchronize()
    return out


def line_serving(afd, ctx, seconds):
    """64 resident float16 cubes (21 x 128^3, 21 x 256^3, 22 x 512x512x128);
    Poisson arrivals; each request a re-filter with K ~ U[0.5, 3] sigma and
    1-50 iterations; admitted by free HBM; p50/p99 latency submit -> done."""
    import numpy as np
    import torch
    import synth
    shapes = synth.serving_shapes()
    b = afd.afd_batch_create(ctx, shapes, "f16", 1.0)
    sig = []
    for i, s in enumerate(shapes):
        t = torch.from_numpy(synth.serving_cube(i)).cuda()
        sig.append(afd.afd_noise_rms(ctx, t))
        q = torch.empty(s, dtype=torch.float16, device="cuda")
        afd.afd_quantize(ctx, t, q, "f16", 1.0)
        afd.afd_batch_set(b, i, q)
        del t
    afd.afd_sync(ctx)
    budget = 16 << 30
    srv = afd.afd_serve_create(b, budget, 128)
    rng = np.random.default_rng(0)
    res = {"unit": "ms", "workload": "64 resident float16 cubes (21 x 128^3, 21 x 256^3, "
           "22 x 512x512x128, seed 0); Poisson arrivals for %.1f s per rate; each request a "
           "random cube, K ~ U[0.5, 3] sigma_cube, n ~ U{1..50}, rational g, dt = 1/8; "
           "HBM budget 16 GiB for results + scratch; latency from the scheduled arrival to "
           "the completion of the request's last round" % seconds, "rates": []}
    for lam in (50, 100, 200, 500):
        gaps = rng.exponential(1.0 / lam, size=int(lam * seconds * 3) + 10)
        arrivals = np.cumsum(gaps)
        arrivals = arrivals[arrivals < seconds]
        reqs = [(int(rng.integers(0, len(shapes))), float(rng.uniform(0.5, 3.0)),
                 int(rng.integers(1, 51))) for _ in arrivals]
        lat, work, live, k = [], 0.0, {}, 0
        t0 = time.perf_counter()
        while k < len(arrivals) or live:
            now = time.perf_counter() - t0
            while k < len(arrivals) and arrivals[k] <= now:
                c, ks, n = reqs[k]
                lag = (time.perf_counter() - t0) - arrivals[k]
                tk = afd.afd_serve_submit(srv, c, ks * sig[c], DT, n, COND)
                live[tk] = (lag, c, n)
                k += 1
            afd.afd_serve_step(srv, wait=False)
            for tk in list(live):
                st, l = afd.afd_serve_poll(srv, tk)
                if st == 2:
                    lag, c, n = live.pop(tk)
                    lat.append((l + lag) * 1e3)
                    a, bb, cc = shapes[c]
                    work += float(a) * bb * cc * n
                    afd.afd_serve_release(srv, tk)
            if not live and k < len(arrivals):
                time.sleep(max(0.0, min(0.001, arrivals[k] - (time.perf_counter() - t0))))
        el = time.perf_counter() - t0
        lat = np.array(lat)
        res["rates"].append({"lambda_per_s": lam, "requests": int(len(lat)),
                             "p50_ms": float(np.percentile(lat, 50)),
                             "p99_ms": float(np.percentile(lat, 99)),
                             "mean_ms": float(lat.mean()),
                             "throughput_req_per_s": len(lat) / el,
                             "throughput_gvox_iter_per_s": work / el / 1e9})
    srv.close()
    b.close()
    torch.cuda.synchronize()
    return res


# ----------------------------------------------------------------------------
def run_afd(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import synth
    from paper_1609_03782_gb300 import afd

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    from paper_1609_03782_gb300 import ranks
    barrier = ranks.barrier

    def max_over_ranks(x: float) -> float:
        return ranks.max_over_ranks(x, dev)

    cube = synth.cube512()
    n_vox = cube.size
    d_in = torch.from_numpy(cube).to(dev)
    d_out = torch.empty_like(d_in)
    out4 = torch.zeros(4, dtype=torch.float64, device=dev)
    ctx = afd.afd_create(local)
    stream = torch.cuda.current_stream(dev)


    K_dev = torch.zeros(1, dtype=torch.float32, device=dev)

    def step():
        # a1 noise rms, a2 K = 1.0 rms and the coefficients (on the device),
        # a3-a6 the 50 passes; then a8 the statistics of the result
        afd.afd_filter_rel(ctx, d_in, d_out, K_SIGMA, DT, N_ITER, COND, K_out=K_dev)
        afd.afd_stats(ctx, d_out, out4)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize(dev)
    afd.afd_sync(ctx)
    sig = float(K_dev.item()) / K_SIGMA
    afd.afd_pass_timing_read(ctx)          # clear
    afd.afd_pass_timing(ctx, True)         # events around each call's passes

    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    clocks.start()
    time.sleep(0.3)
    launches0 = afd.afd_launch_count(ctx)
    barrier()
    torch.cuda.synchronize(dev)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clk = clocks.stop()
    afd.afd_sync(ctx)
    launches = afd.afd_launch_count(ctx) - launches0
    ms = max_over_ranks(t0.elapsed_time(t1))
    afd.afd_pass_timing(ctx, False)
    filt_ms, filt_passes = afd.afd_pass_timing_read(ctx)
    assert filt_passes == args.steps * N_ITER, filt_passes
    launch_ms = max_over_ranks(filt_ms / filt_passes)

    # conservation of the last step's result (FP64 sums of the FP32 fields)
    s_in = afd.afd_sum(ctx, d_in)
    s_out = float(out4[0].item())
    drift = abs(s_out - s_in) / float(np.abs(cube.astype(np.float64)).sum())

    value = world * n_vox * N_ITER * args.steps / (ms / 1e3) / 1e9
    peak, peak_kind = measured_peaks()
    bytes_per_launch = 8.0 * n_vox       # read + write of one float32 cube
    achieved = bytes_per_launch / (launch_ms / 1e3) / 1e9

    # ---- end to end through the host entry point: H2D + filter + D2H ----
    K_host = K_SIGMA * sig
    h_in = torch.from_numpy(cube).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    for _ in range(2):
        afd.afd_filter_host(ctx, h_in, h_out, K_host, DT, N_ITER, COND)
    barrier()
    te = time.perf_counter()
    for _ in range(args.e2e_steps):   # one cube at a time: copies, passes, copies
        afd.afd_filter_host(ctx, h_in, h_out, K_host, DT, N_ITER, COND)
    te = max_over_ranks(time.perf_counter() - te)
    e2e_sync_value = world * n_vox * N_ITER * args.e2e_steps / te / 1e9
    # a stream of cubes: each call's copies overlap the previous call's
    # passes.  Three rounds, the median reported (all listed): the overlap
    # depends on the host keeping ahead of the GPU, and a shared host can
    # delay one round.
    for _ in range(2):
        afd.afd_filter_host_async(ctx, h_in, h_out, K_host, DT, N_ITER, COND)
    afd.afd_sync(ctx)
    e2e_rounds = []
    for _ in range(3):
        barrier()
        te = time.perf_counter()
        for _ in range(args.e2e_steps):
            afd.afd_filter_host_async(ctx, h_in, h_out, K_host, DT, N_ITER, COND)
        afd.afd_sync(ctx)
        te = max_over_ranks(time.perf_counter() - te)
        e2e_rounds.append(world * n_vox * N_ITER * args.e2e_steps / te / 1e9)
    e2e_value = statistics.median(e2e_rounds)

    lines = {}
    if rank == 0 and world == 1 and args.lines != "none":
        want = set(args.lines.split(","))
        if "paper" in want:
            lines["paper"] = line_paper_form(afd, ctx)
        if "smoothing" in want:
            lines["smoothing"] = line_smoothing(afd, ctx)
        if "diagnostics" in want:
            lines["diagnostics"] = line_diagnostics(afd, ctx, d_in, d_out)
        if "precision" in want:
            lines["precision"] = line_precision(afd, ctx, cube, d_in, d_out, sig)
        if "slabs" in want:
            lines["slabs"] = line_slabs(afd, ctx, cube, sig)
        if "batch" in want:
            lines["batch"] = line_batch(afd, ctx)
        if "serving" in want:
            lines["serving"] = line_serving(afd, ctx, args.serve_seconds)

    line = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            shape = (128, 256, 256)
            rate, secs = oracle_rate(cube, K_SIGMA * sig, shape)
            cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": "FP64 C oracle, single thread, on the 256x256x128 corner "
                             "sub-cube of the same cube, 50 rational iterations (%.1f s)"
                             % secs}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD,
                       "parallelism": "one independent cube per GPU" if world > 1 else "1 GPU",
                       "input_sha256": synth.sha256(cube),
                       "l2": "inputs larger than L2 (268 MB cube in + 268 MB out + 268 MB "
                             "ping-pong scratch vs 129 MB L2); no flush",
                       "step": "afd_filter_rel: a1 noise rms, a2 K = 1.0 rms and coefficients "
                               "on the device, 50 filter iterations out of place; then a8 "
                               "statistics of the result (no host round trip in the step)"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "kernel": "pm_step_stream (one iteration per launch)",
                         "timing": "CUDA events recorded by the library on its stream around "
                                   "each call's 50 passes (afd_pass_timing), summed over the "
                                   "timed steps",
                         "bytes_per_launch": bytes_per_launch,
                         "launch_ms": launch_ms, "traffic": profiled_traffic()},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * n_vox,
                    "d2h_bytes_per_step": 4 * n_vox,
                    "path": "afd_filter_host_async, one call per step (a stream of cubes): "
                            "pinned host in -> device -> 50 iterations -> pinned host out; "
                            "a call's copies overlap the previous call's passes; afd_sync "
                            "after the last step; median of 3 rounds",
                    "rounds": e2e_rounds,
                    "sync_value": e2e_sync_value,
                    "sync_path": "afd_filter_host (one cube at a time, synchronous: copies "
                                 "and passes in series)"},
            "gpu_launches": launches,
            "clocks": clk,
            "noise_rms": sig,
            "sum_drift_rel": drift,
            "lines": lines,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_afd(args)


if __name__ == "__main__":
    sys.exit(main())
