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
FIGURES = os.path.join(ROOT, "profiles", "figures.json")


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
    ap.add_argument("--serve-requests", type=int, default=10000,
                    help="requests per arrival rate of the serving line (open loop)")
    ap.add_argument("--serve-max-seconds", type=float, default=60.0,
                    help="cap on the arrival window per rate of the serving line")
    ap.add_argument("--saturation-requests", type=int, default=5000,
                    help="requests of the serving line's closed-loop saturation run")
    ap.add_argument("--no-cpu-openmp", action="store_true",
                    help="skip the multithreaded CPU build's timing")
    ap.add_argument("--split", choices=["cubes", "slabs"], default="cubes",
                    help="with N ranks: 'cubes' gives every rank its own cube (weak "
                         "scaling); 'slabs' splits ONE cube into z-slabs over the ranks, "
                         "exchanging ghost planes each round (strong scaling)")
    ap.add_argument("--slab-halo", type=int, default=10,
                    help="ghost planes (= iterations per round) of --split slabs")
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


def files_hash(files) -> str:
    """sha256 (first 16 hex digits) of the repository files, in order."""
    h = hashlib.sha256()
    for rel in files:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def figure(section: str, key: str):
    """A figure of profiles/figures.json (taken from an ncu capture), or None
    if it is absent or its sources have changed since the capture."""
    try:
        with open(FIGURES) as fh:
            ent = json.load(fh)[section][key]
        if files_hash(ent["files"]) != ent["sha256_16"]:
            return None
        return float(ent["value"])
    except (OSError, KeyError, ValueError):
        return None


def profiled_traffic():
    """DRAM bytes per launch of the headline pass (ncu), if taken on the
    current kernel source."""
    return figure("dram_bytes_per_launch", "pm_step_stream_f32_cube512")


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


# the largest int16 count in units of the scale (AFD_I16FIX: counts of scale/1024)
I16_RANGE = 32767.0 / 1024.0


def i16_scale(max_abs: float) -> float:
    """The finest power-of-two scale whose int16 range (I16_RANGE x scale)
    holds max_abs.  The filter's result stays inside the input's range: each
    explicit update is a convex combination of the voxel and its six
    neighbours (the face weights dt g / h^2 sum to at most 6/8 < 1 with
    g <= 1), so the filtered cube fits the same scale."""
    if not (max_abs > 0 and math.isfinite(max_abs)):
        return 1.0
    return 2.0 ** math.ceil(math.log2(max_abs / I16_RANGE))


class Issue:
    """Thread-instruction issue rate of the GPU: SMs x 4 schedulers x 32
    lanes x SM clock.  The SM count comes from the device, the clock from
    the nvidia-smi samples of the headline's timed region (else the measured
    peaks file's maximum)."""
    sm_count = 152
    sm_mhz = 2070.0

    @classmethod
    def rate(cls) -> float:
        return cls.sm_count * 4 * 32 * cls.sm_mhz * 1e6


def pass_bytes(storage: str, T: int) -> float:
    """HBM bytes per voxel-iteration of afd_filter_ex at depth T (the
    default kernels): one read and one write of the stored cube at depth 1;
    from depth 2 on, a chain of T one-iteration launches whose intermediate
    cubes are float32 (storage -> float32 -> ... -> storage)."""
    b = 4.0 if storage == "f32" else 2.0
    return (2.0 * b + 8.0 * (T - 1)) / T


def ceilings(storage: str, T: int, value: float, peak_gbs: float):
    """HBM and issue ceilings (Gvox-it/s) of a pass, the one that binds, and
    the fraction of it reached.  The issue ceiling needs the pass's
    thread-instructions per voxel-iteration from an ncu capture of the
    current source (profiles/figures.json)."""
    hbm = peak_gbs / pass_bytes(storage, T)
    ins = figure("thread_instr_per_voxel_iter", "%s/%d" % (storage, T))
    issue = Issue.rate() / ins / 1e9 if ins else None
    bound = "issue" if issue is not None and issue < hbm else "hbm"
    lim = issue if bound == "issue" else hbm
    return {"hbm_ceiling": hbm, "issue_ceiling": issue, "thread_instr_per_voxel_iter": ins,
            "bound": bound, "frac_of_bound": value / lim}


GATE_SIGMA = 1e-3   # the 2-byte error gate, in units of sigma


def precision_boxes(cube):
    """Four 16 x 32 x 32 boxes (z, y, x ranges) where the 2-byte results are
    compared with the FP64 oracle: a corner (three cube faces), the box
    around the brightest voxel (a disk centre), and two seeded random
    positions (mostly noise and faint emission)."""
    import numpy as np
    nz, ny, nx = cube.shape
    bz, by, bx = 16, 32, 32
    zc, yc, xc = np.unravel_index(int(np.argmax(cube)), cube.shape)
    clamp = lambda c, n, w: int(min(max(c - w // 2, 0), n - w))
    boxes = [((0, bz), (0, by), (0, bx))]
    z0, y0, x0 = clamp(zc, nz, bz), clamp(yc, ny, by), clamp(xc, nx, bx)
    boxes.append(((z0, z0 + bz), (y0, y0 + by), (x0, x0 + bx)))
    rng = np.random.default_rng(11)
    for _ in range(2):
        z0 = int(rng.integers(0, nz - bz + 1))
        y0 = int(rng.integers(0, ny - by + 1))
        x0 = int(rng.integers(0, nx - bx + 1))
        boxes.append(((z0, z0 + bz), (y0, y0 + by), (x0, x0 + bx)))
    return boxes


def err_norms(got, ref, sig):
    """max, rms, faint-band (|ref| < 3 sigma) max and rms of |got - ref|,
    in units of sigma."""
    import numpy as np
    err = np.abs(got.astype(np.float64) - ref)
    faint = np.abs(ref) < 3.0 * sig
    return {"max": float(err.max()) / sig, "rms": float(np.sqrt(np.mean(err ** 2))) / sig,
            "faint_max": float(err[faint].max()) / sig if faint.any() else 0.0,
            "faint_rms": float(np.sqrt(np.mean(err[faint] ** 2))) / sig if faint.any() else 0.0}


def line_precision(afd, ctx, cube, d_in, ref32, sig):
    """2-byte storage (per-cube power-of-two scale: the one nearest the noise
    rms for f16 and bf16, the finest that holds the cube's range for int16)
    x temporal depth on the benchmark cube.  Errors are measured against the FP64 oracle on four
    sampled boxes (computed through the domain of dependence: exact), and,
    for context, against the float32 GPU result over the whole cube; in
    units of sigma.  gate: RMS and faint-band max within 1e-3 sigma."""
    import numpy as np
    import torch
    import oracle
    n_vox = cube.size
    K = K_SIGMA * sig
    Kf = float(np.float32(K))
    scale = pow2_near(sig)
    scales = {"f16": scale, "bf16": scale, "i16": i16_scale(float(np.abs(cube).max()))}
    boxes = precision_boxes(cube)
    t0 = time.perf_counter()
    orc = [oracle.pm_filter_box(cube, bx, Kf, DT, N_ITER, COND) for bx in boxes]
    oracle_s = time.perf_counter() - t0
    sl = [tuple(slice(a, b) for a, b in bx) for bx in boxes]
    orc_cat = np.concatenate([o.ravel() for o in orc])

    def vs_oracle(full):
        return err_norms(np.concatenate([full[q].ravel() for q in sl]), orc_cat, sig)

    dt = {"f16": torch.float16, "bf16": torch.bfloat16, "i16": torch.int16}
    ref = ref32.cpu().numpy()
    faint = np.abs(ref) < 3.0 * sig
    peak = measured_peaks()[0]
    # float32 through the same entry point, timed on this run
    o32 = torch.empty_like(d_in)
    run32 = lambda: afd.afd_filter_ex(ctx, d_in, o32, "f32", 1.0, K, DT, N_ITER, COND, None, 1)
    run32()
    ms32 = _events_ms(run32, 5)
    v32 = n_vox * N_ITER / (ms32 / 1e3) / 1e9
    afd.afd_sync(ctx)
    e32 = vs_oracle(o32.cpu().numpy())
    rows = [{"storage": "f32", "t_block": 1, "ms": ms32, "value": v32, "speedup_vs_f32": 1.0,
             "bytes_per_voxel_iter": 8.0, **ceilings("f32", 1, v32, peak),
             "err_vs_oracle": e32,
             "gate_pass": e32["rms"] <= GATE_SIGMA and e32["faint_max"] <= GATE_SIGMA}]
    for st in ("f16", "bf16", "i16"):
        q = torch.empty(cube.shape, dtype=dt[st], device=d_in.device)
        o = torch.empty_like(q)
        back = torch.empty_like(d_in)
        afd.afd_quantize(ctx, d_in, q, st, scales[st])
        for T in (1, 2, 4, 8):
            run = lambda: afd.afd_filter_ex(ctx, q, o, st, scales[st], K, DT, N_ITER, COND, None,
                                            T)
            run()
            ms = _events_ms(run, 5)
            afd.afd_dequantize(ctx, o, back, st, scales[st])
            afd.afd_sync(ctx)
            got = back.cpu().numpy()
            err = np.abs(got - ref)
            value = n_vox * N_ITER / (ms / 1e3) / 1e9
            eo = vs_oracle(got)
            rows.append({"storage": st, "scale": scales[st], "t_block": T, "ms": ms,
                         "value": value,
                         "speedup_vs_f32": value / v32,
                         "bytes_per_voxel_iter": pass_bytes(st, T),
                         **ceilings(st, T, value, peak),
                         "err_vs_oracle": eo,
                         "gate_pass": eo["rms"] <= GATE_SIGMA and eo["faint_max"] <= GATE_SIGMA,
                         "err_vs_f32": {"max": float(err.max()) / sig,
                                        "rms": float(np.sqrt(np.mean(err ** 2))) / sig,
                                        "faint_max": float(err[faint].max()) / sig}})
        del q, o, back
    best = max(rows[1:], key=lambda r: r["value"])
    passing = [r for r in rows[1:] if r["gate_pass"]]
    best_pass = max(passing, key=lambda r: r["value"]) if passing else None
    return {"unit": UNIT, "scale": scales, "workload": "the headline cube, K = 1.0 sigma, "
            "dt = 1/8, 50 rational iterations, stored in 2 bytes with a power-of-two scale (f16, "
            "bf16: the one nearest the noise rms; i16: the finest whose range, 32 x scale, holds "
            "the cube's largest |I|); "
            "t_block iterations between roundings to the storage format (afd_filter_ex; "
            "depths 2, 4 and 8 as chains of one-iteration launches with float32 intermediate "
            "cubes); err_vs_oracle: against the FP64 oracle on the float32 input over four 16x32x32 boxes %s (oracle through the "
            "domain of dependence, exact; %.1f s of oracle), in units of sigma (faint: |I| < 3 "
            "sigma); gate_pass: rms and faint max both <= 1e-3 sigma; err_vs_f32: against the "
            "float32 GPU result over the whole cube; per row the HBM ceiling (measured copy "
            "GB/s over the pass's bytes per voxel-iteration: 2 b at depth 1, (2 b + 8 (T - 1)) "
            "/ T for the chains) and the issue ceiling (SMs x 4 x 32 lanes x sampled SM "
            "clock over the ncu thread-instructions per voxel-iteration), and which binds"
            % (boxes, oracle_s),
            "issue_rate": {"sm_count": Issue.sm_count, "sm_mhz": Issue.sm_mhz},
            "best": {"storage": best["storage"], "t_block": best["t_block"],
                     "value": best["value"], "speedup_vs_f32": best["speedup_vs_f32"]},
            "best_gate_pass": None if best_pass is None else {
                "storage": best_pass["storage"], "t_block": best_pass["t_block"],
                "value": best_pass["value"], "speedup_vs_f32": best_pass["speedup_vs_f32"]},
            "rows": rows}


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

    def host_ms(fn, reps=5):
        fn()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        return (time.perf_counter() - t0) / reps * 1e3

    def e2e_sync():   # copy in, filter, copy out, one after the other
        d_in.copy_(h_in, non_blocking=True)
        afd.afd_filter_intensity(ctx, d_in, d_out, 1.5, rms, 0.0325, 20, C)
        h_out.copy_(d_out, non_blocking=True)
        torch.cuda.current_stream().synchronize()

    sync_ms = host_ms(e2e_sync)
    # one call, host cube in and out: z-slabs with 20 ghost planes (one
    # round), the copies of one slab overlapping the passes of another
    slab_ms = {}
    for slab_nz in (128, 180, 268):
        slab_ms[slab_nz] = host_ms(lambda: afd.afd_filter_intensity_slabs(
            ctx, h_in, h_out, 1.5, rms, 0.0325, 20, C, slab_nz, 20))
    best_slab = min(slab_ms, key=slab_ms.get)
    e_ms = slab_ms[best_slab]
    return {"unit": UNIT, "workload": "intensity-driven form, K = 1.5 (units of the GPU noise "
            "rms), tau = 0.0325, n = 20, C = 5 (the paper's defaults), on a 512x512x536 "
            "synthetic cube (1.41e8 voxels, the size of the paper's benchmark cube)",
            "value": n_vox * 20 / (ms / 1e3) / 1e9, "ms": ms,
            "e2e_value": n_vox * 20 / (e_ms / 1e3) / 1e9, "e2e_ms": e_ms,
            "e2e_path": "afd_filter_intensity_slabs, pinned host cube in and out in one "
                        "synchronous call: %d-plane z-slabs with 20 ghost planes (best of "
                        "128/180/268)" % best_slab,
            "e2e_slab_ms": {str(k): v for k, v in slab_ms.items()},
            "e2e_sync_value": n_vox * 20 / (sync_ms / 1e3) / 1e9, "e2e_sync_ms": sync_ms,
            "e2e_sync_path": "copy in, afd_filter_intensity, copy out, in series",
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
    estimate), 20 iterations, one CUDA-graph launch per call; tile kind and
    z-chunk picked by the autotuner."""
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
        tiles, zc = tuner.tune_batch(afd, b, K, DT, 20, COND)
        run = lambda: afd.afd_batch_filter(b, K, DT, 20, COND)
        run()
        ms = _events_ms(run, 10)
        out[st] = {"ms_per_call": ms, "value": nvox * 20 / (ms / 1e3) / 1e9, "tiles": tiles,
                   "zchunk": zc,
                   "tuning_ms": tuner.cache[tune.batch_key(shapes, st, COND, 20)]["ms"]}
        b.close()
        torch.cuda.synchronize()
    return out


def line_serving(afd, ctx, max_requests, max_seconds, saturation_requests):
    """64 resident float16 cubes (21 x 128^3, 21 x 256^3, 22 x 512x512x128).
    Open loop: Poisson arrivals at each rate, each request a re-filter with
    K ~ U[0.5, 3] sigma and 1-50 iterations, admitted by free HBM; p50/p99
    latency from the scheduled arrival to completion, until max_requests
    have arrived or max_seconds have passed.  The slowest 1 % are split
    into host lag, waiting for memory, waiting for a round and running.
    Closed loop (saturation): as many requests outstanding as the service
    has slots, a new one submitted as each completes."""
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
    budget, slots = 16 << 30, 128
    srv = afd.afd_serve_create(b, budget, slots)
    rng = np.random.default_rng(0)
    vox = [float(a) * bb * cc for a, bb, cc in shapes]
    res = {"unit": "ms", "workload": "64 resident float16 cubes (21 x 128^3, 21 x 256^3, "
           "22 x 512x512x128, seed 0); each request a random cube, K ~ U[0.5, 3] sigma_cube, "
           "n ~ U{1..50}, rational g, dt = 1/8; HBM budget 16 GiB for results + scratch, %d "
           "slots; open loop: Poisson arrivals until %d requests or %.0f s per rate, latency "
           "from the scheduled arrival to the completion of the request's last round; "
           "closed loop: %d requests with every slot kept busy" % (slots, max_requests,
                                                                 max_seconds,
                                                                 saturation_requests),
           "rates": []}

    def draw():
        return (int(rng.integers(0, len(shapes))), float(rng.uniform(0.5, 3.0)),
                int(rng.integers(1, 51)))

    for lam in (50, 100, 200, 500):
        n_req = int(min(max_requests, lam * max_seconds))
        arrivals = np.cumsum(rng.exponential(1.0 / lam, size=n_req))
        reqs = [draw() for _ in range(n_req)]
        rec, work, live, k = [], 0.0, {}, 0
        t0 = time.perf_counter()
        while k < n_req or live:
            now = time.perf_counter() - t0
            while k < n_req and arrivals[k] <= now:
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
                    ts = afd.afd_serve_times(srv, tk)
                    rec.append((l + lag, lag, ts[1] - ts[0], ts[2] - ts[1], ts[3] - ts[2], c, n))
                    work += vox[c] * n
                    afd.afd_serve_release(srv, tk)
            if not live and k < n_req:
                time.sleep(max(0.0, min(0.001, arrivals[k] - (time.perf_counter() - t0))))
        el = time.perf_counter() - t0
        lat = np.array([r[0] for r in rec]) * 1e3
        p99 = float(np.percentile(lat, 99))
        tail = [r for r in rec if r[0] * 1e3 >= p99]
        med = lambda j: float(np.median([r[j] for r in tail])) * 1e3
        res["rates"].append({
            "lambda_per_s": lam, "requests": int(len(lat)), "seconds": el,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": p99,
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
            "throughput_req_per_s": len(lat) / el,
            "throughput_gvox_iter_per_s": work / el / 1e9,
            "slowest_1pct": {"count": len(tail), "median_host_lag_ms": med(1),
                             "median_wait_memory_ms": med(2), "median_wait_round_ms": med(3),
                             "median_run_ms": med(4),
                             "median_iterations": float(np.median([r[6] for r in tail])),
                             "share_512x512x128": sum(1 for r in tail if vox[r[5]] > 2 ** 25)
                             / max(1, len(tail))}})
    # closed loop: keep every slot busy
    live, done, work = set(), 0, 0.0
    n_sub = 0
    t0 = time.perf_counter()
    while done < saturation_requests:
        while len(live) < slots and n_sub < saturation_requests:
            c, ks, n = draw()
            live.add((afd.afd_serve_submit(srv, c, ks * sig[c], DT, n, COND), c, n))
            n_sub += 1
        afd.afd_serve_step(srv, wait=True)
        for item in list(live):
            if afd.afd_serve_poll(srv, item[0])[0] == 2:
                live.discard(item)
                afd.afd_serve_release(srv, item[0])
                done += 1
                work += vox[item[1]] * item[2]
    el = time.perf_counter() - t0
    res["saturation"] = {"requests": done, "seconds": el, "req_per_s": done / el,
                         "saturation_gvox_iter_per_s": work / el / 1e9}
    srv.close()
    b.close()
    torch.cuda.synchronize()
    return res


def cpu_openmp_baseline(cube, K):
    """The multithreaded FP32 CPU build (cpu_omp, OpenMP) on the full
    benchmark cube on every host core the process may use: median of 5 runs
    after 1 warm-up; host STREAM-copy bandwidth as its roofline."""
    import numpy as np
    import cpu_omp
    cpu_omp.build()
    cores = cpu_cores()
    work = np.empty_like(cube)
    secs = []
    for r in range(6):
        np.copyto(work, cube)
        t0 = time.perf_counter()
        cpu_omp.filter_inplace(work, K, DT, N_ITER, COND, threads=cores)
        el = time.perf_counter() - t0
        if r > 0:
            secs.append(el)
    sec = statistics.median(secs)
    value = cube.size * N_ITER / sec / 1e9
    host_gbs = cpu_omp.stream_copy_gbs(1 << 30, 5, cores)
    achieved = 8.0 * cube.size * N_ITER / sec / 1e9
    return {"value": value, "unit": UNIT, "cores": cores, "threads": cores,
            "kind": "openmp_f32", "cpu_model": cpu_omp.cpu_model(),
            "sample": "the full 512x512x256 cube, 50 rational iterations, float32, per-face "
                      "conductance, OpenMP over z slabs (cpu_omp/afd_omp.c, gcc -O3 -fopenmp, "
                      "no target-specific flags); median of 5 runs after 1 warm-up",
            "s_per_run": sec, "samples_s": secs,
            "roofline": {"bound": "host memory", "achieved": achieved, "peak": host_gbs,
                         "unit": "GB/s", "frac": achieved / host_gbs if host_gbs > 0 else None,
                         "peak_kind": "measured STREAM copy (read + write) on the same host "
                                      "cores, 1 GiB per buffer, best of 5",
                         "bytes_per_voxel_iter": 8.0}}


def summary(line):
    """The line's key figures in a few hundred characters (rounded)."""
    r3 = lambda v: None if v is None else float("%.3g" % v)
    out = {"value": r3(line["value"]), "roofline_frac": r3(line["roofline"]["frac"]),
           "e2e": r3(line["e2e"]["value"])}
    if line.get("cpu_openmp"):
        c = line["cpu_openmp"]
        out["cpu_openmp"] = {"value": r3(c["value"]), "cores": c["cores"],
                             "host_frac": r3(c["roofline"]["frac"])}
    if line.get("cpu_baseline"):
        out["cpu_oracle"] = r3(line["cpu_baseline"]["value"])
    L = line.get("lines", {})
    if "precision" in L:
        out["precision"] = [[r["storage"], r["t_block"], r3(r["value"]),
                             r3(r["speedup_vs_f32"]), r3(r["err_vs_oracle"]["rms"]),
                             r3(r["err_vs_oracle"]["faint_max"]), r["gate_pass"]]
                            for r in L["precision"]["rows"]]
        out["precision_cols"] = "storage,T,Gvox-it/s,x f32,rms/sig,faint max/sig,gate"
        bp = L["precision"].get("best_gate_pass")
        out["precision_best_gate_pass"] = None if bp is None else [
            bp["storage"], bp["t_block"], r3(bp["value"]), r3(bp["speedup_vs_f32"])]
    if "batch" in L:
        out["batch"] = {k: r3(L["batch"][k]["value"]) for k in ("f32", "f16") if k in L["batch"]}
    if "serving" in L:
        sv = L["serving"]
        out["serving"] = [[r["lambda_per_s"], r["requests"], r3(r["p50_ms"]), r3(r["p99_ms"])]
                          for r in sv["rates"]]
        out["serving_cols"] = "lambda,requests,p50 ms,p99 ms"
        if "saturation" in sv:
            out["saturation_gvox_iter_per_s"] = r3(sv["saturation"]["saturation_gvox_iter_per_s"])
    return out


def split_slabs_run(cube, world, rank, n_iter, halo, step, steps, to_device, sync):
    """One cube over `world` ranks (rank `rank` here): this rank's z-slab of
    the numpy cube, moved by to_device, filtered `steps` times by
    slabs.filter_slab (ghost-plane exchange with the neighbour ranks each
    round of `halo` iterations, `step` doing the arithmetic); sync() before
    and after the timed loop.  Returns (z0, z1, the slab's last result,
    seconds for the `steps` calls)."""
    from paper_1609_03782_gb300 import slabs
    nz = cube.shape[0]
    z0, z1 = slabs.slab_bounds(nz, world, rank)
    own = to_device(cube[z0:z1])
    res = None
    sync()
    t0 = time.perf_counter()
    for _ in range(steps):
        res = slabs.filter_slab(own, z0, z1, nz, n_iter, halo, step)
    sync()
    return z0, z1, res, time.perf_counter() - t0


def run_slabs(args):
    """--split slabs: the headline cube split into z-slabs over the ranks
    (strong scaling): every round of `halo` iterations each rank swaps `halo`
    edge planes with its neighbours (NCCL point-to-point into its own
    buffer, no remote loads) and filters its slab with its ghost planes."""
    import numpy as np
    import torch
    import torch.distributed as dist
    import synth
    from paper_1609_03782_gb300 import afd, ranks, slabs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    cube = synth.cube512()
    ctx = afd.afd_create(local)
    whole = torch.from_numpy(cube).to(dev)
    sig = afd.afd_noise_rms(ctx, whole)
    K = K_SIGMA * sig
    step = slabs.gpu_step(ctx, K, DT, COND)
    to_dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    def sync():
        torch.cuda.synchronize(dev)
        ranks.barrier()

    split_slabs_run(cube, world, rank, N_ITER, args.slab_halo, step, max(args.warmup, 1),
                    to_dev, sync)
    z0, z1, res, sec = split_slabs_run(cube, world, rank, N_ITER, args.slab_halo, step,
                                       args.steps, to_dev, sync)
    sec = ranks.max_over_ranks(sec, dev)
    # the slab result against the library's whole-cube filter, bit for bit
    ref = torch.empty_like(whole)
    afd.afd_filter_out(ctx, whole, ref, K, DT, N_ITER, COND)
    afd.afd_sync(ctx)
    mism = float(0.0 if torch.equal(res, ref[z0:z1]) else 1.0)
    mism = ranks.max_over_ranks(mism, dev)
    value = cube.size * N_ITER * args.steps / sec / 1e9
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": sec / args.steps * 1e3, "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD + " (K fixed before the timed region)",
                           "parallelism": "z-slabs over %d ranks, %d ghost planes per round"
                                          % (world, args.slab_halo),
                           "step": "slabs.filter_slab: per round of %d iterations a ghost-"
                                   "plane exchange (NCCL send/recv into each rank's own "
                                   "buffer) and afd_filter on the slab" % args.slab_halo},
                "bit_exact_vs_whole_cube": mism == 0.0}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


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
    Issue.sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    if clk and clk.get("sm_mhz"):
        Issue.sm_mhz = float(clk["sm_mhz"])
    else:
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
                Issue.sm_mhz = float(json.load(fh)["sm_max_mhz"])
        except (OSError, KeyError, ValueError):
            pass
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
    # passes.  Five rounds, the median reported (all listed): the overlap
    # depends on the host keeping ahead of the GPU, and a shared host can
    # delay a round or two.
    for _ in range(2):
        afd.afd_filter_host_async(ctx, h_in, h_out, K_host, DT, N_ITER, COND)
    afd.afd_sync(ctx)
    e2e_rounds = []
    for _ in range(5):
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
            lines["serving"] = line_serving(afd, ctx, args.serve_requests,
                                            args.serve_max_seconds, args.saturation_requests)

    line = None
    if rank == 0:
        cpu_mt = None
        if world == 1 and not args.no_cpu_openmp:
            cpu_mt = cpu_openmp_baseline(cube, K_SIGMA * sig)
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
            "cpu_openmp": cpu_mt,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * n_vox,
                    "d2h_bytes_per_step": 4 * n_vox,
                    "path": "afd_filter_host_async, one call per step (a stream of cubes): "
                            "pinned host in -> device -> 50 iterations -> pinned host out; "
                            "a call's copies overlap the previous call's passes; afd_sync "
                            "after the last step; median of 5 rounds",
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
        # last, so that a reader that keeps only the end of the line keeps it
        line["summary"] = summary(line)
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.split == "slabs":
        return run_slabs(args)
    return run_afd(args)


if __name__ == "__main__":
    sys.exit(main())
