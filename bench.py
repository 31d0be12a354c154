#!/usr/bin/env python
"""Benchmark of the semi-implicit Fourier-spectral phase-field step on GB300.

Workload (default): 2D periodic 1024 x 1024 grid, c plus two order parameters
(p = 2), FP32 fields and transforms, seeded uniform noise +-0.01 about
c = eta = 0.5, dt = 6 x the explicit-FD stable dt, the paper's parameters.
One timed "step" is one time step of Algorithm 1 (row pass + column pass)
through the C ABI, with the L2 cache flushed (a 512 MB buffer written)
before every timed step.  The FP64 step of the same workload is timed the same
way and reported beside it.

Output: one JSON line on rank 0 (see the keys at the end of main()).
  --impl reference times the CPU oracle (the plain FP64 C++ solver) on the
  host cores on a bounded sample of the same workload.
Multi-GPU (torchrun): every rank runs an independent replica (the step has no
exchange between simulations); value = all ranks' grid-point-steps / the
slowest rank's time.
  --slab instead decomposes ONE grid (--slab-n^2, c + 2 eta, FP32) over the
  ranks (include/fs_slab.h; NCCL point-to-point transposes): strong scaling,
  value = the grid's points x steps / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "FS grid-point-steps/s & % HBM roofline, FP32/batched vs plain FP64, 1 GB300"
UNIT = "grid-point-steps/s"
GRID = (1024, 1024)
P = 2
WORKLOAD = "2D periodic 1024x1024, c + 2 eta, FP32, dt = 6 x FD-stable dt, seeded +-0.01 noise"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-extras", action="store_true", help="skip the 3D and ensemble measurements")
    ap.add_argument("--slab", action="store_true", help="one grid decomposed over the ranks (strong scaling)")
    ap.add_argument("--slab-n", type=int, default=1024, help="grid side of --slab")
    return ap.parse_args()


def problem():
    from paper_2306_04322_gb300 import inputs as I
    pr = I.Problem(n=GRID, p=P)
    pr.dt = 6.0 * I.fd_stable_dt(pr)
    return pr


def dist_info():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dram_traffic(kernel: str, precision: str, table: str = "traffic_2d_1024_p2.txt"):
    """DRAM bytes per launch from a committed ncu summary, or None."""
    path = os.path.join(ROOT, "profiles", table)
    try:
        for line in open(path):
            parts = line.split()
            if len(parts) >= 4 and parts[0] == "traffic" and parts[1] == kernel and parts[2] == precision:
                return float(parts[3])
    except OSError:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    count = 0

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        ClockSampler.count += 1
        # the samples go to a temporary file of this sampler, or to FS_CLOCKS_CSV
        # (suffixed by the sampler's number) when set
        env = os.environ.get("FS_CLOCKS_CSV")
        self.keep = bool(env)
        self.path = (f"{env}.{ClockSampler.count}" if env else
                     os.path.join(tempfile.gettempdir(), f"fs_clocks_{os.getpid()}_{index}_{ClockSampler.count}.csv"))

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path) or ".", exist_ok=True)
            self.fh = open(self.path, "w")
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not self.keep:
            try:
                os.remove(self.path)  # the temporary sample file
            except OSError:
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def time_gpu(precision: str, steps: int, warmup: int, device: int):
    """Device time of `steps` single time steps, L2 flushed before each."""
    import torch
    from paper_2306_04322_gb300 import fs, inputs as I
    pr = problem()
    dtype = torch.float64 if precision == "f64" else torch.float32
    f0 = torch.tensor(I.noise_fields(pr, seed=0), dtype=dtype, device=f"cuda:{device}")
    plan = fs.Plan(pr, precision)
    plan.set_fields(f0)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{device}")
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        flush.zero_()
        fs.fs_step_async(plan.h, 1)
    torch.cuda.synchronize()
    # timed: the call a user makes (kernels may overlap at pass boundaries)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        evs[i][0].record(stream)
        fs.fs_step_async(plan.h, 1)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    per = sorted(a.elapsed_time(b) for a, b in evs)
    total_ms = sum(per)
    launches = fs.fs_last_launch_count(plan.h) * steps
    # steady state of a long run: fs_step_async(plan, 32) replays the captured
    # 32-step graph (the state stays in L2 from step to step, as in a long
    # run); the L2 is flushed before every 32-step call
    calls = max(2, steps // 32)
    flush.zero_()
    fs.fs_step_async(plan.h, 32)  # builds and warms the graph
    torch.cuda.synchronize()
    gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(calls)]
    for i in range(calls):
        flush.zero_()
        gev[i][0].record(stream)
        fs.fs_step_async(plan.h, 32)
        gev[i][1].record(stream)
    torch.cuda.synchronize()
    graph_ms = sum(a.elapsed_time(b) for a, b in gev) / (32 * calls)
    # per-pass breakdown: the same steps with an event pair around every pass
    fs.fs_profile_read(plan.h)
    for i in range(steps):
        flush.zero_()
        fs.fs_step_profiled(plan.h, 1)
    torch.cuda.synchronize()
    kern_ms, kern_cnt = fs.fs_profile_read(plan.h)
    ws = plan.workspace_bytes
    plan.close()
    return {"total_ms": total_ms, "kern_ms": kern_ms, "kern_cnt": kern_cnt, "launches": launches,
            "workspace_bytes": ws, "npts": pr.npoints, "median_ms": per[len(per) // 2], "best_ms": per[0],
            "graph_ms_per_step": graph_ms, "graph_steps": 32 * calls}


def time_cufft_structure(steps: int, warmup: int, device: int):
    """The paper's step structure on the same GPU, as a comparison point only:
    pointwise derivatives as PyTorch elementwise kernels, R2C transforms of c,
    df/dc, eta_i and df/deta_i with cuFFT (torch.fft), the per-mode update,
    C2R transforms.  Same workload, FP32, L2 flushed before every step."""
    import math
    import torch
    from paper_2306_04322_gb300 import inputs as I
    pr = problem()
    dev = f"cuda:{device}"
    u = torch.tensor(I.noise_fields(pr, seed=0), dtype=torch.float32, device=dev)
    ny, nx = pr.shape
    kx = 2 * math.pi * torch.fft.rfftfreq(nx, d=pr.dx[0], device=dev, dtype=torch.float32)
    ky = 2 * math.pi * torch.fft.fftfreq(ny, d=pr.dx[1], device=dev, dtype=torch.float32)
    k2 = ky[:, None] ** 2 + kx[None, :] ** 2
    dc = 1.0 / (1.0 + pr.M * pr.dt * pr.kappa_c * k2 * k2)
    de = 1.0 / (1.0 + pr.L * pr.dt * pr.kappa_eta * k2)
    dcab, cab = pr.c_beta - pr.c_alpha, pr.c_beta + pr.c_alpha

    def step(u):
        c, e = u[0], u[1:]
        h = (e ** 3 * (6 * e * e - 15 * e + 10)).sum(0)
        s2 = (e * e).sum(0)
        fc = 2 * pr.rho2 * (c - pr.c_alpha - dcab * h)
        q = e * (1 - e)
        fe = (pr.rho2 * dcab * (cab - 2 * c) * 30 * q * q
              + pr.w * (2 * q * (1 - 2 * e) + 4 * pr.alpha * e * (s2 - e * e)))
        F = torch.fft.rfft2(torch.cat([u, fc[None], fe]))
        p = pr.p
        chat = (F[0] - pr.M * pr.dt * k2 * F[1 + p]) * dc
        ehat = (F[1:1 + p] - pr.L * pr.dt * F[2 + p:]) * de
        return torch.fft.irfft2(torch.cat([chat[None], ehat]), s=(ny, nx))

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        flush.zero_()
        u = step(u)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        evs[i][0].record(stream)
        u = step(u)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs) / steps
    ok = bool(torch.isfinite(u).all())
    # The same step captured once in a CUDA graph and replayed: the library
    # kernels' own time without the Python dispatch of ~30 eager operations.
    # The state is copied back into the graph's input outside the timed window.
    static_u = u.clone()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        for _ in range(3):
            step(static_u)
    stream.wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        static_out = step(static_u)
    torch.cuda.synchronize()
    for _ in range(warmup):
        flush.zero_()
        g.replay()
        static_u.copy_(static_out)
    torch.cuda.synchronize()
    gevs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        gevs[i][0].record(stream)
        g.replay()
        gevs[i][1].record(stream)
        static_u.copy_(static_out)
    torch.cuda.synchronize()
    gms = sum(a.elapsed_time(b) for a, b in gevs) / steps
    ok = ok and bool(torch.isfinite(static_u).all())
    del g
    return {"value": pr.npoints / (gms / 1e3), "unit": UNIT, "ms_per_step": gms, "finite": ok,
            "eager": {"value": pr.npoints / (ms / 1e3), "unit": UNIT, "ms_per_step": ms},
            "what": "paper's step structure with cuFFT R2C/C2R (torch.fft) and PyTorch elementwise kernels, "
                    "FP32, same workload, L2 flushed before every step; the value is one CUDA-graph replay "
                    "of the whole step (library kernels only), 'eager' the same step launched op by op; "
                    "comparison only"}


def time_plan(probs, precision: str, steps: int, warmup: int, device: int, flush_mb: int = 512, chunk: int = 1):
    """Device time of `steps` steps of a plan (a list of problems = ensemble),
    in calls of fs_step_async(plan, chunk) (chunk >= 32: the captured graph of
    the time loop), L2 flushed before every timed call; per-pass times from
    the plan's profiled steps."""
    import torch
    from paper_2306_04322_gb300 import fs, inputs as I
    dtype = torch.float64 if precision == "f64" else torch.float32
    batch = isinstance(probs, list)
    plist = probs if batch else [probs]
    fields = [torch.tensor(I.noise_fields(p, seed=i), dtype=dtype, device=f"cuda:{device}")
              for i, p in enumerate(plist)]
    plan = fs.Plan(plist if batch else plist[0], precision)
    plan.set_fields(fields if batch else fields[0])
    sched = fs.fs_batch_schedule(plan.h) if batch else None
    flush = torch.empty(flush_mb * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{device}")
    stream = torch.cuda.current_stream()
    calls = max(1, steps // chunk)
    for _ in range(warmup):
        flush.zero_()
        fs.fs_step_async(plan.h, chunk)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(calls)]
    for i in range(calls):
        flush.zero_()
        evs[i][0].record(stream)
        fs.fs_step_async(plan.h, chunk)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    total_ms = sum(a.elapsed_time(b) for a, b in evs)
    launches_timed = fs.fs_last_launch_count(plan.h) * calls
    steps = calls * chunk
    fs.fs_profile_read(plan.h)
    for i in range(steps):
        flush.zero_()
        fs.fs_step_profiled(plan.h, 1)
    torch.cuda.synchronize()
    kern_ms, kern_cnt = fs.fs_profile_read(plan.h)
    ws = plan.workspace_bytes
    plan.close()
    del fields, flush
    npts = sum(p.npoints for p in plist)
    return {"total_ms": total_ms, "kern_ms": kern_ms, "kern_cnt": kern_cnt, "launches": launches_timed,
            "workspace_bytes": ws, "npts": npts, "schedule": sched, "steps": steps}


def roofline_entry(names, alg_bytes, r, peak, peak_kind, traffic_table=None):
    avg_ms = [m / max(c, 1) for m, c in zip(r["kern_ms"], r["kern_cnt"])]
    dom = max(range(len(avg_ms)), key=lambda i: r["kern_ms"][i])
    achieved = alg_bytes[dom] / (avg_ms[dom] / 1e3) / 1e9
    traffic = dram_traffic(names[dom], "f32", traffic_table) if traffic_table else None
    return {"bound": "hbm", "kernel": names[dom], "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": peak_kind, "traffic": traffic,
            "alg_bytes_per_launch": alg_bytes[dom], "avg_launch_ms": avg_ms[dom],
            "kernels": {n: {"avg_ms": a, "launches": c, "share": m / max(sum(r["kern_ms"]), 1e-30),
                            "alg_GBps": b / (a / 1e3) / 1e9 if a > 0 else None}
                        for n, a, c, m, b in zip(names, avg_ms, r["kern_cnt"], r["kern_ms"], alg_bytes)}}


def step_entry(alg_bytes: int, comp_bytes: int, ms: float, peak: float, design_bytes=None) -> dict:
    """A whole step against its algorithmic bytes (3 s N per field and pass of
    the minimal pass structure), the compulsory lower bound (state read once
    and written once) and, when given, the bytes this design's passes move
    (fewer than the algorithmic count: c^ carried, one transform of
    eta - L dt df/deta)."""
    gb = lambda b: b / (ms / 1e3) / 1e9
    out = {"ms": ms, "algorithmic_bytes": alg_bytes, "compulsory_bytes": comp_bytes,
           "algorithmic_GBps": gb(alg_bytes), "compulsory_GBps": gb(comp_bytes),
           "frac_algorithmic": gb(alg_bytes) / peak, "frac_compulsory": gb(comp_bytes) / peak}
    if design_bytes:
        out.update({"design_bytes": design_bytes, "frac_design_bytes": gb(design_bytes) / peak})
    return out


def fp64_ops(kernel: str, table: str = "fp64_ops_2d_1024_p2.txt"):
    """FP64 thread-instructions (DADD + DMUL + DFMA) per launch of a kernel of
    the 1024^2 p = 2 FP64 step, counted by ncu (committed summary), or None."""
    path = os.path.join(ROOT, "profiles", table)
    try:
        for line in open(path):
            parts = line.split()
            if len(parts) >= 3 and parts[0] == "fp64_ops" and parts[1] == kernel:
                return float(parts[2])
    except OSError:
        pass
    return None


def fp64_roofline(r64, rate64, hbm_peak, npts: int, nf: int) -> dict:
    """The FP64 step against min(HBM, FP64 pipe): its floor time is the larger
    of bytes / HBM bandwidth and FP64 instructions / the measured FP64
    instruction rate (DADD, DMUL and DFMA each take one FP64 issue slot).
    Reported for the dominant pass and for the whole step."""
    names = ["fs_row_kernel", "fs_col_kernel"]
    dfma, dadd = rate64
    avg_ms = [m / max(c, 1) for m, c in zip(r64["kern_ms"], r64["kern_cnt"])]
    dom = max(range(len(avg_ms)), key=lambda i: r64["kern_ms"][i])
    ops = [fp64_ops(n) for n in names]
    alg = [3 * nf * npts * 8] * 2
    step_ms = r64["total_ms"] / max(r64["kern_cnt"][0], 1)
    out = {"bound": "alu", "kernel": names[dom], "unit": "FP64 Ginst/s", "peak": dfma / 1e9,
           "peak_source": "measured (project-written DFMA loop, CUDA events, this run)",
           "peak_dadd": dadd / 1e9, "peak_tflops": 2 * dfma / 1e12, "avg_launch_ms": avg_ms[dom],
           "hbm": {"achieved": alg[dom] / (avg_ms[dom] / 1e3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                   "frac": alg[dom] / (avg_ms[dom] / 1e3) / 1e9 / hbm_peak},
           "ops_source": "ncu smsp__sass_thread_inst_executed_op_{dadd,dmul,dfma}_pred_on.sum "
                         "(profiles/fp64_ops_2d_1024_p2.txt)"}
    if ops[dom] is not None:
        ach = ops[dom] / (avg_ms[dom] / 1e3) / 1e9
        out.update({"achieved": ach, "frac": ach / (dfma / 1e9), "ops_per_launch": ops[dom]})
    else:
        out.update({"achieved": None, "frac": None, "ops_per_launch": None})
    if all(o is not None for o in ops):
        t_alu = sum(ops) / dfma
        t_hbm = sum(alg) / (hbm_peak * 1e9)
        out["step"] = {"ms": step_ms, "floor_ms_alu": t_alu * 1e3, "floor_ms_hbm": t_hbm * 1e3,
                       "frac": max(t_alu, t_hbm) * 1e3 / step_ms}
    return out


def extras(steps: int, warmup: int, device: int, peak, peak_kind):
    """3D 256^3 (p = 2, FP32), 2D 2048^2 (p = 4, FP32) and the 512-member
    ensemble (FP32): throughput and per-pass rooflines, reported beside the
    headline."""
    from paper_2306_04322_gb300 import inputs as I
    out = {}
    pr = I.Problem(n=(256, 256, 256), p=P)
    pr.dt = 6.0 * I.fd_stable_dt(pr)
    k = max(3, min(steps, 20))
    r = time_plan(pr, "f32", k, min(warmup, 3), device)
    nf, s, N = 1 + P, 4, r["npts"]
    # the algorithmic bytes of the minimal 3D pass structure: 3 s N per field
    # and pass (12 s N per field and step over the x, y-forward, z and
    # y-inverse passes)
    alg = [3 * nf * N * s] * 4
    out["3d_256_p2_f32"] = {"value": N * k / (r["total_ms"] / 1e3), "unit": UNIT, "steps": k,
                            "ms_per_step": r["total_ms"] / k, "dt": pr.dt, "launches": r["launches"],
                            "workspace_bytes": r["workspace_bytes"],
                            "roofline": roofline_entry(["x_pass(fs_row_kernel)", "fs_ypass_kernel<-1>",
                                                        "fs_zstep_kernel", "fs_ypass_kernel<+1>"],
                                                       alg, r, peak, peak_kind, "traffic_3d_256_p2.txt")}
    out["3d_256_p2_f32"]["roofline"]["step"] = step_entry(sum(alg), 2 * nf * N * s, r["total_ms"] / k, peak,
                                                          design_bytes=25 * N * s)
    # the finest 2D grid of the paper's Table 1 with its five fields (p = 4)
    pr = I.Problem(n=(2048, 2048), p=4)
    pr.dt = 6.0 * I.fd_stable_dt(pr)
    k = max(3, min(steps, 20))
    r = time_plan(pr, "f32", k, min(warmup, 3), device)
    nf4, N = 1 + pr.p, r["npts"]
    out["2d_2048_p4_f32"] = {"value": N * k / (r["total_ms"] / 1e3), "unit": UNIT, "steps": k,
                             "ms_per_step": r["total_ms"] / k, "dt": pr.dt, "launches": r["launches"],
                             "workspace_bytes": r["workspace_bytes"],
                             "roofline": roofline_entry(["fs_row_kernel", "fs_col_kernel"],
                                                        [3 * nf4 * N * s] * 2, r, peak, peak_kind,
                                                        "traffic_2d_2048_p4.txt")}
    out["2d_2048_p4_f32"]["roofline"]["step"] = step_entry(6 * nf4 * N * s, 2 * nf4 * N * s,
                                                           r["total_ms"] / k, peak,
                                                           design_bytes=(4 * nf4 + 1) * N * s)
    # config 4: the ensemble advanced through its captured graph (32 steps per
    # graph launch, one persistent launch per pass), two graph calls timed
    probs = I.batch_problems(512, seed=0)
    r = time_plan(probs, "f32", 64, 1, device, chunk=32)
    kb = r["steps"]
    N = r["npts"]
    alg = [3 * nf * N * s] * 2
    out["batched_512_f32"] = {"value": N * kb / (r["total_ms"] / 1e3), "unit": UNIT, "steps": kb,
                              "ms_per_step": r["total_ms"] / kb, "members": 512, "points": N,
                              "launches": r["launches"], "path": "fs_step_async(plan, 32): CUDA-graph replay",
                              "schedule": {"row_grid": r["schedule"][0], "col_grid": r["schedule"][1],
                                           "row_items": r["schedule"][2], "col_items": r["schedule"][3],
                                           "row_form": r["schedule"][4], "col_form": r["schedule"][5],
                                           "forms": "1: half-length rows / column tiles, radix-16 lines; "
                                                    "2: warp-per-line rows (pair form) and columns, radix up "
                                                    "to 32, two-column tiles"},
                              "roofline": roofline_entry(["fs_row_batch_kernel", "fs_col_batch_kernel"],
                                                         alg, r, peak, peak_kind)}
    return out


def time_e2e(steps: int, warmup: int, device: int, depth: int = 2):
    """Through the C ABI with pinned host buffers: every step copies its
    fields in (fs_set_fields), takes one time step (fs_step_async) and copies
    the fields out (fs_get_fields, which synchronises).  Pipelined: `depth`
    plans on their own streams take steps in turn, so one step's copy in
    (host to device) and time step run while the previous step's copy out
    (device to host) does.  The serial form (one plan, one step after the
    other) is timed beside it.  Measured at 1024^2, p = 2: 129 us per step
    against 189 us serial (with the two copy directions fully overlapped it
    would be about 95 us: copy in plus step); a third plan adds nothing."""
    import torch
    from paper_2306_04322_gb300 import fs, inputs as I
    pr = problem()
    host_in = [torch.tensor(I.noise_fields(pr, seed=k), dtype=torch.float32).pin_memory() for k in range(depth)]
    host_out = [torch.empty_like(h).pin_memory() for h in host_in]
    ins = [[h[f] for f in range(pr.nf)] for h in host_in]
    outs = [[h[f] for f in range(pr.nf)] for h in host_out]
    streams = [torch.cuda.Stream(device=device) for _ in range(depth)]
    plans = [fs.Plan(pr, "f32", stream=st.cuda_stream) for st in streams]

    def issue(i):
        fs.fs_set_fields(plans[i].h, ins[i])
        fs.fs_step_async(plans[i].h, 1)

    def pipelined(n):
        for k in range(min(depth - 1, n)):
            issue(k)
        for k in range(n):
            if k + depth - 1 < n:
                issue((k + depth - 1) % depth)  # its previous step was read back at k - 1
            fs.fs_get_fields(plans[k % depth].h, outs[k % depth])

    def serial(n):
        for _ in range(n):
            issue(0)
            fs.fs_get_fields(plans[0].h, outs[0])

    pipelined(warmup)
    serial(warmup)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pipelined(steps)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    t0 = time.perf_counter()
    serial(steps)
    torch.cuda.synchronize()
    dt_serial = time.perf_counter() - t0
    for pl in plans:
        pl.close()
    nbytes = host_in[0].numel() * 4
    return {"seconds": dt, "seconds_serial": dt_serial, "npts": pr.npoints, "h2d": nbytes, "d2h": nbytes,
            "depth": depth}


def _oracle_rate(O, pr, f, seconds: float, min_steps: int = 2):
    """Whole oracle time steps until `seconds` have passed; (steps, seconds)."""
    t0 = time.perf_counter()
    n = 0
    while True:
        f, _ = O.step(pr, f, 1)
        n += 1
        if time.perf_counter() - t0 >= seconds and n >= min_steps:
            break
    return n, time.perf_counter() - t0


def cpu_model() -> str:
    """Host CPU model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def cpu_baseline(seconds: float):
    """The oracle (plain FP64 C++ solver) on the host cores, bounded samples of
    whole time steps: the 1024x1024 workload with OpenMP over all cores (the
    reported value) and single-threaded, and the 3D 256^3 configuration."""
    from oracle import oracle as O
    from paper_2306_04322_gb300 import inputs as I
    pr = problem()
    cores = os.cpu_count() or 1
    used = O.set_threads(cores)
    f = I.noise_fields(pr, seed=0)
    O.step(pr, f, 1)  # warm (page-in, tables)
    n, dt = _oracle_rate(O, pr, f, seconds)
    out = {"value": pr.npoints * n / dt, "unit": UNIT, "cores": used, "kind": "oracle",
           "sample": f"{n} whole FP64 oracle time steps of the 1024x1024 p=2 workload "
                     f"({dt:.1f} s, OpenMP over FFT lines, {used} threads)",
           "cpu": cpu_model(), "host_cores": cores}
    O.set_threads(1)
    n1, dt1 = _oracle_rate(O, pr, f, seconds / 3, min_steps=1)
    out["single_thread"] = {"value": pr.npoints * n1 / dt1, "unit": UNIT, "cores": 1,
                            "sample": f"{n1} whole steps, {dt1:.1f} s"}
    O.set_threads(cores)
    p3 = I.Problem(n=(256, 256, 256), p=P)
    p3.dt = 6.0 * I.fd_stable_dt(p3)
    f3 = I.noise_fields(p3, seed=0)
    n3, dt3 = _oracle_rate(O, p3, f3, seconds / 3, min_steps=1)
    out["3d_256"] = {"value": p3.npoints * n3 / dt3, "unit": UNIT, "cores": used,
                     "sample": f"{n3} whole FP64 steps of 256^3 p=2, {dt3:.1f} s"}
    return out


def reference_arm(args):
    world, rank, local = dist_info()
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2306_04322_gb300 import inputs as I
    pr = problem()
    cores = os.cpu_count() or 1
    used = O.set_threads(cores)
    f = I.noise_fields(pr, seed=0)
    for _ in range(args.warmup):
        f, _ = O.step(pr, f, 1)
    budget = 150.0
    t0 = time.perf_counter()
    done = 0
    for _ in range(args.steps):
        f, _ = O.step(pr, f, 1)
        done += 1
        if time.perf_counter() - t0 > budget:
            break
    dt = time.perf_counter() - t0
    per = dt / done
    total = per * args.steps
    value = pr.npoints * args.steps / total
    sample = (f"{done} of {args.steps} whole FP64 oracle time steps timed "
              f"({'all' if done == args.steps else 'time-bounded sample, per-step time extrapolated'}), "
              f"{used} threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD.replace("FP32", "FP64 (oracle)"), "grid": list(GRID), "p": P},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample,
                             "cpu": cpu_model(), "host_cores": cores},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def reduce_max(v: float, dist, device: str = "cpu") -> float:
    """Maximum of a per-rank float over the process group (identity without
    one); `device` is where the reduction tensor lives (CUDA for NCCL, CPU for
    gloo)."""
    if not dist:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, npts: int, steps: int, slowest_seconds: float) -> float:
    """Whole-job throughput of independent replicas: every rank advanced its
    own simulation of npts points by `steps` steps; the job took as long as
    the slowest rank."""
    return world * npts * steps / slowest_seconds


def slab_bench(args):
    """One grid decomposed over the ranks: every timed step is the row pass,
    the forward transpose (NCCL point-to-point), the column pass and the back
    transpose on every rank; L2 flushed (512 MB write) before every step,
    outside the timed events."""
    import socket
    import torch
    import torch.distributed as dist
    world, rank, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    else:
        with socket.socket() as so:
            so.bind(("127.0.0.1", 0))
            port = so.getsockname()[1]
        dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    from paper_2306_04322_gb300 import build as B
    from paper_2306_04322_gb300 import fs
    from paper_2306_04322_gb300 import inputs as I
    from paper_2306_04322_gb300 import slab as S
    B.build()
    fs.lib()
    pr = I.Problem(n=(args.slab_n, args.slab_n), p=P)
    pr.dt = 6.0 * I.fd_stable_dt(pr)
    d = S.DistributedSlab(pr, "f32")
    f0 = I.noise_fields(pr, seed=0)
    d.set_fields(torch.tensor(f0[:, d.layout.row_range()], dtype=torch.float32, device="cuda"))
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    d.step(args.warmup)
    torch.cuda.synchronize()
    dist.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(torch.cuda.current_device()) as clk:
        for e0, e1 in ev:
            flush.fill_(1.0)
            e0.record()
            d.step(1)
            e1.record()
        torch.cuda.synchronize()
    d.sync()
    dist.barrier()
    t = reduce_max(sum(e0.elapsed_time(e1) for e0, e1 in ev) / 1e3, dist, f"cuda:{local}")
    npts = pr.n[0] * pr.n[1]
    fwd, back = d.layout.exchange_bytes(8)
    d.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": npts * args.steps / t, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"2D periodic {pr.n[0]}x{pr.n[1]}, c + 2 eta, FP32, dt = 6 x FD-stable dt, "
                                   "seeded +-0.01 noise, one grid decomposed into slabs",
                       "grid": list(pr.n), "p": P, "parallelism": f"slab{world}",
                       "l2": "flushed (512 MB write) before every timed step"},
            "exchange": {"bytes_per_rank_per_step": fwd + back, "forward": fwd, "back": back},
            "gpu_launches": 4 * args.steps,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    dist.destroy_process_group()


def main():
    args = parse()
    world, rank, local = dist_info()
    if args.impl == "reference":
        reference_arm(args)
        return
    if args.slab:
        slab_bench(args)
        return
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    from paper_2306_04322_gb300 import build as B
    from paper_2306_04322_gb300 import fs
    B.build()
    fs.lib()

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    def max_over_ranks(v: float) -> float:
        return reduce_max(v, dist, f"cuda:{local}")

    barrier()
    with ClockSampler(torch.cuda.current_device()) as clk:
        r32 = time_gpu("f32", args.steps, args.warmup, local)
    barrier()
    with ClockSampler(torch.cuda.current_device()) as clk64:
        r64 = time_gpu("f64", args.steps, args.warmup, local)
        rate64 = fs.fs_measure_fp64_rate()
    barrier()
    e2e = time_e2e(args.steps, args.warmup, local)
    barrier()
    cufft = time_cufft_structure(args.steps, args.warmup, local)
    barrier()
    peak, peak_kind = load_peaks()
    ext = {} if args.no_extras else extras(args.steps, args.warmup, local, peak, peak_kind)
    barrier()

    t32 = max_over_ranks(r32["total_ms"]) / 1e3
    t64 = max_over_ranks(r64["total_ms"]) / 1e3
    te2e = max_over_ranks(e2e["seconds"])
    te2e_serial = max_over_ranks(e2e["seconds_serial"])
    npts = r32["npts"]
    value = job_value(world, npts, args.steps, t32)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    s = 4
    nf = 1 + P
    names = ["fs_row_kernel", "fs_col_kernel"]
    # algorithmic bytes per launch: the minimal 2D pass structure moves 3 s N
    # per field in each pass (row: read the half spectrum, write the packed
    # field and derivative spectra; column: read both, write the update)
    alg = [3 * nf * npts * s] * 2
    avg_ms = [m / max(c, 1) for m, c in zip(r32["kern_ms"], r32["kern_cnt"])]
    dom = max(range(len(avg_ms)), key=lambda i: r32["kern_ms"][i])
    achieved = alg[dom] / (avg_ms[dom] / 1e3) / 1e9
    roof = {"bound": "hbm", "kernel": names[dom], "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": peak_kind,
            "traffic": dram_traffic(names[dom], "f32"),
            "alg_bytes_per_launch": alg[dom], "avg_launch_ms": avg_ms[dom],
            "kernels": {n: {"avg_ms": a, "launches": c, "share": m / max(sum(r32["kern_ms"]), 1e-30)}
                        for n, a, c, m in zip(names, avg_ms, r32["kern_cnt"], r32["kern_ms"])}}
    # the whole step against the algorithmic bytes of the two passes, the
    # compulsory lower bound (state read once, written once) and the bytes
    # this design moves ((4 nf + 1) s N: c^ carried, one transform of g_i)
    roof["step"] = step_entry(sum(alg), 2 * nf * npts * s, t32 * 1e3 / args.steps, peak,
                              design_bytes=(4 * nf + 1) * npts * s)
    fp64 = {"value": job_value(world, npts, args.steps, t64), "unit": UNIT, "ms_per_step": t64 * 1e3 / args.steps,
            "kernels_ms": r64["kern_ms"], "launches": r64["launches"]}
    fp64["roofline"] = fp64_roofline(r64, rate64, peak, npts, nf)
    fp64["clocks"] = clk64.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t32 * 1e3 / args.steps,
        "ms_per_step_median": r32["median_ms"], "ms_per_step_best": r32["best_ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": list(GRID), "p": P, "dt": problem().dt,
                   "l2": "flushed (512 MB write) before every timed step",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "workspace_bytes": r32["workspace_bytes"]},
        "roofline": roof,
        "e2e": {"value": job_value(world, npts, args.steps, te2e), "unit": UNIT, "h2d_bytes_per_step": e2e["h2d"],
                "d2h_bytes_per_step": e2e["d2h"],
                "how": "every step: fs_set_fields from pinned host + fs_step_async(1) + fs_get_fields to pinned "
                       "host, wall clock; two plans on their own streams take alternate steps, so a step's copy "
                       "in and time step overlap the previous step's copy out",
                "serial": {"value": job_value(world, npts, args.steps, te2e_serial), "unit": UNIT,
                           "how": "the same calls on one plan, one step after the other"}},
        "gpu_launches": r32["launches"],
        "steady_state": {"value": job_value(world, npts, 1, r32["graph_ms_per_step"] / 1e3), "unit": UNIT,
                         "ms_per_step": r32["graph_ms_per_step"], "steps": r32["graph_steps"],
                         "how": "fs_step_async(plan, 32): one replay of the captured 32-step graph per call, "
                                "L2 flushed before each call only (the state stays L2-resident within a call, "
                                "as in a long run); the headline value flushes before every step"},
        "clocks": clk.summary(),
        "fp64": fp64,
        "cufft_structure": cufft,
    }
    line.update(ext)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
