"""Configuration-level studies on the GPU (each prints one JSON object).

    python -m paper_2306_04322_gb300.experiments precision   [--steps 2000]
    python -m paper_2306_04322_gb300.experiments accuracy    [--steps 10000]
    python -m paper_2306_04322_gb300.experiments cost        [--steps 200]
    python -m paper_2306_04322_gb300.experiments table1      [--t-span 1]
    python -m paper_2306_04322_gb300.experiments table2      [--t-span 0.5]
    python -m paper_2306_04322_gb300.experiments slab        [--steps 20]

precision and accuracy start from the benchmark initial condition of
Section 3 (Eqs. ic_c, ic_eta with p = 2, dx = 1), made periodic as the paper
does: the explicit FD scheme, run in FP64 on the GPU at half its stable dt,
takes it to t = 1 (table1 does the same on the paper's 200 x 200 domain).

precision: 3D 256^3, p = 2, dt = 5e-3: the t = 1 state of the 256^2 problem
    extruded along z (Eq. ic_eta_3d, c = c0); FP32, TF32 x 3 and BF16 x 3 runs
    against an FP64 GPU run of the same steps: relative L-inf of every field
    and the phase fraction (share of points with eta_i > 1/2).
accuracy: 2D 1024^2, p = 2 (FP64): the semi-implicit FS step at dt = 6 dt_FD
    (spectral |xi|^2 and the FS-FD O(dl^2) / O(dl^4) forms) and the explicit
    FD scheme (Section 2.2) at 0.95 dt_FD, all to the same end time, against
    a spectral FS reference at dt / 16; E_phi of Eq. (error_field) for c and
    for eta = sum_i eta_i, and the device time each run took.
cost: device time per step of the FS step and of the explicit FD scheme on
    the grid sizes of the paper's Tables 1 and 2 (2D 128^2 .. 2048^2,
    3D 16^3 .. 256^3), p = 4 as in the paper, FP64 and FP32; the
    ratio FS / FD is the paper's per-step cost comparison (Section 3).
table1: the paper's 2D accuracy study (Table 1 grids and time steps,
    domain 200, p = 4, E_phi against spectral FS FP64 on 2048^2 at
    dt = 1e-4) over t = 1 -> 1 + t_span; see table1_study.
table2: the paper's 3D cases (Table 2 grids 16^3 .. 256^3 on the 100^3
    domain, FS at dt = 5e-3, explicit FD at the paper's dt, p = 4, the 3D
    initial condition of Eq. ic_eta_3d) over t = 1 -> 1 + t_span: device
    time per unit of t and per step and point (the quantities of the
    paper's 3D performance figure), and E_phi against spectral FS FP64 on
    256^3 at a finer dt; see table2_study.
slab: the slab decomposition (include/fs_slab.h) of 2D 1024^2 and 2048^2,
    p = 2, FP32, over R = 1, 2, 4, 8 ranks held by one process: per-rank
    device time of the row pass (with its transposes) and of the column
    pass per step, against the single plan's step; see slab_study.
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def _run(fs, pr, f0, steps, precision, scheme=None):
    import torch
    dtype = torch.float64 if precision == "f64" else torch.float32
    plan = fs.Plan(pr, precision, scheme=fs.FS_SCHEME_SEMI_IMPLICIT_FS if scheme is None else scheme)
    plan.set_fields(torch.as_tensor(f0, dtype=dtype, device="cuda"))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    plan.step(steps)
    e1.record()
    out = plan.get_fields().double()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    plan.close()
    return out, ms


def ac_stable_dt(pr) -> float:
    """Forward-Euler bound of the Allen-Cahn equations linearised with
    eta_j <= 1: dt = 2 / (L (kappa_eta lambda + 2 w (1 + 2 alpha (p - 1)))),
    lambda = sum_d 4 / dx_d^2; below the Cahn-Hilliard bound of
    inputs.fd_stable_dt except on coarse grids (dx of a few units)."""
    lam = sum(4.0 / (d * d) for d in pr.dx)
    return 2.0 / (pr.L * (pr.kappa_eta * lam + 2.0 * pr.w * (1.0 + 2.0 * pr.alpha * max(pr.p - 1, 0))))


def periodic_benchmark_state(fs, pr2d, t_end: float = 1.0):
    """Benchmark initial condition (Section 3) advanced to t_end by the
    explicit FD scheme in FP64 at half its stable dt (the smaller of the
    Cahn-Hilliard and Allen-Cahn bounds); an (nf, ny, nx) float64 CUDA
    tensor."""
    import torch
    from . import inputs as I
    n = int(np.ceil(t_end / (0.5 * min(I.fd_stable_dt(pr2d), ac_stable_dt(pr2d)))))
    pre = pr2d.replace(dt=t_end / n)
    f0 = torch.tensor(I.benchmark_ic_fields(pr2d), dtype=torch.float64, device="cuda")
    out, _ = _run(fs, pre, f0, n, "f64", scheme=fs.FS_SCHEME_EXPLICIT_FD)
    return out


def precision_study(steps: int, n: int = 256):
    import torch
    from . import fs, inputs as I
    pr = I.Problem(n=(n, n, n), p=2)
    pr.dt = 6.0 * I.fd_stable_dt(pr)
    s2d = periodic_benchmark_state(fs, I.Problem(n=(n, n), p=2)).cpu().numpy()
    f0 = torch.tensor(I.extrude_3d(s2d, n), dtype=torch.float64, device="cuda")
    del s2d
    ref, ms_ref = _run(fs, pr, f0, steps, "f64")
    out = {"workload": f"3D {n}^3, p=2, dt=5e-3, benchmark IC at t=1 extruded along z (Eq. ic_eta_3d)",
           "steps": steps,
           "initial_phase_fraction": [float((f0[1 + i] > 0.5).double().mean()) for i in range(pr.p)],
           "f64": {"ms_per_step": ms_ref / steps,
                   "phase_fraction": [float((ref[1 + i] > 0.5).double().mean()) for i in range(pr.p)]}}
    for prec in ("f32", "tf32", "bf16x3"):
        g, ms = _run(fs, pr, f0.float(), steps, prec)
        linf = [float((g[f] - ref[f]).abs().max() / ref[f].abs().max()) for f in range(pr.nf)]
        pf = [float((g[1 + i] > 0.5).double().mean()) for i in range(pr.p)]
        out[prec] = {"ms_per_step": ms / steps, "rel_linf_vs_f64": linf, "phase_fraction": pf,
                     "speedup_vs_f64": ms_ref / ms}
    return out


def error_field(ref, phi):
    """E_phi = int (phi_0 - phi)^2 / int phi_0^2 (Eq. error_field)."""
    return float(((ref - phi) ** 2).sum() / (ref ** 2).sum())


def accuracy_study(steps: int, n: int = 1024):
    import torch
    from . import fs, inputs as I
    pr = I.Problem(n=(n, n), p=2)
    dt_fd = I.fd_stable_dt(pr)
    pr.dt = 6.0 * dt_fd
    t_end = steps * pr.dt
    f0 = periodic_benchmark_state(fs, pr)
    ref_pr = pr.replace(dt=pr.dt / 16)
    ref, ms_ref = _run(fs, ref_pr, f0, 16 * steps, "f64")
    res = {"workload": f"2D {n}^2, p=2, benchmark IC at t=1, FP64", "t_start": 1.0, "t_end": 1.0 + t_end,
           "reference": {"scheme": "FS", "dt": ref_pr.dt, "steps": 16 * steps, "ms": ms_ref}}

    def errs(g):
        return {"E_c": error_field(ref[0], g[0]), "E_eta": error_field(ref[1:].sum(0), g[1:].sum(0))}

    g, ms = _run(fs, pr, f0, steps, "f64")
    res["FS_f64"] = {"dt": pr.dt, "steps": steps, "ms": ms, **errs(g)}
    g, ms = _run(fs, pr, f0.float(), steps, "f32")
    res["FS_f32"] = {"dt": pr.dt, "steps": steps, "ms": ms, **errs(g)}
    for name, lap in (("FSFD2_f64", 1), ("FSFD4_f64", 2)):
        g, ms = _run(fs, pr.replace(lap=lap), f0, steps, "f64")
        res[name] = {"dt": pr.dt, "steps": steps, "ms": ms, **errs(g)}
    fd_dt_nominal = 0.95 * dt_fd
    n_fd = int(np.ceil(t_end / fd_dt_nominal))
    fd_pr = pr.replace(dt=t_end / n_fd)
    g, ms = _run(fs, fd_pr, f0, n_fd, "f64", scheme=fs.FS_SCHEME_EXPLICIT_FD)
    res["FD_f64"] = {"dt": fd_pr.dt, "steps": n_fd, "ms": ms, **errs(g)}
    res["FD_over_FS_time"] = res["FD_f64"]["ms"] / res["FS_f64"]["ms"]
    return res


def _time_steps(fs, pr, precision, scheme, steps):
    import torch
    from . import inputs as I
    dtype = torch.float64 if precision == "f64" else torch.float32
    plan = fs.Plan(pr, precision, scheme=scheme)
    plan.set_fields(torch.tensor(I.noise_fields(pr, seed=0), dtype=dtype, device="cuda"))
    plan.step(max(3, steps // 10))  # warm-up (graph capture, caches)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    plan.step(steps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    plan.close()
    return ms


COST_GRIDS = [(128, 128), (256, 256), (512, 512), (1024, 1024), (2048, 2048), (16, 16, 16), (32, 32, 32), (64, 64, 64),
              (128, 128, 128), (256, 256, 256)]


def cost_study(steps: int, grids=COST_GRIDS):
    from . import fs, inputs as I
    rows = []
    for n in grids:
        pr = I.Problem(n=n, p=4)
        pr.dt = 0.95 * I.fd_stable_dt(pr)
        for prec in ("f64", "f32"):
            k = steps if pr.npoints <= 1 << 21 else max(10, steps // 10)
            fs_ms = _time_steps(fs, pr, prec, fs.FS_SCHEME_SEMI_IMPLICIT_FS, k)
            fd_ms = _time_steps(fs, pr, prec, fs.FS_SCHEME_EXPLICIT_FD, k)
            rows.append({"grid": list(n), "precision": prec, "steps": k, "fs_ms_per_step": fs_ms,
                         "fd_ms_per_step": fd_ms, "fs_over_fd": fs_ms / fd_ms,
                         "fs_gpts_per_s": pr.npoints / (fs_ms / 1e3)})
    return {"workload": "p = 4 (5 fields), seeded +-0.01 noise, dt = 0.95 dt_FD for both schemes", "rows": rows}


# Table 1 of the paper: grids and time steps of the 2D accuracy study; the
# explicit FD time steps are the paper's own (stable, below the linearised
# bound of inputs.fd_stable_dt).
TABLE1_GRIDS = (128, 256, 512, 1024, 2048)
TABLE1_FS_DTS = (1e-4, 1e-3, 5e-3)
TABLE1_FD_DT = {128: 8.138e-3, 256: 5.086e-4, 512: 3.560e-5, 1024: 2.225e-6, 2048: 1.490e-7}


def spectral_resample(f: np.ndarray, n: int) -> np.ndarray:
    """Periodic fields (..., m, m) on an n x n grid of the same domain by
    Fourier interpolation: the modes |k_x|, |k_y| < min(m, n) / 2 are kept
    (the Nyquist bins are dropped, so the result is real) and the rest are
    zero.  For n >= m every grid receives the same band-limited field; for
    n < m the field is truncated to what the coarse grid represents.  Input
    preparation only (host numpy), not part of the time step."""
    m = f.shape[-1]
    F = np.fft.fft2(f, axes=(-2, -1))
    h = min(m, n) // 2
    idx = np.r_[0:h, -h + 1:0]
    out = np.zeros(f.shape[:-2] + (n, n), dtype=complex)
    out[..., idx[:, None], idx[None, :]] = F[..., idx[:, None], idx[None, :]]
    return np.real(np.fft.ifft2(out, axes=(-2, -1))) * (n * n) / (m * m)


def table1_study(t_span: float = 1.0, grids=TABLE1_GRIDS, dts=TABLE1_FS_DTS, ref_dt: float = 1e-4,
                 pre_n: int = 512, l: float = 200.0, p: int = 4, precision: str = "f64", fd_dts=None,
                 fd_max_steps: int = 100_000, fsfd_ref_dt_max_grid: int | None = None):
    """The 2D accuracy study of Section 3 (Table 1, Eq. error_field) over a
    shortened time window.

    Setting of the paper: domain 200 x 200, p = 4, the benchmark initial
    condition made periodic by the explicit FD scheme up to t = 1 (here on a
    pre_n^2 grid in FP64 at half its stable dt), the same t = 1 state on
    every grid (spectral_resample), then t = 1 -> 1 + t_span with the FS
    scheme (spectral |xi|^2 and the FS-FD O(dl^2) / O(dl^4) forms) at every
    (grid, dt) of Table 1, and with the explicit FD scheme at the paper's FD
    dt where that takes at most fd_max_steps steps.  Reference: spectral FS
    in FP64 on the finest grid at ref_dt (the paper's choice: 2048^2, 1e-4);
    the sweep case equal to it is the reference run itself (E = 0).  E_c and
    E_eta (eta = sum_i eta_i) of Eq. error_field are taken at the points of
    each grid (the reference sampled every finest/n points).  `f32_floor`:
    the reference case run in FP32 against the FP64 reference, the error
    FP32 rounding alone leaves after the dynamics amplify it.  The FS-FD
    forms at ref_dt run only on grids up to fsfd_ref_dt_max_grid (None: all;
    on the finest grid they cost as much as the reference each)."""
    import torch
    from . import fs, inputs as I
    nmax = max(grids)
    pre = I.Problem(n=(pre_n, pre_n), dx=(l / pre_n, l / pre_n), p=p)
    s_pre = periodic_benchmark_state(fs, pre).cpu().numpy()

    def problem(n, dt, lap=0):
        return I.Problem(n=(n, n), dx=(l / n, l / n), p=p, dt=dt, lap=lap)

    def start(n):
        return torch.tensor(spectral_resample(s_pre, n), dtype=torch.float64, device="cuda")

    ref_steps = int(round(t_span / ref_dt))
    f_ref0 = start(nmax)
    ref, ms_ref = _run(fs, problem(nmax, ref_dt), f_ref0, ref_steps, "f64")
    refsum = {}

    def errs(n, g):
        stride = nmax // n
        if n not in refsum:
            r = ref[:, ::stride, ::stride]
            refsum[n] = (r[0], r[1:].sum(0))
        rc, re = refsum[n]
        return {"E_c": error_field(rc, g[0]), "E_eta": error_field(re, g[1:].sum(0))}

    g, ms = _run(fs, problem(nmax, ref_dt), f_ref0.float(), ref_steps, "f32")
    floor = {"grid": nmax, "dt": ref_dt, "steps": ref_steps, "precision": "f32", "ms": ms, **errs(nmax, g)}
    del f_ref0, g
    rows = []
    for n in grids:
        f0 = start(n) if precision == "f64" else start(n).float()
        for lap, name in ((0, "FS"), (1, "FSFD2"), (2, "FSFD4")):
            for dt in dts:
                steps = int(round(t_span / dt))
                if lap and dt == ref_dt and fsfd_ref_dt_max_grid is not None and n > fsfd_ref_dt_max_grid:
                    continue
                if n == nmax and lap == 0 and dt == ref_dt and precision == "f64":
                    g, ms = ref, ms_ref
                else:
                    g, ms = _run(fs, problem(n, dt, lap), f0, steps, precision)
                rows.append({"grid": n, "scheme": name, "precision": precision, "dt": dt, "steps": steps, "ms": ms,
                             **errs(n, g)})
        fd_dt = (TABLE1_FD_DT if fd_dts is None else fd_dts).get(n)
        if fd_dt is not None:
            steps = int(np.ceil(t_span / fd_dt))
            if steps <= fd_max_steps:
                g, ms = _run(fs, problem(n, t_span / steps), start(n), steps, "f64", scheme=fs.FS_SCHEME_EXPLICIT_FD)
                rows.append({"grid": n, "scheme": "FD", "precision": "f64", "dt": t_span / steps, "steps": steps,
                             "ms": ms, **errs(n, g)})
        del f0
    return {"workload": f"2D {l:g} x {l:g}, p = {p}, benchmark IC at t = 1 (FD on {pre_n}^2), "
                        f"t = 1 -> {1 + t_span:g}",
            "reference": {"grid": nmax, "dt": ref_dt, "steps": ref_steps, "precision": "f64", "ms": ms_ref},
            "f32_floor": floor, "rows": rows}


# Table 2 of the paper: grids and explicit FD time steps of the 3D cases
# (FS at 5e-3 on every grid).
TABLE2_GRIDS = (16, 32, 64, 128, 256)
TABLE2_FD_DT = {16: 4.06e-2, 32: 2.54e-2, 64: 3.17e-3, 128: 7.94e-5, 256: 9.93e-6}


def table2_study(t_span: float = 0.5, grids=TABLE2_GRIDS, fs_dt: float = 5e-3, ref_dt: float = 5e-4,
                 pre_n: int = 512, l2d: float = 200.0, l3d: float = 100.0, p: int = 4, fd_dts=None,
                 fd_f64_max_steps: int = 10_000, fd_max_steps: int = 60_000):
    """The 3D cases of Section 3 (Table 2) over a shortened time window.

    Setting of the paper: the 2D benchmark state at t = 1 (domain 200 x
    200, p = 4, made periodic by explicit FD as in table1_study) placed on
    the z = lz/2 plane of a cube of side lz = 100 with the (2x, 2y) scaling
    (the n^2 grid of the 200-wide domain, index by index) and extruded along
    z by Eq. ic_eta_3d, c = c0 (inputs.extrude_3d); every grid of Table 2
    gets its own resampled state.  Runs t = 1 -> 1 + t_span: FS (spectral
    |xi|^2 and the FS-FD O(dl^2) / O(dl^4) forms) at fs_dt, FP64, and
    explicit FD at the paper's dt (FP64 up to fd_f64_max_steps steps, else
    FP32 up to fd_max_steps).  Timing: device time of each run, per unit of
    t and per step and point (the paper's 3D performance figure plots the
    wall time of t = 1 -> 100 and the time per step and point).  Accuracy:
    the paper compares none in 3D (its 256^3 grid is not fine enough for a
    reference); here E_phi of Eq. error_field against spectral FS FP64 on
    the finest grid at ref_dt < fs_dt, at the points of each grid -- a
    measure of each grid and scheme against the best run this sweep has, not
    against the continuum solution."""
    import torch
    from . import fs, inputs as I
    nmax = max(grids)
    pre = I.Problem(n=(pre_n, pre_n), dx=(l2d / pre_n, l2d / pre_n), p=p)
    s_pre = periodic_benchmark_state(fs, pre).cpu().numpy()

    def problem(n, dt, lap=0):
        h = l3d / n
        return I.Problem(n=(n, n, n), dx=(h, h, h), p=p, dt=dt, lap=lap)

    def start(n, dtype=torch.float64):
        f3 = I.extrude_3d(spectral_resample(s_pre, n), n, dz=l3d / n)
        return torch.tensor(f3, dtype=dtype, device="cuda")

    ref_steps = int(round(t_span / ref_dt))
    ref, ms_ref = _run(fs, problem(nmax, ref_dt), start(nmax), ref_steps, "f64")
    ref = ref.cpu()

    def errs(n, g):
        s = nmax // n
        r = ref[:, ::s, ::s, ::s]
        g = g.cpu()
        return {"E_c": error_field(r[0], g[0]), "E_eta": error_field(r[1:].sum(0), g[1:].sum(0))}

    rows = []
    for n in grids:
        npts = n ** 3
        f0 = start(n)
        steps = int(round(t_span / fs_dt))
        for lap, name in ((0, "FS"), (1, "FSFD2"), (2, "FSFD4")):
            g, ms = _run(fs, problem(n, fs_dt, lap), f0, steps, "f64")
            rows.append({"grid": n, "scheme": name, "precision": "f64", "dt": fs_dt, "steps": steps, "ms": ms,
                         "ms_per_t": ms / t_span, "ns_per_step_point": ms * 1e6 / (steps * npts), **errs(n, g)})
        fd_dt = (TABLE2_FD_DT if fd_dts is None else fd_dts)[n]
        steps = int(np.ceil(t_span / fd_dt))
        prec = "f64" if steps <= fd_f64_max_steps else "f32"
        if steps <= fd_max_steps:
            row = {"grid": n, "scheme": "FD", "precision": prec, "dt": t_span / steps, "steps": steps}
            try:
                g, ms = _run(fs, problem(n, t_span / steps), f0 if prec == "f64" else f0.float(), steps, prec,
                             scheme=fs.FS_SCHEME_EXPLICIT_FD)
                row.update(ms=ms, ms_per_t=ms / t_span, ns_per_step_point=ms * 1e6 / (steps * npts), **errs(n, g))
            except fs.FSError as e:  # a non-finite value: the FD step is unstable at this dt
                row.update(unstable=str(e))
            rows.append(row)
        del f0
    return {"workload": f"3D {l3d:g}^3, p = {p}, benchmark state at t = 1 (FD on {pre_n}^2 of the "
                        f"{l2d:g}^2 domain) extruded by Eq. ic_eta_3d, t = 1 -> {1 + t_span:g}",
            "reference": {"grid": nmax, "dt": ref_dt, "steps": ref_steps, "precision": "f64", "ms": ms_ref},
            "rows": rows}


def slab_study(steps: int = 20, grids=(1024, 2048), ranks=(1, 2, 4, 8)):
    """Per-rank kernel time of the slab step: R ranks of one grid held by one
    process, every rank's row pass (unpack, row kernel, pack) timed as one
    group and every column pass as another, the L2 flushed before each step;
    per rank = the group times / R (the GPU runs one rank's kernels at a
    time, as each GPU would).  The exchanges between the groups are device
    copies here (host-dispatch bound, not reported); between GPUs they are
    (2 nf + 1) (R - 1) N s / R^2 bytes per rank and step (`exchange_bytes`)."""
    import torch
    from . import fs, inputs as I, slab as S
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    rows = []
    for n in grids:
        pr = I.Problem(n=(n, n), p=2)
        pr.dt = 6.0 * I.fd_stable_dt(pr)
        f0 = torch.tensor(I.noise_fields(pr, seed=0), dtype=torch.float32, device="cuda")
        plan = fs.Plan(pr, "f32")
        plan.set_fields(f0)
        plan.step(3)
        plan_ms = 0.0
        for _ in range(steps):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            plan.step_async(1)
            b.record()
            torch.cuda.synchronize()
            plan_ms += a.elapsed_time(b) / steps
        plan.close()
        for R in ranks:
            L = S.LocalSlabs(pr, "f32", R)
            L.set_fields(f0)
            L.step(3)
            row_ms = col_ms = 0.0
            for _ in range(steps):
                flush.fill_(1.0)
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
                ev[0].record()
                for s in L.slabs:
                    s.row_pass()
                ev[1].record()
                S.exchange_local_forward(L.lays, [s.send for s in L.slabs], [s.colspec for s in L.slabs])
                ev[2].record()
                for s in L.slabs:
                    s.col_pass()
                ev[3].record()
                S.exchange_local_back(L.lays, [s.colspec for s in L.slabs], [s.recv for s in L.slabs])
                torch.cuda.synchronize()
                row_ms += ev[0].elapsed_time(ev[1]) / steps
                col_ms += ev[2].elapsed_time(ev[3]) / steps
            L.sync()
            L.close()
            fwd, back = L.lays[0].exchange_bytes(8)
            rows.append({"grid": n, "ranks": R, "row_ms_per_rank": row_ms / R, "col_ms_per_rank": col_ms / R,
                         "step_ms_per_rank": (row_ms + col_ms) / R, "plan_step_ms": plan_ms,
                         "exchange_bytes_per_rank": fwd + back})
    return {"workload": "2D n^2, p = 2, FP32, seeded +-0.01 noise, dt = 6 dt_FD; L2 flushed before each step",
            "rows": rows}


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_2306_04322_gb300.experiments")
    ap.add_argument("study", choices=["precision", "accuracy", "cost", "table1", "table2", "slab"])
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--t-span", type=float, default=None, help="time window (table1: 1, table2: 0.5)")
    ap.add_argument("--fd-max-steps", type=int, default=100_000, help="table1: longest explicit FD run")
    ap.add_argument("--fsfd-ref-dt-max-grid", type=int, default=None,
                    help="table1: largest grid of the FS-FD forms at the reference dt")
    args = ap.parse_args(argv)
    from . import build as B
    B.build()
    if args.study == "precision":
        out = precision_study(args.steps or 2000)
    elif args.study == "accuracy":
        out = accuracy_study(args.steps or 10000)
    elif args.study == "cost":
        out = cost_study(args.steps or 200)
    elif args.study == "slab":
        out = slab_study(args.steps or 20)
    elif args.study == "table2":
        out = table2_study(args.t_span or 0.5)
    else:
        out = table1_study(args.t_span or 1.0, fd_max_steps=args.fd_max_steps,
                           fsfd_ref_dt_max_grid=args.fsfd_ref_dt_max_grid)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
