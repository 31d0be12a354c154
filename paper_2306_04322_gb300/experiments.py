"""Configuration-level studies on the GPU (each prints one JSON object).

    python -m paper_2306_04322_gb300.experiments precision   [--steps 2000]
    python -m paper_2306_04322_gb300.experiments accuracy    [--steps 10000]
    python -m paper_2306_04322_gb300.experiments cost        [--steps 200]

Both start from the benchmark initial condition of Section 3 (Eqs. ic_c,
ic_eta with p = 2, dx = 1), made periodic as the paper does: the explicit FD
scheme, run in FP64 on the GPU at half its stable dt, takes it to t = 1.

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
    the grid sizes of the paper's Tables 1 and 2 that fit here (2D 128^2 ..
    1024^2, 3D 16^3 .. 256^3), p = 4 as in the paper, FP64 and FP32; the
    ratio FS / FD is the paper's per-step cost comparison (Section 3).
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


def periodic_benchmark_state(fs, pr2d, t_end: float = 1.0):
    """Benchmark initial condition (Section 3) advanced to t_end by the
    explicit FD scheme in FP64 at half its stable dt; an (nf, ny, nx) float64
    CUDA tensor."""
    import torch
    from . import inputs as I
    n = int(np.ceil(t_end / (0.5 * I.fd_stable_dt(pr2d))))
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


COST_GRIDS = [(128, 128), (256, 256), (512, 512), (1024, 1024), (16, 16, 16), (32, 32, 32), (64, 64, 64),
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


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_2306_04322_gb300.experiments")
    ap.add_argument("study", choices=["precision", "accuracy", "cost"])
    ap.add_argument("--steps", type=int, default=None)
    args = ap.parse_args(argv)
    from . import build as B
    B.build()
    if args.study == "precision":
        out = precision_study(args.steps or 2000)
    elif args.study == "accuracy":
        out = accuracy_study(args.steps or 10000)
    else:
        out = cost_study(args.steps or 200)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
