"""Command-line runner: advance one seeded synthetic problem on the GPU.

    python -m paper_2306_04322_gb300 --grid 1024 1024 --p 2 --precision f32 --steps 100
    python -m paper_2306_04322_gb300 --grid 256 256 256 --p 2 --precision f32 --steps 10 --dt-factor 6

Prints the elapsed device time, throughput and mean(c) drift.  Fields are the
seeded noise of `inputs.noise_fields`; dt is dt-factor x the explicit-FD
stable dt.  Useful as a fixed command line for profilers.
"""
from __future__ import annotations

import argparse
import sys


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_2306_04322_gb300")
    ap.add_argument("--grid", type=int, nargs="+", default=[1024, 1024])
    ap.add_argument("--p", type=int, default=2)
    ap.add_argument("--precision", default="f32", choices=["f32", "f64", "tf32", "bf16x3"])
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--dt-factor", type=float, default=6.0)
    ap.add_argument("--scheme", default="fs", choices=["fs", "fd"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--forms", type=int, nargs=2, default=None, metavar=("ROW", "COL"),
                    help="kernel forms of the row and column passes (fs_set_pass_forms: 0 default, 1 half-length "
                         "/ tile, 2 warp per line, 3 two warps per line)")
    args = ap.parse_args(argv)

    import torch
    from . import fs, inputs as I
    pr = I.Problem(n=tuple(args.grid), p=args.p)
    pr.dt = args.dt_factor * I.fd_stable_dt(pr)
    dtype = torch.float64 if args.precision == "f64" else torch.float32
    f0 = torch.tensor(I.noise_fields(pr, seed=args.seed), dtype=dtype, device="cuda")
    scheme = fs.FS_SCHEME_EXPLICIT_FD if args.scheme == "fd" else fs.FS_SCHEME_SEMI_IMPLICIT_FS
    plan = fs.Plan(pr, args.precision, scheme=scheme)
    if args.forms:
        fs.fs_set_pass_forms(plan.h, *args.forms)
    plan.set_fields(f0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    plan.step(args.steps)
    e1.record()
    out = plan.get_fields()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    drift = float(out[0].double().mean() - f0[0].double().mean())
    print(f"grid {tuple(args.grid)} p={args.p} {args.precision} {args.scheme}: {args.steps} steps in {ms:.3f} ms, "
          f"{pr.npoints * args.steps / (ms / 1e3):.4g} grid-point-steps/s, mean(c) drift {drift:.3e}, "
          f"launches {plan.last_launch_count}")
    plan.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
