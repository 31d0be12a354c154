"""Differentiable trajectories of the FS step for parameter fitting.

`FSTrajectory.apply(theta, u0, prob, precision, nsteps, every)` runs `nsteps`
time steps from u0 with theta = (M, L, kappa_c, kappa_eta) and returns the
snapshots u(every * s), s = 1..nsteps/every, stacked.  Its backward pass is
the hand-written adjoint: for each segment in reverse it recomputes the
segment's states from the checkpoint stored at its start (one checkpoint
every `every` steps), then runs fs_step_adjoint backwards through them,
accumulating the sensitivities of the loss to theta and to u0.  Every step of
the computation runs in libfs_gb300.so; this module only orders the calls.
"""
from __future__ import annotations

import torch
from torch.autograd.function import once_differentiable

from . import fs as _fs

THETA_NAMES = ("M", "L", "kappa_c", "kappa_eta")


def _with_theta(prob, theta):
    vals = [float(v) for v in theta]
    return prob.replace(**dict(zip(THETA_NAMES, vals)))


class FSTrajectory(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, u0, prob, precision, nsteps, every):
        if nsteps % every:
            raise ValueError("nsteps must be a multiple of every")
        pr = _with_theta(prob, theta.detach().cpu().tolist())
        plan = _fs.Plan(pr, precision)
        plan.set_fields(u0.detach().contiguous())
        checkpoints, snaps = [u0.detach().clone()], []
        nseg = nsteps // every
        for s in range(nseg):
            plan.step(every)
            u = plan.get_fields()
            snaps.append(u)
            if s + 1 < nseg:
                checkpoints.append(u.clone())
        ctx.plan, ctx.checkpoints, ctx.every = plan, checkpoints, every
        ctx.theta_dtype, ctx.theta_device = theta.dtype, theta.device
        return torch.stack(snaps)

    @staticmethod
    @once_differentiable
    def backward(ctx, gsnap):
        # The plan (and its device workspace) lives from forward to the one
        # backward pass that may follow; a second backward through the same
        # graph (retain_graph=True) would find it closed.
        if ctx.plan is None:
            raise RuntimeError("FSTrajectory.backward ran twice on one forward: the plan was released after "
                               "the first backward; run the forward again")
        plan, every = ctx.plan, ctx.every
        nf = plan.nf
        lam = torch.zeros_like(ctx.checkpoints[0])
        grad = [0.0, 0.0, 0.0, 0.0]
        for s in reversed(range(len(ctx.checkpoints))):
            if gsnap is not None:
                lam = lam + gsnap[s].to(lam.dtype)
            states = [ctx.checkpoints[s]]
            plan.set_fields(states[0])
            for _ in range(1, every):
                plan.step(1)
                states.append(plan.get_fields())
            for j in reversed(range(every)):
                out = torch.empty_like(lam)
                g = _fs.fs_step_adjoint(plan.h, [states[j][f] for f in range(nf)],
                                        [lam[f].contiguous() for f in range(nf)],
                                        [out[f] for f in range(nf)])
                grad = [a + b for a, b in zip(grad, g)]
                lam = out
        plan.close()
        ctx.plan = None
        ctx.checkpoints = None
        gtheta = torch.tensor(grad, dtype=ctx.theta_dtype, device=ctx.theta_device)
        return gtheta, lam, None, None, None, None


def trajectory(theta, u0, prob, precision="f32", nsteps=500, every=50):
    return FSTrajectory.apply(theta, u0, prob, precision, nsteps, every)


def misfit_loss(snaps, target):
    """L2 misfit of the snapshots to a target trajectory, sum over snapshots of
    ||u - u*||^2 / N (N grid points per field)."""
    npts = snaps[0, 0].numel()
    return ((snaps - target.to(snaps.dtype)) ** 2).sum() / npts
