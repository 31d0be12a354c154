"""The differentiable 512^2 run: a target trajectory from the FP64 oracle
with the paper's (M, L, kappa_c, kappa_eta), the model run from 1.2 theta*
(FP32 and FP64), 500 steps with a checkpoint and a snapshot every 50, loss =
sum of ||u(50 s) - u*(50 s)||^2 / N.  The adjoint gradients are checked
against central differences of the FP64 GPU loss (h = 1e-4 relative; bound
1e-4) and against the oracle adjoint over the same trajectory."""
import json
import os

import numpy as np
import pytest

from paper_2306_04322_gb300 import inputs as I

pytestmark = pytest.mark.gpu

STEPS, EVERY = 500, 50


@pytest.fixture(scope="module")
def F():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_04322_gb300 import build as B
    from paper_2306_04322_gb300 import fs
    B.build()
    fs.lib()
    return fs


def test_config5_adjoint_gradients(F, O):
    import torch
    from paper_2306_04322_gb300 import adjoint as A
    O.set_threads(os.cpu_count() or 1)
    pr = I.Problem(n=(512, 512), p=2)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    star = np.array([5.0, 5.0, 3.0, 3.0])
    u0 = I.noise_fields(pr, seed=0)
    tgt, u = [], u0.copy()
    for _ in range(STEPS // EVERY):
        u, _ = O.step(pr, u, EVERY)
        tgt.append(u)
    target = torch.tensor(np.stack(tgt), device="cuda")
    theta = 1.2 * star
    grads, losses = {}, {}
    for prec in ("f32", "f64"):
        th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
        u0t = torch.tensor(u0, dtype=torch.float64 if prec == "f64" else torch.float32, device="cuda")
        loss = A.misfit_loss(A.trajectory(th, u0t, pr, prec, STEPS, EVERY), target)
        loss.backward()
        grads[prec], losses[prec] = th.grad.numpy(), float(loss.detach())
    fd = []
    u0t = torch.tensor(u0, device="cuda")
    for q in range(4):
        h = 1e-4 * theta[q]
        vals = []
        for sgn in (1, -1):
            tq = theta.copy()
            tq[q] += sgn * h
            with torch.no_grad():
                vals.append(float(A.misfit_loss(A.trajectory(torch.tensor(tq), u0t, pr, "f64", STEPS, EVERY),
                                                target)))
        fd.append((vals[0] - vals[1]) / (2 * h))
    fd = np.array(fd)
    # oracle adjoint through the same trajectory (checkpointed the same way)
    prt = pr.replace(M=theta[0], L=theta[1], kappa_c=theta[2], kappa_eta=theta[3])
    N = pr.npoints
    ckpt, u = [u0.copy()], u0.copy()
    for _ in range(STEPS // EVERY - 1):
        u, _ = O.step(prt, u, EVERY)
        ckpt.append(u.copy())
    lam, gor = np.zeros_like(u0), np.zeros(4)
    for s in reversed(range(STEPS // EVERY)):
        states = [ckpt[s]]
        for _ in range(EVERY):
            nxt, _ = O.step(prt, states[-1], 1)
            states.append(nxt)
        lam = lam + 2.0 * (states[EVERY] - tgt[s]) / N
        for j in reversed(range(EVERY)):
            lam, g = O.adjoint_step(prt, states[j], lam)
            gor += g
    report = {"loss_f32": losses["f32"], "loss_f64": losses["f64"], "grad_f32": grads["f32"].tolist(),
              "grad_f64": grads["f64"].tolist(), "grad_fd_f64": fd.tolist(), "grad_oracle": gor.tolist()}
    out_dir = os.environ.get("FS_RESULTS_DIR")  # optional record of the numbers
    if out_dir:
        os.makedirs(out_dir, exist_ok=True)
        with open(os.path.join(out_dir, "config5_adjoint.json"), "w") as fh:
            json.dump(report, fh)
    assert np.all(np.abs(grads["f64"] - fd) <= 1e-4 * np.abs(fd)), report
    assert np.all(np.abs(grads["f64"] - gor) <= 1e-8 * np.max(np.abs(gor))), report
    # FP32 adjoint: error against the FP64 gradient stated in the report, bounded here
    assert np.all(np.abs(grads["f32"] - grads["f64"]) <= 2e-2 * np.max(np.abs(grads["f64"]))), report
