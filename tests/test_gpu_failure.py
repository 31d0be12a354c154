"""Failure detection on the GPU without a fault.

* Timeout path: the plan's test hook cuts the first bounded wait of every pass
  short (no poll at all), so every pass reports a timeout and returns early
  after waiting, bounded, for its own copies.  fs_step must return
  FS_ERR_TIMEOUT, and the plan must step correctly again (against the oracle)
  once the hook is off and the fields are set again.
* Bounds-checked build (FS_DEBUG_BOUNDS, the substitute for a memory checker):
  every checked global access outside its buffer sets an error bit instead of
  reaching memory; the small-grid parity cases must run with no bit set and
  still match the oracle.
"""
import contextlib

import numpy as np
import pytest

from paper_2306_04322_gb300 import inputs as I

pytestmark = pytest.mark.gpu


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


def rel_linf(a, b):
    return max(np.max(np.abs(a[f] - b[f])) / max(np.max(np.abs(b[f])), 1e-300) for f in range(b.shape[0]))


@pytest.mark.parametrize("n,precision", [((64, 64), "f64"), ((128, 64), "f32"), ((32, 16, 16), "f32")])
def test_timeout_reported_then_clean_step(F, O, n, precision):
    import torch
    dt = torch.float64 if precision == "f64" else torch.float32
    pr = I.Problem(n=n, p=2)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=11)
    plan = F.Plan(pr, precision)
    plan.set_fields(torch.tensor(f0, dtype=dt, device="cuda"))
    F.fs_test_short_wait(plan.h, True)
    with pytest.raises(F.FSError) as ei:
        plan.step(3)
    assert ei.value.status == F.FS_ERR_TIMEOUT
    F.fs_test_short_wait(plan.h, False)
    plan.set_fields(torch.tensor(f0, dtype=dt, device="cuda"))
    plan.step(3)
    got = plan.get_fields().double().cpu().numpy()
    plan.close()
    ref, _ = O.step(pr, f0, 3)
    assert rel_linf(got, ref) <= (1e-12 if precision == "f64" else 2e-5)


def test_timeout_hook_also_cuts_the_graph_path(F):
    """Long runs replay a captured graph; the hook rebuilds it."""
    import torch
    pr = I.Problem(n=(64, 64), p=1)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    plan = F.Plan(pr, "f32")
    plan.set_fields(torch.tensor(I.noise_fields(pr, seed=12), dtype=torch.float32, device="cuda"))
    plan.step(40)  # builds the graph
    F.fs_test_short_wait(plan.h, True)
    with pytest.raises(F.FSError) as ei:
        plan.step(40)
    assert ei.value.status == F.FS_ERR_TIMEOUT
    F.fs_test_short_wait(plan.h, False)
    plan.close()


@contextlib.contextmanager
def bounds_library(F):
    """Route the binding through the bounds-checked build for the block."""
    from paper_2306_04322_gb300 import build as B
    L = F.bind(B.build(variant="bounds"))
    saved = F._lib
    F._lib = L
    try:
        yield L
    finally:
        F._lib = saved


@pytest.mark.parametrize("n,p,precision,lap", [
    ((8, 8), 1, "f64", 0), ((16, 32), 2, "f64", 1), ((64, 64), 1, "f32", 0), ((64, 8), 0, "f64", 2),
    ((32, 64), 2, "f32", 0), ((8, 16, 8), 1, "f64", 0), ((16, 16, 32), 2, "f32", 0),
    ((256, 256), 2, "f32", 0), ((256, 8, 8), 1, "f32", 0)])
def test_bounds_checked_build_small_grids(F, O, n, p, precision, lap):
    import torch
    dt = torch.float64 if precision == "f64" else torch.float32
    pr = I.Problem(n=n, p=p, lap=lap)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=13)
    with bounds_library(F) as L:
        assert L.fs_version()
        plan = F.Plan(pr, precision)
        plan.set_fields(torch.tensor(f0, dtype=dt, device="cuda"))
        plan.step(1)
        plan.step(4)  # fs_step returns FS_ERR_CUDA ("index out of bounds") if a check fired
        got = plan.get_fields().double().cpu().numpy()
        plan.sync()
        plan.close()
    ref, _ = O.step(pr, f0, 5)
    assert rel_linf(got, ref) <= (1e-11 if precision == "f64" else 2e-5)


def test_bounds_checked_build_fd_batch_and_static(F, O):
    import torch
    with bounds_library(F):
        # explicit FD scheme
        pr = I.Problem(n=(32, 16), p=1)
        pr.dt = 0.5 * I.fd_stable_dt(pr)
        f0 = I.noise_fields(pr, seed=14)
        plan = F.Plan(pr, "f64", scheme=F.FS_SCHEME_EXPLICIT_FD)
        plan.set_fields(torch.tensor(f0, device="cuda"))
        plan.step(3)
        got = plan.get_fields().cpu().numpy()
        plan.close()
        ref = O.fd_step(pr, f0, 3)
        assert rel_linf(got, ref) <= 1e-12
        # batched ensemble of two members (FP32: the ensemble's precision)
        probs = [I.Problem(n=(128, 128), p=1), I.Problem(n=(256, 128), p=1)]
        for q in probs:
            q.dt = 5.0 * I.fd_stable_dt(q)
        fields = [I.noise_fields(q, seed=15 + i) for i, q in enumerate(probs)]
        plan = F.Plan(probs, "f32")
        plan.set_fields([torch.tensor(f, dtype=torch.float32, device="cuda") for f in fields])
        plan.step(2)
        outs = [o.double().cpu().numpy() for o in plan.get_fields()]
        plan.sync()
        plan.close()
        for q, f, g in zip(probs, fields, outs):
            assert rel_linf(g, O.step(q, f, 2)[0]) <= 8e-6
        # allocation-free entry point
        pr = I.Problem(n=(32, 32), p=2)
        pr.dt = 5.0 * I.fd_stable_dt(pr)
        f0 = I.noise_fields(pr, seed=17)
        buf = torch.tensor(f0, device="cuda")
        assert F.fs_step2d_static(F.make_params(pr, "f64"), buf, 3) == F.FS_OK
        assert rel_linf(buf.cpu().numpy(), O.step(pr, f0, 3)[0]) <= 1e-12
