"""Batched ensembles: many 2D simulations of uneven sizes and parameters in
one plan (one persistent launch per pass), checked member by member against
the FP64 oracle and against single-simulation plans."""
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


def run_batch(F, probs, fields, nsteps, precision):
    import torch
    dt = torch.float64 if precision == "f64" else torch.float32
    plan = F.Plan(probs, precision)
    plan.set_fields([torch.tensor(np.ascontiguousarray(f), dtype=dt, device="cuda") for f in fields])
    plan.step(nsteps)
    out = [o.double().cpu().numpy() for o in plan.get_fields()]
    sched = F.fs_batch_schedule(plan.h)
    plan.close()
    return out, sched


def mixed_problems(sizes, p, seed):
    rng = np.random.default_rng(seed)
    probs = []
    for n in sizes:
        pr = I.Problem(n=n, p=p, M=5.0 * rng.uniform(0.5, 1.5), L=5.0 * rng.uniform(0.5, 1.5),
                       kappa_c=3.0 * rng.uniform(0.5, 1.5), kappa_eta=3.0 * rng.uniform(0.5, 1.5))
        pr.dt = 5.0 * I.fd_stable_dt(pr)
        probs.append(pr)
    return probs


def test_fp64_batch_matches_oracle_per_member(F, O):
    probs = mixed_problems([(64, 64), (128, 64), (64, 128), (256, 128), (64, 64)], p=2, seed=1)
    fields = [I.noise_fields(pr, seed=20 + i) for i, pr in enumerate(probs)]
    out1, sched = run_batch(F, probs, fields, 1, "f64")
    out5, _ = run_batch(F, probs, fields, 5, "f64")
    for pr, f0, g1, g5 in zip(probs, fields, out1, out5):
        r1, _ = O.step(pr, f0, 1)
        r5, _ = O.step(pr, f0, 5)
        assert rel_linf(g1, r1) <= 1e-12
        assert rel_linf(g5, r5) <= 1e-11
    row_grid, col_grid, row_items, col_items, row_form, col_form = sched
    assert 0 < row_grid <= row_items and 0 < col_grid <= col_items


def test_fp32_batch_matches_oracle_per_member(F, O):
    probs = mixed_problems([(128, 128), (256, 256), (128, 512), (512, 128)], p=2, seed=2)
    fields = [I.noise_fields(pr, seed=30 + i).astype(np.float32) for i, pr in enumerate(probs)]
    out, _ = run_batch(F, probs, fields, 1, "f32")
    for pr, f0, g in zip(probs, fields, out):
        r, _ = O.step(pr, f0.astype(np.float64), 1)
        assert rel_linf(g, r) <= 2e-6


def test_batch_equals_single_plans(F):
    """The ensemble launch runs the same per-simulation code as a plan of one:
    after 40 steps every member agrees with its own single-plan run.  The two
    kernels are compiled separately (FMA contraction may differ), so FP32
    rounding differences of one ulp per step grow along the trajectory; a
    member or parameter mix-up would differ by O(1e-2)."""
    import torch
    probs = I.batch_problems(12, seed=3, sizes=(128, 256, 512))
    fields = [I.noise_fields(pr, seed=40 + i).astype(np.float32) for i, pr in enumerate(probs)]
    out, _ = run_batch(F, probs, fields, 40, "f32")
    for pr, f0, g in zip(probs, fields, out):
        plan = F.Plan(pr, "f32")
        plan.set_fields(torch.tensor(f0, device="cuda"))
        plan.step(40)
        ref = plan.get_fields().double().cpu().numpy()
        plan.close()
        # FP32 parity bound of 2e-6 per step, times 40 steps, times 2 (growth)
        assert rel_linf(g, ref) <= 2e-6 * 40 * 2


@pytest.mark.parametrize("forms", [(1, 1), (2, 2), (2, 1), (1, 2)])
def test_fp32_batch_forms_match_oracle(F, O, forms):
    """Both ensemble kernel forms, pinned per pass, against the oracle member
    by member after one step and after 34 (the graph path)."""
    import torch
    probs = mixed_problems([(128, 128), (256, 256), (1024, 512), (512, 1024), (64, 128)], p=2, seed=4)
    fields = [I.noise_fields(pr, seed=50 + i) for i, pr in enumerate(probs)]
    plan = F.Plan(probs, "f32")
    F.fs_set_pass_forms(plan.h, *forms)
    plan.set_fields([torch.tensor(f, dtype=torch.float32, device="cuda") for f in fields])
    sched = F.fs_batch_schedule(plan.h)
    assert sched[4:] == forms
    plan.step(1)
    out1 = [o.double().cpu().numpy() for o in plan.get_fields()]
    plan.step(33)
    out34 = [o.double().cpu().numpy() for o in plan.get_fields()]
    plan.close()
    for pr, f0, g1, g34 in zip(probs, fields, out1, out34):
        r1, _ = O.step(pr, f0, 1)
        r34, _ = O.step(pr, r1, 33)
        assert rel_linf(g1, r1) <= 2e-6 * 2, (pr.n, forms)
        assert rel_linf(g34, r34) <= 2e-6 * 34 * 2, (pr.n, forms)


def test_batch_rejects_unsupported_members(F):
    probs = [I.Problem(n=(64, 32), p=1, dt=1e-3), I.Problem(n=(128, 128), p=1, dt=1e-3)]
    with pytest.raises(F.FSError) as ei:
        F.Plan(probs, "f32")
    assert ei.value.status == F.FS_ERR_UNSUPPORTED
