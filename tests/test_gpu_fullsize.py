"""Parity at the benchmark sizes, element by element against the FP64 oracle,
through the launch paths the benchmark times (long runs replay the captured
32-step graph: fs_step(40) is one eager step from the real fields, one graph
replay of 32 steps and 7 eager steps).

Tolerances (relative L-inf per field, max over fields):
  FP64: 1e-12 after one step; 1e-11 after 40 steps (Algorithm 1 in FP64
        differs from the oracle by rounding only; 40 steps of growth at rate
        <= w L stay well inside a factor 10).
  FP32: 2e-6 after one step (FP32 transforms of length up to 1024: about
        log2(N) roundings of 6e-8 each); after k steps at most k times that,
        times the growth factor exp(w L k dt) of the linearised step, which is
        below 2 at the time steps here: 2e-6 * 40 * 2 = 1.6e-4 after 40 steps.
"""
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


def fp32_bound(k: int) -> float:
    return 2e-6 * k * 2.0


def headline():
    pr = I.Problem(n=(1024, 1024), p=2)
    pr.dt = 6.0 * I.fd_stable_dt(pr)
    return pr


def run_plan(F, pr, f0, chunks, precision):
    import torch
    dt = torch.float64 if precision == "f64" else torch.float32
    plan = F.Plan(pr, precision)
    plan.set_fields(torch.tensor(np.ascontiguousarray(f0), dtype=dt, device="cuda"))
    outs = []
    for n in chunks:
        plan.step(n)
        outs.append(plan.get_fields().double().cpu().numpy())
    plan.close()
    return outs


def test_headline_fp32_40_steps_graph_path(F, O):
    """2D 1024^2, p = 2, FP32, dt = 6 dt_FD: the benchmark's workload."""
    pr = headline()
    f0 = I.noise_fields(pr, seed=0)
    g1, g41 = run_plan(F, pr, f0.astype(np.float32), [1, 40], "f32")
    r1, _ = O.step(pr, f0, 1)
    r41, _ = O.step(pr, r1, 40)
    e1, e41 = rel_linf(g1, r1), rel_linf(g41, r41)
    print(f"1024^2 FP32: 1 step {e1:.2e}, 41 steps {e41:.2e}")
    assert e1 <= fp32_bound(1)
    assert e41 <= fp32_bound(41)


def test_1024_fp64_40_steps_graph_path(F, O):
    pr = headline()
    f0 = I.noise_fields(pr, seed=4)
    (g40,) = run_plan(F, pr, f0, [40], "f64")
    r40, _ = O.step(pr, f0, 40)
    e = rel_linf(g40, r40)
    print(f"1024^2 FP64: 40 steps {e:.2e}")
    assert e <= 1e-11


def test_3d_256_fp32_five_steps(F, O):
    pr = I.Problem(n=(256, 256, 256), p=2)
    pr.dt = 6.0 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=0)
    (g5,) = run_plan(F, pr, f0.astype(np.float32), [5], "f32")
    r5, _ = O.step(pr, f0, 5)
    e = rel_linf(g5, r5)
    print(f"256^3 FP32: 5 steps {e:.2e}")
    assert e <= fp32_bound(5)


def test_batch_with_1024_members_fp32(F, O):
    """An ensemble holding two 1024^2 members (the batch row kernel with 16
    values per thread and the batch column kernel at their largest size) and
    two smaller ones, after 1 step and after 41 steps (graph path)."""
    import torch
    rng = np.random.default_rng(5)
    probs = []
    for n in [(1024, 1024), (256, 256), (1024, 1024), (128, 128)]:
        pr = I.Problem(n=n, p=2, M=5.0 * rng.uniform(0.5, 1.5), L=5.0 * rng.uniform(0.5, 1.5),
                       kappa_c=3.0 * rng.uniform(0.5, 1.5), kappa_eta=3.0 * rng.uniform(0.5, 1.5))
        pr.dt = 5.0 * I.fd_stable_dt(pr)
        probs.append(pr)
    fields = [I.noise_fields(pr, seed=30 + i) for i, pr in enumerate(probs)]
    plan = F.Plan(probs, "f32")
    plan.set_fields([torch.tensor(f, dtype=torch.float32, device="cuda") for f in fields])
    plan.step(1)
    out1 = [o.double().cpu().numpy() for o in plan.get_fields()]
    plan.step(40)
    out41 = [o.double().cpu().numpy() for o in plan.get_fields()]
    plan.close()
    for pr, f0, g1, g41 in zip(probs, fields, out1, out41):
        r1, _ = O.step(pr, f0, 1)
        r41, _ = O.step(pr, r1, 40)
        e1, e41 = rel_linf(g1, r1), rel_linf(g41, r41)
        print(f"batch member {pr.n}: 1 step {e1:.2e}, 41 steps {e41:.2e}")
        assert e1 <= fp32_bound(1)
        assert e41 <= fp32_bound(41)
