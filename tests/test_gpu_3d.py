"""GPU parity of the 3D step (x pass, y forward, z step, y inverse; Eq.
Gamma_fft_3d and the FS-FD 3D forms) against the FP64 CPU oracle."""
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


def gpu_run(F, prob, fields, nsteps, precision="f64"):
    import torch
    dt = torch.float64 if precision == "f64" else torch.float32
    plan = F.Plan(prob, precision)
    plan.set_fields(torch.tensor(np.ascontiguousarray(fields), dtype=dt, device="cuda"))
    plan.step(nsteps)
    out = plan.get_fields().double().cpu().numpy()
    plan.close()
    return out


@pytest.mark.parametrize("n,p,lap,dx", [
    ((8, 8, 8), 1, 0, (1.0, 1.0, 1.0)),
    ((16, 32, 8), 2, 0, (1.0, 0.5, 2.0)),
    ((32, 16, 64), 0, 1, (1.0, 1.0, 1.0)),
    ((8, 64, 16), 3, 2, (0.7, 1.0, 1.3)),
    ((64, 64, 64), 2, 0, (1.0, 1.0, 1.0)),
    ((128, 8, 32), 1, 0, (1.0, 1.0, 1.0)),
])
def test_fp64_3d_matches_oracle(F, O, n, p, lap, dx):
    pr = I.Problem(n=n, dx=dx, p=p, lap=lap)
    pr.dt = 6.0 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=11, amp=0.05)
    ref1, _ = O.step(pr, f0, 1)
    assert rel_linf(gpu_run(F, pr, f0, 1), ref1) <= 1e-12
    ref, _ = O.step(pr, f0, 5)
    assert rel_linf(gpu_run(F, pr, f0, 5), ref) <= 1e-11


def test_fp64_3d_graph_path(F, O):
    pr = I.Problem(n=(16, 16, 16), p=2)
    pr.dt = 6.0 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=12)
    ref, _ = O.step(pr, f0, 70)
    assert rel_linf(gpu_run(F, pr, f0, 70), ref) <= 1e-10


def test_fp32_3d_256_one_step(F, O):
    """The 256^3, p = 2 FP32 workload (dt = 6 x FD-stable = 5e-3): one step
    against the FP64 oracle, every element."""
    pr = I.Problem(n=(256, 256, 256), p=2)
    pr.dt = 6.0 * I.fd_stable_dt(pr)
    assert abs(pr.dt - 5e-3) < 1e-15
    f0 = I.noise_fields(pr, seed=0)
    ref, _ = O.step(pr, f0, 1)
    got = gpu_run(F, pr, f0.astype(np.float32), 1, "f32")
    assert rel_linf(got, ref) <= 2e-6


def test_fp32_3d_mean_conserved(F):
    pr = I.Problem(n=(64, 64, 64), p=2)
    pr.dt = 6.0 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=13).astype(np.float32)
    m0 = f0[0].astype(np.float64).mean()
    got = gpu_run(F, pr, f0, 200, "f32")
    assert abs(got[0].mean() - m0) <= 2e-7


def test_3d_reading_fields_does_not_perturb_the_run(F, O):
    """3D carries c between steps in (kx, ky, z) space and keeps c's x spectrum
    in the df/dc slot: reading the fields between steps leaves the run bit for
    bit unchanged, and the run matches the oracle."""
    import torch
    pr = I.Problem(n=(32, 16, 64), p=2, dx=(1.0, 0.5, 1.0))
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    f0 = torch.tensor(I.noise_fields(pr, seed=21), device="cuda")
    plan = F.Plan(pr, "f64")
    plan.set_fields(f0)
    plan.step(12)
    full = plan.get_fields().cpu().numpy()
    plan.set_fields(f0)
    plan.step(5)
    plan.get_fields()
    plan.step(7)
    assert np.array_equal(full, plan.get_fields().cpu().numpy())
    plan.close()
    ref, _ = O.step(pr, f0.cpu().numpy(), 12)
    assert rel_linf(full, ref) <= 1e-11
