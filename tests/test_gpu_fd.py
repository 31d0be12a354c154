"""GPU parity of the explicit finite-difference comparison scheme (Section
2.2: forward Euler, 5-point (2D) / 7-point (3D) Laplacian, periodic) against
the FP64 oracle."""
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


def run_fd(F, pr, f0, n, precision="f64"):
    import torch
    dt = torch.float64 if precision == "f64" else torch.float32
    plan = F.Plan(pr, precision, scheme=F.FS_SCHEME_EXPLICIT_FD)
    plan.set_fields(torch.tensor(np.ascontiguousarray(f0), dtype=dt, device="cuda"))
    plan.step(n)
    out = plan.get_fields().double().cpu().numpy()
    plan.close()
    return out


@pytest.mark.parametrize("n,p,dx", [((64, 64), 1, (1.0, 1.0)), ((128, 32), 2, (0.5, 1.0)),
                                    ((8, 8), 0, (1.0, 1.0)), ((256, 16), 4, (1.0, 2.0)),
                                    ((1024, 1024), 2, (1.0, 1.0))])
def test_fd_fp64_matches_oracle(F, O, n, p, dx):
    pr = I.Problem(n=n, dx=dx, p=p)
    pr.dt = 0.95 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=8)
    ref1 = O.fd_step(pr, f0, 1)
    assert rel_linf(run_fd(F, pr, f0, 1), ref1) <= 1e-12
    if pr.npoints <= 65536:
        ref = O.fd_step(pr, f0, 50)
        assert rel_linf(run_fd(F, pr, f0, 50), ref) <= 1e-10


def test_fd_fp32_matches_oracle(F, O):
    pr = I.Problem(n=(128, 128), p=2)
    pr.dt = 0.95 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=9)
    ref = O.fd_step(pr, f0, 10)
    assert rel_linf(run_fd(F, pr, f0.astype(np.float32), 10, "f32"), ref) <= 1e-5


def test_fd_conserves_mean_c(F):
    pr = I.Problem(n=(256, 256), p=2)
    pr.dt = 0.95 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=10)
    out = run_fd(F, pr, f0, 333)
    assert abs(out[0].mean() - f0[0].mean()) < 1e-13


@pytest.mark.parametrize("n,p,dx", [((16, 16, 16), 2, (1.0, 1.0, 1.0)), ((32, 16, 8), 1, (1.0, 0.5, 2.0)),
                                    ((8, 8, 8), 0, (1.0, 1.0, 1.0)), ((64, 32, 16), 4, (1.0, 1.0, 1.0))])
def test_fd3_fp64_matches_oracle(F, O, n, p, dx):
    pr = I.Problem(n=n, dx=dx, p=p)
    pr.dt = 0.95 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=11)
    assert rel_linf(run_fd(F, pr, f0, 1), O.fd_step(pr, f0, 1)) <= 1e-12
    assert rel_linf(run_fd(F, pr, f0, 20), O.fd_step(pr, f0, 20)) <= 1e-10


def test_fd3_fp32_and_mean(F, O):
    pr = I.Problem(n=(32, 32, 32), p=2)
    pr.dt = 0.95 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=12)
    assert rel_linf(run_fd(F, pr, f0.astype(np.float32), 10, "f32"), O.fd_step(pr, f0, 10)) <= 1e-5
    out = run_fd(F, pr, f0, 200)
    assert abs(out[0].mean() - f0[0].mean()) < 1e-13
