"""Axes of 2048, the finest 2D grid of the paper's Table 1: rows of 2048 run
the x pass with 32 values per thread (FP32 and FP64), columns of 2048 the y
pass with 16 (FP32) / 8 (FP64) values per thread and two / one columns per
tile.  CUDA step through the C ABI against the FP64 CPU oracle, relative
L-inf per field; the tolerances are those of the 1024 cases."""
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
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return max(np.max(np.abs(a[f] - b[f])) / max(np.max(np.abs(b[f])), 1e-300) for f in range(b.shape[0]))


def gpu_run(F, prob, fields, nsteps, precision="f64", scheme=None):
    import torch
    dt = torch.float64 if precision == "f64" else torch.float32
    kw = {} if scheme is None else {"scheme": scheme}
    plan = F.Plan(prob, precision, **kw)
    plan.set_fields(torch.tensor(np.ascontiguousarray(fields), dtype=dt, device="cuda"))
    plan.step(nsteps)
    out = plan.get_fields().double().cpu().numpy()
    plan.close()
    return out


def test_fp64_2048_square_p4(F, O):
    """The paper's 2D setting: 2048^2 with p = 4 (five fields)."""
    pr = I.Problem(n=(2048, 2048), p=4)
    pr.dt = 6.0 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=20)
    ref, _ = O.step(pr, f0, 1)
    assert rel_linf(gpu_run(F, pr, f0, 1), ref) <= 1e-12


@pytest.mark.parametrize("n,p,lap", [((2048, 8), 1, 0), ((8, 2048), 2, 0), ((2048, 64), 3, 2), ((64, 2048), 0, 1)])
def test_fp64_2048_thin_grids(F, O, n, p, lap):
    pr = I.Problem(n=n, p=p, lap=lap, dx=(0.5, 1.0))
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=21, amp=0.05)
    ref, _ = O.step(pr, f0, 1)
    assert rel_linf(gpu_run(F, pr, f0, 1), ref) <= 1e-12
    ref5, _ = O.step(pr, f0, 5)
    assert rel_linf(gpu_run(F, pr, f0, 5), ref5) <= 1e-11


def test_fp32_2048_square(F, O):
    pr = I.Problem(n=(2048, 2048), p=2)
    pr.dt = 6.0 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=22)
    ref, _ = O.step(pr, f0, 1)
    err = rel_linf(gpu_run(F, pr, f0.astype(np.float32), 1, "f32"), ref)
    assert err <= 2e-6, err


@pytest.mark.parametrize("n,p", [((2048, 128), 2), ((128, 2048), 1)])
def test_fp32_2048_several_steps_and_mean(F, O, n, p):
    """Steady state (carried spectra) and the final inverse pass; the FP64
    mean carry keeps mean(c) to FP32 rounding of the input."""
    pr = I.Problem(n=n, p=p)
    pr.dt = 6.0 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=23).astype(np.float32)
    ref, _ = O.step(pr, f0.astype(np.float64), 10)
    got = gpu_run(F, pr, f0, 10, "f32")
    assert rel_linf(got, ref) <= 1e-5
    assert abs(got[0].mean() - f0[0].astype(np.float64).mean()) <= 2e-7


@pytest.mark.parametrize("precision,tol", [("tf32", 4e-6), ("bf16x3", 5e-5)])
@pytest.mark.parametrize("n", [(2048, 128), (128, 2048)])
def test_tc_variants_2048(F, O, precision, tol, n):
    pr = I.Problem(n=n, p=2)
    pr.dt = 6.0 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=24).astype(np.float32)
    ref, _ = O.step(pr, f0.astype(np.float64), 1)
    assert rel_linf(gpu_run(F, pr, f0, 1, precision), ref) <= tol


def test_free_energy_2048(F, O):
    import torch
    pr = I.Problem(n=(2048, 64), dx=(1.0, 0.5), p=2)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=25, amp=0.1)
    plan = F.Plan(pr, "f64")
    plan.set_fields(torch.tensor(f0, dtype=torch.float64, device="cuda"))
    E0, _ = plan.free_energy()
    plan.close()
    Fo = O.free_energy(pr, f0)
    assert abs(E0 - Fo) <= 1e-12 * abs(Fo)


def test_fd_2048_square(F, O):
    pr = I.Problem(n=(2048, 2048), p=2)
    pr.dt = 0.95 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=26)
    ref = O.fd_step(pr, f0, 1)
    assert rel_linf(gpu_run(F, pr, f0, 1, scheme=F.FS_SCHEME_EXPLICIT_FD), ref) <= 1e-12


def test_adjoint_and_batch_stop_at_1024(F):
    import torch
    pr = I.Problem(n=(2048, 64), p=1)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    plan = F.Plan(pr, "f32")
    u = torch.zeros((pr.nf,) + pr.shape, dtype=torch.float32, device="cuda")
    with pytest.raises(F.FSError) as ei:
        plan.step_adjoint(u, u, torch.empty_like(u))
    assert ei.value.status == F.FS_ERR_UNSUPPORTED
    plan.close()
    with pytest.raises(F.FSError) as ei:
        F.Plan([pr, I.Problem(n=(128, 128), p=1, dt=1e-3)], "f32")
    assert ei.value.status == F.FS_ERR_UNSUPPORTED
