"""GPU parity: the CUDA step (through the C ABI) against the FP64 CPU oracle,
element by element on seeded inputs.

Tolerances (relative L-inf per field, max|gpu - oracle| / max|oracle|):
  FP64: 1e-12 after one step, 1e-8 after 200 steps (64^2, p = 1, config 1);
  FP32: stated per test (one-step rounding of FP32 transforms).
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
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return max(np.max(np.abs(a[f] - b[f])) / max(np.max(np.abs(b[f])), 1e-300) for f in range(b.shape[0]))


def gpu_run(F, prob, fields, nsteps, precision="f64", chunks=None):
    import torch
    dt = torch.float64 if precision == "f64" else torch.float32
    plan = F.Plan(prob, precision)
    plan.set_fields(torch.tensor(np.ascontiguousarray(fields), dtype=dt, device="cuda"))
    for n in (chunks or [nsteps]):
        plan.step(n)
    out = plan.get_fields().double().cpu().numpy()
    plan.close()
    return out


def config1():
    pr = I.Problem(n=(64, 64), p=1)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    return pr


def test_config1_fp64_one_and_200_steps(F, O):
    pr = config1()
    f0 = I.noise_fields(pr, seed=0)
    ref1, _ = O.step(pr, f0, 1)
    assert rel_linf(gpu_run(F, pr, f0, 1), ref1) <= 1e-12
    ref200, _ = O.step(pr, f0, 200)
    got = gpu_run(F, pr, f0, 200)
    assert rel_linf(got, ref200) <= 1e-8


@pytest.mark.parametrize("n,p,lap,dx", [
    ((8, 8), 1, 0, (1.0, 1.0)),
    ((16, 128), 2, 0, (1.0, 1.0)),
    ((128, 16), 2, 1, (0.5, 2.0)),
    ((256, 32), 0, 0, (1.0, 1.0)),
    ((32, 256), 3, 2, (0.7, 1.3)),
    ((64, 512), 4, 0, (1.0, 1.0)),
    ((1024, 8), 1, 0, (1.0, 1.0)),
    ((8, 1024), 2, 0, (1.0, 1.0)),
])
def test_fp64_one_step_shapes(F, O, n, p, lap, dx):
    pr = I.Problem(n=n, dx=dx, p=p, lap=lap)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=3, amp=0.05)
    ref, _ = O.step(pr, f0, 1)
    assert rel_linf(gpu_run(F, pr, f0, 1), ref) <= 1e-12
    ref5, _ = O.step(pr, f0, 5)
    assert rel_linf(gpu_run(F, pr, f0, 5), ref5) <= 1e-11


def test_fp64_1024_square_p2(F, O):
    pr = I.Problem(n=(1024, 1024), p=2)
    pr.dt = 6.0 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=0)
    ref, _ = O.step(pr, f0, 1)
    assert rel_linf(gpu_run(F, pr, f0, 1), ref) <= 1e-12


@pytest.mark.parametrize("n,p", [((64, 64), 1), ((256, 128), 2), ((1024, 1024), 2)])
def test_fp32_one_step(F, O, n, p):
    pr = I.Problem(n=n, p=p)
    pr.dt = 6.0 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=1)
    ref, _ = O.step(pr, f0, 1)
    err = rel_linf(gpu_run(F, pr, f0.astype(np.float32), 1, "f32"), ref)
    assert err <= 2e-6, err


@pytest.mark.parametrize("n,p", [((1024, 64), 2), ((1024, 16, 16), 1)])
def test_fp32_1024_rows_several_steps(F, O, n, p):
    """FP32 rows of 1024 run the x-pass variant with 32 values per thread;
    several steps exercise its steady state (carried spectra) and the final
    inverse pass, against the FP64 oracle."""
    pr = I.Problem(n=n, p=p)
    pr.dt = 6.0 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=3)
    ref, _ = O.step(pr, f0, 10)
    err = rel_linf(gpu_run(F, pr, f0.astype(np.float32), 10, "f32"), ref)
    assert err <= 1e-5, err


def test_fp32_mean_carried_in_fp64(F):
    """FP32 plans carry sum(c) in FP64: mean(c) stays at its initial value to
    FP32 rounding of one inverse transform, with no drift over 500 steps."""
    pr = I.Problem(n=(256, 256), p=2)
    pr.dt = 6.0 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=2).astype(np.float32)
    m0 = f0[0].astype(np.float64).mean()
    got = gpu_run(F, pr, f0, 500, "f32")
    assert abs(got[0].mean() - m0) <= 2e-7


def test_graph_and_eager_paths_agree_bitwise(F):
    pr = config1()
    f0 = I.noise_fields(pr, seed=4)
    a = gpu_run(F, pr, f0, 70)
    b = gpu_run(F, pr, f0, 70, chunks=[1] * 70)
    assert np.array_equal(a, b)


def test_reading_fields_does_not_perturb_the_run(F):
    """fs_get_fields between steps leaves the carried spectra in place: a run
    with reads in between equals an uninterrupted one bit for bit."""
    import torch
    pr = I.Problem(n=(128, 64), p=2)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    f0 = torch.tensor(I.noise_fields(pr, seed=5), device="cuda")
    plan = F.Plan(pr, "f64")
    plan.set_fields(f0)
    plan.step(20)
    full = plan.get_fields().cpu().numpy()
    plan.set_fields(f0)
    plan.step(7)
    plan.get_fields()
    plan.step(13)
    assert np.array_equal(full, plan.get_fields().cpu().numpy())
    plan.close()


def test_checkpoint_resume(F):
    """Resuming in a new plan from the real fields recomputes c^ from c (the
    uninterrupted run carries c^, as Algorithm 1 does): equal to rounding."""
    import torch
    pr = I.Problem(n=(128, 64), p=2)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    f0 = torch.tensor(I.noise_fields(pr, seed=5), device="cuda")
    plan = F.Plan(pr, "f64")
    plan.set_fields(f0)
    plan.step(20)
    full = plan.get_fields().cpu().numpy()
    plan.set_fields(f0)
    plan.step(10)
    mid = plan.get_fields()
    plan2 = F.Plan(pr, "f64")
    plan2.set_fields(mid)
    plan2.step(10)
    resumed = plan2.get_fields().cpu().numpy()
    assert rel_linf(resumed, full) <= 1e-13


def test_host_pointers_round_trip(F, O):
    """Pointers may be host memory (cudaMemcpyDefault)."""
    pr = I.Problem(n=(32, 64), p=1)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    f0 = np.ascontiguousarray(I.noise_fields(pr, seed=6))
    plan = F.Plan(pr, "f64")
    F.fs_set_fields(plan.h, [f0[0], f0[1]])
    plan.step(3)
    out = np.empty_like(f0)
    F.fs_get_fields(plan.h, [out[0], out[1]])
    ref, _ = O.step(pr, f0, 3)
    assert rel_linf(out, ref) <= 1e-12


def test_nonfinite_input_reported(F):
    import torch
    pr = config1()
    f0 = I.noise_fields(pr, seed=0)
    f0[1, 3, 5] = np.nan
    plan = F.Plan(pr, "f64")
    plan.set_fields(torch.tensor(f0, device="cuda"))
    with pytest.raises(F.FSError) as ei:
        plan.step(2)
    assert ei.value.status == F.FS_ERR_NONFINITE
    # the flag is consumed: a clean state steps without error afterwards
    plan.set_fields(torch.tensor(I.noise_fields(pr, seed=0), device="cuda"))
    plan.step(2)


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("field,value", [(0, np.inf), (0, np.nan), (1, -np.inf), (2, np.inf), (2, np.nan)])
def test_nonfinite_in_any_field_reported_by_the_first_step(F, precision, field, value):
    """One non-finite value in c or in any eta_i is reported by the step that
    first reads it (p = 2, both precisions)."""
    import torch
    pr = I.Problem(n=(64, 32), p=2)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=2)
    f0[field, 7, 9] = value
    plan = F.Plan(pr, precision)
    plan.set_fields(torch.tensor(f0, dtype=torch.float64 if precision == "f64" else torch.float32, device="cuda"))
    with pytest.raises(F.FSError) as ei:
        plan.step(1)
    assert ei.value.status == F.FS_ERR_NONFINITE
    plan.close()


def test_step_before_set_is_a_state_error(F):
    plan = F.Plan(config1(), "f64")
    with pytest.raises(F.FSError) as ei:
        plan.step(1)
    assert ei.value.status == F.FS_ERR_STATE


def test_set_params_changes_dt(F, O):
    import torch
    pr = config1()
    f0 = I.noise_fields(pr, seed=0)
    plan = F.Plan(pr, "f64")
    plan.set_fields(torch.tensor(f0, device="cuda"))
    pr2 = pr.replace(dt=pr.dt / 2, M=4.0)
    plan.set_params(pr2)
    plan.step(40)
    ref, _ = O.step(pr2, f0, 40)
    assert rel_linf(plan.get_fields().cpu().numpy(), ref) <= 1e-11


@pytest.mark.parametrize("precision,n,p,tol", [("f64", (64, 64), 1, 1e-12), ("f64", (128, 32), 3, 1e-12),
                                               ("f32", (256, 256), 2, 1e-5)])
def test_free_energy_matches_oracle(F, O, precision, n, p, tol):
    """Eq. (fe) diagnostic: chemical and gradient parts against the oracle,
    before and after steps (spectral state materialised first)."""
    import torch
    pr = I.Problem(n=n, dx=(1.0, 0.5), p=p)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=14, amp=0.1)
    dt = torch.float64 if precision == "f64" else torch.float32
    plan = F.Plan(pr, precision)
    plan.set_fields(torch.tensor(f0, dtype=dt, device="cuda"))
    E0, parts0 = plan.free_energy()
    f_in = f0.astype(np.float32).astype(np.float64) if precision == "f32" else f0
    Fo, po = O.free_energy(pr, f_in, parts=True)
    assert abs(E0 - Fo) <= tol * abs(Fo)
    assert np.allclose(parts0, po, rtol=tol * 10, atol=tol * abs(Fo))
    plan.step(10)
    E1, _ = plan.free_energy()
    g = plan.get_fields().double().cpu().numpy()
    assert abs(E1 - O.free_energy(pr, g)) <= tol * abs(Fo)
    assert E1 < E0
    # the diagnostic leaves the state usable: stepping on gives the same as without it
    plan.step(5)
    h = plan.get_fields().double().cpu().numpy()
    plan.close()
    ref, _ = O.step(pr, g, 5)
    assert rel_linf(h, ref) <= (1e-12 if precision == "f64" else 2e-5)


@pytest.mark.parametrize("precision,n,dx,p,tol", [
    ("f64", (16, 32, 8), (1.0, 0.5, 2.0), 2, 1e-12), ("f64", (32, 16, 64), (0.7, 1.0, 1.3), 1, 1e-12),
    ("f64", (8, 8, 8), (1.0, 1.0, 1.0), 3, 1e-12), ("f32", (64, 64, 64), (1.0, 1.0, 1.0), 2, 1e-5)])
def test_free_energy_3d_matches_oracle(F, O, precision, n, dx, p, tol):
    """Eq. (fe) with the 3D frequency vector (Eq. Gamma_fft_3d): the x pass's
    chemical sum, then y and z transforms with the packed kx = 0 / Nyquist
    column weighted mode by mode; against the oracle before and after steps."""
    import torch
    pr = I.Problem(n=n, dx=dx, p=p)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=15, amp=0.1)
    dt = torch.float64 if precision == "f64" else torch.float32
    plan = F.Plan(pr, precision)
    plan.set_fields(torch.tensor(f0, dtype=dt, device="cuda"))
    E0, parts0 = plan.free_energy()
    f_in = f0.astype(np.float32).astype(np.float64) if precision == "f32" else f0
    Fo, po = O.free_energy(pr, f_in, parts=True)
    assert abs(E0 - Fo) <= tol * abs(Fo)
    assert np.allclose(parts0, po, rtol=tol * 10, atol=tol * abs(Fo))
    plan.step(6)
    E1, _ = plan.free_energy()
    g = plan.get_fields().double().cpu().numpy()
    assert abs(E1 - O.free_energy(pr, g)) <= tol * abs(Fo)
    assert E1 < E0
    plan.step(3)
    h = plan.get_fields().double().cpu().numpy()
    plan.close()
    ref, _ = O.step(pr, g, 3)
    assert rel_linf(h, ref) <= (1e-12 if precision == "f64" else 2e-5)
