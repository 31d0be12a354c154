"""The hand-written adjoint of the 2D and 3D steps: one step against the
oracle adjoint (and, in 3D, against central differences of the GPU's own
forward step), and trajectory gradients (autograd + checkpointing) against
central finite differences and the oracle."""
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


def gpu_adjoint(F, pr, u, lam, precision):
    import torch
    dt = torch.float64 if precision == "f64" else torch.float32
    plan = F.Plan(pr, precision)
    ut = torch.tensor(u, dtype=dt, device="cuda")
    lt = torch.tensor(lam, dtype=dt, device="cuda")
    out = torch.empty_like(lt)
    g = plan.step_adjoint(ut, lt, out)
    plan.close()
    return out.double().cpu().numpy(), np.array(g)


@pytest.mark.parametrize("n,p,lap,dx", [((32, 32), 1, 0, (1.0, 1.0)), ((64, 128), 2, 0, (1.0, 0.5)),
                                        ((128, 16), 3, 2, (1.0, 1.0)), ((16, 64), 0, 1, (0.5, 1.0))])
def test_adjoint_step_fp64_matches_oracle(F, O, n, p, lap, dx):
    pr = I.Problem(n=n, dx=dx, p=p, lap=lap)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    rng = np.random.default_rng(5)
    u = I.noise_fields(pr, seed=50, amp=0.3)
    lam = rng.standard_normal(u.shape)
    ref, gref = O.adjoint_step(pr, u, lam)
    got, g = gpu_adjoint(F, pr, u, lam, "f64")
    assert rel_linf(got, ref) <= 1e-11
    scale = np.max(np.abs(gref))
    assert np.max(np.abs(g - gref)) <= 1e-10 * scale


def test_adjoint_step_fp32_matches_oracle(F, O):
    pr = I.Problem(n=(256, 128), p=2)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    rng = np.random.default_rng(6)
    u = I.noise_fields(pr, seed=51, amp=0.3).astype(np.float32)
    lam = rng.standard_normal(u.shape).astype(np.float32)
    ref, gref = O.adjoint_step(pr, u.astype(np.float64), lam.astype(np.float64))
    got, g = gpu_adjoint(F, pr, u, lam, "f32")
    assert rel_linf(got, ref) <= 2e-5
    assert np.max(np.abs(g - gref)) <= 2e-4 * np.max(np.abs(gref))


@pytest.mark.parametrize("n,p,lap,dx", [((16, 16, 16), 1, 0, (1.0, 1.0, 1.0)), ((32, 16, 8), 2, 0, (1.0, 0.5, 1.0)),
                                        ((16, 32, 16), 2, 2, (1.0, 1.0, 0.5)), ((8, 16, 32), 0, 1, (0.5, 1.0, 1.0))])
def test_adjoint3_step_fp64_matches_oracle(F, O, n, p, lap, dx):
    """3D: x, y, z transforms of the adjoint with the packed kx = 0 / Nyquist
    column split into (kx, ky) modes, pair rows included."""
    pr = I.Problem(n=n, dx=dx, p=p, lap=lap)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    rng = np.random.default_rng(7)
    u = I.noise_fields(pr, seed=52, amp=0.3)
    lam = rng.standard_normal(u.shape)
    ref, gref = O.adjoint_step(pr, u, lam)
    got, g = gpu_adjoint(F, pr, u, lam, "f64")
    assert rel_linf(got, ref) <= 1e-11
    assert np.max(np.abs(g - gref)) <= 1e-10 * np.max(np.abs(gref))


def test_adjoint3_step_fp32_matches_oracle(F, O):
    pr = I.Problem(n=(64, 64, 64), p=2)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    rng = np.random.default_rng(8)
    u = I.noise_fields(pr, seed=53, amp=0.3).astype(np.float32)
    lam = rng.standard_normal(u.shape).astype(np.float32)
    ref, gref = O.adjoint_step(pr, u.astype(np.float64), lam.astype(np.float64))
    got, g = gpu_adjoint(F, pr, u, lam, "f32")
    assert rel_linf(got, ref) <= 2e-5
    assert np.max(np.abs(g - gref)) <= 2e-4 * np.max(np.abs(gref))


def test_adjoint3_is_the_transpose_of_the_gpu_step(F):
    """<lam, (S(u + h v) - S(u - h v)) / 2h> with the GPU's FP64 3D step equals
    <J^T lam, v> from the GPU adjoint: the adjoint transposes the forward
    kernels themselves, not only the oracle."""
    import torch
    pr = I.Problem(n=(32, 16, 16), p=2)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    rng = np.random.default_rng(9)
    u = I.noise_fields(pr, seed=54, amp=0.3)
    lam = rng.standard_normal(u.shape)
    v = rng.standard_normal(u.shape)

    def step(x):
        plan = F.Plan(pr, "f64")
        plan.set_fields(torch.tensor(x, device="cuda"))
        plan.step(1)
        out = plan.get_fields().cpu().numpy()
        plan.close()
        return out
    h = 1e-6
    fd = np.sum(lam * (step(u + h * v) - step(u - h * v))) / (2 * h)
    got, _ = gpu_adjoint(F, pr, u, lam, "f64")
    assert np.sum(got * v) == pytest.approx(fd, rel=1e-7)


def _loss(F, pr, theta, u0, target, precision, nsteps, every):
    import torch
    from paper_2306_04322_gb300 import adjoint as A
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    snaps = A.trajectory(th, u0, pr, precision, nsteps, every)
    loss = A.misfit_loss(snaps, target)
    return loss, th


def test_trajectory_gradient_matches_central_differences(F):
    """64^2, p = 2, 60 steps with a checkpoint every 20: the adjoint gradient of
    the snapshot misfit equals central differences (h = 1e-4 relative) of the
    FP64 loss to 1e-4 relative, and the FP32 adjoint stays close to FP64."""
    import torch
    pr = I.Problem(n=(64, 64), p=2)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    star = np.array([5.0, 5.0, 3.0, 3.0])
    u0 = torch.tensor(I.noise_fields(pr, seed=60), device="cuda")
    from paper_2306_04322_gb300 import adjoint as A
    with torch.no_grad():
        target = A.trajectory(torch.tensor(star), u0, pr, "f64", 60, 20)
    theta = 1.2 * star
    loss, th = _loss(F, pr, theta, u0, target, "f64", 60, 20)
    loss.backward()
    g = th.grad.numpy()
    for q in range(4):
        h = 1e-4 * theta[q]
        tp, tm = theta.copy(), theta.copy()
        tp[q] += h
        tm[q] -= h
        with torch.no_grad():
            lp = A.misfit_loss(A.trajectory(torch.tensor(tp), u0, pr, "f64", 60, 20), target).item()
            lm = A.misfit_loss(A.trajectory(torch.tensor(tm), u0, pr, "f64", 60, 20), target).item()
        fd = (lp - lm) / (2 * h)
        assert abs(g[q] - fd) <= 1e-4 * max(abs(fd), 1e-12), (q, g[q], fd)
    loss32, th32 = _loss(F, pr, theta, u0.float(), target, "f32", 60, 20)
    loss32.backward()
    g32 = th32.grad.numpy()
    assert np.max(np.abs(g32 - g)) <= 1e-2 * np.max(np.abs(g))


def test_trajectory_gradient_matches_oracle_adjoint(F, O):
    """The GPU trajectory gradient equals the oracle's: oracle forward states,
    oracle adjoint steps backwards through the same loss."""
    import torch
    pr = I.Problem(n=(32, 32), p=1)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    u0 = I.noise_fields(pr, seed=61)
    star = np.array([5.0, 5.0, 3.0, 3.0])
    nsteps, every = 20, 5
    # target from the oracle with theta*
    tgt, u = [], u0.copy()
    for s in range(nsteps // every):
        u, _ = O.step(pr, u, every)
        tgt.append(u)
    target = torch.tensor(np.stack(tgt), device="cuda")
    theta = 1.2 * star
    loss, th = _loss(F, pr, theta, torch.tensor(u0, device="cuda"), target, "f64", nsteps, every)
    loss.backward()
    # oracle: forward states and adjoint
    prt = pr.replace(M=theta[0], L=theta[1], kappa_c=theta[2], kappa_eta=theta[3])
    states = [u0.copy()]
    for _ in range(nsteps):
        nxt, _ = O.step(prt, states[-1], 1)
        states.append(nxt)
    N = pr.npoints
    lam = np.zeros_like(u0)
    gsum = np.zeros(4)
    for n in range(nsteps, 0, -1):
        if n % every == 0:
            lam = lam + 2.0 * (states[n] - tgt[n // every - 1]) / N
        lam, g = O.adjoint_step(prt, states[n - 1], lam)
        gsum += g
    assert np.max(np.abs(th.grad.numpy() - gsum)) <= 1e-9 * np.max(np.abs(gsum))


def test_adjoint3_under_the_bounds_checked_build(F, O):
    """Every checked access of the 3D adjoint's five launches stays inside
    its buffer (FS_DEBUG_BOUNDS build); results still match the oracle."""
    from paper_2306_04322_gb300 import build as B
    pr = I.Problem(n=(16, 8, 8), p=1)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    rng = np.random.default_rng(10)
    u = I.noise_fields(pr, seed=55, amp=0.3)
    lam = rng.standard_normal(u.shape)
    ref, gref = O.adjoint_step(pr, u, lam)
    L = F.bind(B.build(variant="bounds"))
    saved = F._lib
    F._lib = L
    try:
        got, g = gpu_adjoint(F, pr, u, lam, "f64")
    finally:
        F._lib = saved
    assert rel_linf(got, ref) <= 1e-11
    assert np.max(np.abs(g - gref)) <= 1e-10 * np.max(np.abs(gref))
