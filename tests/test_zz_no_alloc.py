"""The allocation-free entry point fs_step2d_static.  It serves callers that
cannot allocate device memory (a host program whose own pool allocator owns
all device memory, or code on a real-time / signal path where cudaMalloc is
not allowed): it must give the same fields as a plan, call after call,
although every call reuses one fixed device scratch array, and it must
allocate nothing.  Collected last so that a run stopping at the first
failure has run everything else first."""
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


def plan_fields(F, pr, precision, f0, nsteps):
    plan = F.Plan(pr, precision)
    plan.set_fields(f0)
    plan.step(nsteps)
    ref = plan.get_fields().double().cpu().numpy()
    plan.close()
    return ref


# FP64 agrees with a plan to rounding.  FP32 plans run other kernel forms
# for rows and columns of 256 to 1024 points than this entry point (which
# keeps the half-length rows and column tiles), so the two differ by FP32
# rounding: the parity bound of the FP32 tests, 2e-6 per step and field
# (relative L-inf), times the number of steps, times 2 for growth.
def tol(precision, steps):
    return 1e-12 if precision == "f64" else 2e-6 * steps * 2.0


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_static_step_matches_plan_on_two_calls(F, precision):
    import torch
    dt = torch.float64 if precision == "f64" else torch.float32
    probs = [I.Problem(n=(128, 64), p=2), I.Problem(n=(64, 256), p=1)]
    for call, pr in enumerate(probs):
        pr.dt = 5.0 * I.fd_stable_dt(pr)
        f0 = torch.tensor(I.noise_fields(pr, seed=70 + call), dtype=dt, device="cuda")
        ref = plan_fields(F, pr, precision, f0, 7)
        buf = f0.clone().contiguous()
        status = F.fs_step2d_static(F.make_params(pr, precision), buf, 7)
        torch.cuda.synchronize()
        assert status == F.FS_OK
        assert rel_linf(buf.double().cpu().numpy(), ref) <= tol(precision, 7)


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("n,lap", [((1024, 64), 0), ((64, 1024), 0), ((256, 256), 2)])
def test_static_step_at_the_size_limit(F, precision, n, lap):
    """65536 points with p = 2 fill the scratch; 1024-point rows and columns
    and the FS-FD O(dl^4) Laplacian; two calls in a row."""
    import torch
    dt = torch.float64 if precision == "f64" else torch.float32
    pr = I.Problem(n=n, p=2, lap=lap)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    for call in range(2):
        f0 = torch.tensor(I.noise_fields(pr, seed=80 + call), dtype=dt, device="cuda")
        ref = plan_fields(F, pr, precision, f0, 4)
        buf = f0.clone().contiguous()
        assert F.fs_step2d_static(F.make_params(pr, precision), buf, 4) == F.FS_OK
        assert rel_linf(buf.double().cpu().numpy(), ref) <= tol(precision, 4)


def test_static_step_allocates_no_device_memory(F):
    import torch
    pr = I.Problem(n=(256, 256), p=2)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    buf = torch.tensor(I.noise_fields(pr, seed=90), dtype=torch.float32, device="cuda")
    prm = F.make_params(pr, "f32")
    # the first call loads the kernels it uses (the driver's code memory)
    assert F.fs_step2d_static(prm, buf, 2) == F.FS_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert F.fs_step2d_static(prm, buf, 3) == F.FS_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_step_rejects_sizes_beyond_the_limit(F):
    import torch
    pr = I.Problem(n=(512, 256), p=2, dt=1e-3)
    buf = torch.zeros((3, 256, 512), dtype=torch.float32, device="cuda")
    assert F.fs_step2d_static(F.make_params(pr, "f32"), buf, 1) == F.FS_ERR_UNSUPPORTED
    for p in (3, 4):
        pr = I.Problem(n=(64, 64), p=p, dt=1e-3)
        buf = torch.zeros((p + 1, 64, 64), dtype=torch.float32, device="cuda")
        assert F.fs_step2d_static(F.make_params(pr, "f32"), buf, 1) == F.FS_ERR_UNSUPPORTED
    pr = I.Problem(n=(64, 64), p=1, dt=1e-3)
    buf = torch.zeros((2, 64, 64), dtype=torch.float32, device="cuda")
    for prec in ("tf32", "bf16x3"):
        assert F.fs_step2d_static(F.make_params(pr, prec), buf, 1) == F.FS_ERR_UNSUPPORTED
    assert F.fs_step2d_static(F.make_params(pr, "f32", scheme=F.FS_SCHEME_EXPLICIT_FD), buf, 1) == \
        F.FS_ERR_UNSUPPORTED
    p3 = I.Problem(n=(16, 16, 16), p=1, dt=1e-3)
    b3 = torch.zeros((2, 16, 16, 16), dtype=torch.float32, device="cuda")
    assert F.fs_step2d_static(F.make_params(p3, "f32"), b3, 1) == F.FS_ERR_UNSUPPORTED


def test_static_step_rejects_malformed_arguments_on_the_host(F):
    """A misaligned field array (a view with an odd storage offset), a
    negative step count and p out of range are refused before any kernel
    runs: the fields are left untouched."""
    import torch
    pr = I.Problem(n=(64, 64), p=1)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    base = torch.tensor(I.noise_fields(pr, seed=91), dtype=torch.float32, device="cuda").view(-1)
    store = torch.empty(base.numel() + 1, dtype=torch.float32, device="cuda")
    view = store[1:]
    view.copy_(base)
    before = view.clone()
    assert view.data_ptr() % 16 != 0
    assert F.fs_step2d_static(F.make_params(pr, "f32"), view, 3) == F.FS_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert torch.equal(view, before)
    assert F.fs_step2d_static(F.make_params(pr, "f32"), store, -1) == F.FS_ERR_INVALID_ARG
    bad = F.make_params(pr, "f32")
    bad.p = 5
    assert F.fs_step2d_static(bad, store, 1) == F.FS_ERR_INVALID_ARG
    bad = F.make_params(pr, "f32")
    bad.dt = 0.0
    assert F.fs_step2d_static(bad, store, 1) == F.FS_ERR_INVALID_ARG


def test_static_step_refuses_a_capturing_stream(F):
    """The call synchronises its stream, which a stream capture cannot
    record: it returns FS_ERR_UNSUPPORTED and enqueues nothing."""
    import torch
    pr = I.Problem(n=(64, 64), p=1)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    buf = torch.tensor(I.noise_fields(pr, seed=92), dtype=torch.float32, device="cuda")
    prm = F.make_params(pr, "f32")
    assert F.fs_step2d_static(prm, buf, 1) == F.FS_OK  # first call: set-up outside the capture
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    statuses = []
    with torch.cuda.graph(g, stream=side):
        statuses.append(F.fs_step2d_static(prm, buf, 1, stream=side.cuda_stream))
    assert statuses == [F.FS_ERR_UNSUPPORTED]
