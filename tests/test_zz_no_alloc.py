"""The allocation-free entry point fs_step2d_static, for callers that cannot
allocate device memory (for example inside a capture or an embedding that owns
all device memory): it must give the same fields as a plan, call after call,
although every call reuses one fixed device scratch array.  Collected last so
that a run stopping at the first failure has run everything else first."""
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


@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 1e-6)])
def test_static_step_matches_plan_on_two_calls(F, precision, tol):
    import torch
    dt = torch.float64 if precision == "f64" else torch.float32
    probs = [I.Problem(n=(128, 64), p=2), I.Problem(n=(64, 256), p=1)]
    for call, pr in enumerate(probs):
        pr.dt = 5.0 * I.fd_stable_dt(pr)
        f0 = torch.tensor(I.noise_fields(pr, seed=70 + call), dtype=dt, device="cuda")
        plan = F.Plan(pr, precision)
        plan.set_fields(f0)
        plan.step(7)
        ref = plan.get_fields().double().cpu().numpy()
        plan.close()
        buf = f0.clone().contiguous()
        status = F.fs_step2d_static(F.make_params(pr, precision), buf, 7)
        torch.cuda.synchronize()
        assert status == F.FS_OK
        assert rel_linf(buf.double().cpu().numpy(), ref) <= tol


def test_static_step_rejects_sizes_beyond_the_limit(F):
    pr = I.Problem(n=(512, 256), p=2, dt=1e-3)
    import torch
    buf = torch.zeros((3, 256, 512), dtype=torch.float32, device="cuda")
    assert F.fs_step2d_static(F.make_params(pr, "f32"), buf, 1) == F.FS_ERR_UNSUPPORTED
    pr = I.Problem(n=(64, 64), p=3, dt=1e-3)
    buf = torch.zeros((4, 64, 64), dtype=torch.float32, device="cuda")
    assert F.fs_step2d_static(F.make_params(pr, "f32"), buf, 1) == F.FS_ERR_UNSUPPORTED
