"""The slab decomposition (include/fs_slab.h) on one GPU against the oracle.

R ranks of one grid are held by one process (paper_2306_04322_gb300.slab's
LocalSlabs): every rank's row pass, the forward transpose as device copies,
every rank's column pass, the back transpose.  No kernel waits on another
rank, so this is safe on one GPU; the NCCL transport between processes is
the same block moves (its host logic is checked over gloo on CPU).

Tolerances (relative L-inf per field): FP64 1e-12 after one step and 1e-11
after several (Algorithm 1 in the same arithmetic as the single plans); FP32
the parity bound of the other FP32 tests, 2e-6 per step times 2.
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


def tol(precision, k):
    if precision == "f64":
        return 1e-12 if k == 1 else 1e-11
    return 2e-6 * k * 2.0


def run_local(pr, precision, R, f0, chunks):
    import torch
    from paper_2306_04322_gb300 import slab as S
    dt = torch.float64 if precision == "f64" else torch.float32
    L = S.LocalSlabs(pr, precision, R)
    L.set_fields(torch.tensor(f0, dtype=dt, device="cuda"))
    outs = []
    for n in chunks:
        L.step(n)
        outs.append(L.get_fields().double().cpu().numpy())
    L.sync()
    L.close()
    return outs


@pytest.mark.parametrize("n,p,precision,R", [
    ((64, 128), 1, "f64", 2), ((128, 64), 4, "f64", 8), ((256, 256), 2, "f32", 2), ((128, 256), 3, "f32", 4),
    ((512, 128), 0, "f32", 4), ((64, 64), 2, "f64", 1), ((256, 64), 2, "f64", 4)])
def test_local_slabs_match_the_oracle(F, O, n, p, precision, R):
    pr = I.Problem(n=n, p=p)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=41)
    r1, _ = O.step(pr, f0, 1)
    r4, _ = O.step(pr, r1, 3)
    g1, g4 = run_local(pr, precision, R, f0, [1, 3])
    assert rel_linf(g1, r1) <= tol(precision, 1)
    assert rel_linf(g4, r4) <= tol(precision, 4)


@pytest.mark.parametrize("lap", [1, 2])
def test_local_slabs_fs_fd_laplacians(F, O, lap):
    """The FS-FD |xi|^2 forms take the global kx of each rank's columns."""
    pr = I.Problem(n=(128, 64), p=2, lap=lap)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=42)
    ref, _ = O.step(pr, f0, 3)
    (g,) = run_local(pr, "f64", 4, f0, [3])
    assert rel_linf(g, ref) <= tol("f64", 3)


def test_local_slabs_headline_grid(F, O):
    """1024^2 with c and two eta (FP32) over 4 slabs: the warp-per-line
    forms run on each rank's 1024 x 256 rows and 256 x 1024 columns."""
    pr = I.Problem(n=(1024, 1024), p=2)
    pr.dt = 6.0 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=0)
    ref, _ = O.step(pr, f0, 6)
    (g,) = run_local(pr, "f32", 4, f0, [6])
    assert rel_linf(g, ref) <= tol("f32", 6)


def test_slab_equals_plan_bitwise_in_fp64_on_one_rank(F):
    """R = 1: the slab's row and column plans are the single plan's passes,
    and the transposes are pure copies -- the same numbers bit for bit."""
    import torch
    pr = I.Problem(n=(128, 128), p=2)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    f0 = torch.tensor(I.noise_fields(pr, seed=43), device="cuda")
    plan = F.Plan(pr, "f64")
    plan.set_fields(f0)
    plan.step(4)
    ref = plan.get_fields().cpu().numpy()
    plan.close()
    (g,) = run_local(pr, "f64", 1, f0.cpu().numpy(), [4])
    assert np.array_equal(g, ref)


def test_slab_state_and_argument_errors(F):
    import torch
    from paper_2306_04322_gb300 import slab as S
    pr = I.Problem(n=(64, 64), p=1, dt=1e-3)
    s = S.Slab(pr, "f32", 0, 2)
    with pytest.raises(F.FSError) as ei:
        s.row_pass()
    assert ei.value.status == F.FS_ERR_STATE
    s.set_fields(torch.zeros((2, 32, 64), dtype=torch.float32, device="cuda"))
    s.row_pass()
    with pytest.raises(F.FSError) as ei:
        s.col_pass()  # FP32 needs the global c sum first
    assert ei.value.status == F.FS_ERR_STATE
    s.close()
    P = F.make_params(pr, "f32")
    for args, status in [((0, 3), F.FS_ERR_UNSUPPORTED), ((2, 2), F.FS_ERR_INVALID_ARG),
                         ((0, 16), F.FS_ERR_UNSUPPORTED)]:
        with pytest.raises(F.FSError) as ei:
            F.fs_slab_create(P, *args)
        assert ei.value.status == status
    with pytest.raises(F.FSError) as ei:
        F.fs_slab_create(F.make_params(pr, "tf32"), 0, 2)
    assert ei.value.status == F.FS_ERR_UNSUPPORTED


def test_distributed_slab_over_nccl_on_one_rank(F, O):
    """The process-group driver end to end with one NCCL rank: the global c
    sum goes through all_reduce, the transposes have no peer."""
    import torch
    import torch.distributed as dist
    from paper_2306_04322_gb300 import slab as S
    import socket
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    pr = I.Problem(n=(256, 128), p=2)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=44)
    ref, _ = O.step(pr, f0, 3)
    torch.cuda.set_device(0)
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        d = S.DistributedSlab(pr, "f32")
        d.set_fields(torch.tensor(f0, dtype=torch.float32, device="cuda"))
        d.step(3)
        g = d.get_fields().double().cpu().numpy()
        d.sync()
        d.close()
    finally:
        dist.destroy_process_group()
    assert rel_linf(g, ref) <= tol("f32", 3)


@contextlib.contextmanager
def bounds_library(F):
    from paper_2306_04322_gb300 import build as B
    L = F.bind(B.build(variant="bounds"))
    saved = F._lib
    F._lib = L
    try:
        yield L
    finally:
        F._lib = saved


@pytest.mark.parametrize("n,p,precision,R", [((64, 32), 2, "f64", 2), ((256, 256), 1, "f32", 4)])
def test_slabs_under_the_bounds_checked_build(F, O, n, p, precision, R):
    """Every checked access of the column plans (their nx covers only a
    rank's columns) stays inside its buffer."""
    pr = I.Problem(n=n, p=p)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=45)
    with bounds_library(F):
        (g,) = run_local(pr, precision, R, f0, [3])
    ref, _ = O.step(pr, f0, 3)
    assert rel_linf(g, ref) <= tol(precision, 3)
