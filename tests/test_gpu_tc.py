"""The FP32 tensor-core DFT-stage variants (first radix-16 pass of the forward
column transforms as a split TF32 x 3 or BF16 x 3 GEMM on tensor cores)
against the FP64 oracle, 2D and 3D.

Tolerances (relative L-inf after one step): TF32 x 3 keeps about 21
significant bits per product, like the CUDA-core FP32 path (2e-6 there);
BF16 x 3 keeps about 16 bits: 5e-5."""
import numpy as np
import pytest

from paper_2306_04322_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"tf32": 4e-6, "bf16x3": 5e-5}


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


def gpu_run(F, prob, fields, nsteps, precision):
    import torch
    plan = F.Plan(prob, precision)
    plan.set_fields(torch.tensor(np.ascontiguousarray(fields), dtype=torch.float32, device="cuda"))
    plan.step(nsteps)
    out = plan.get_fields().double().cpu().numpy()
    plan.close()
    return out


@pytest.mark.parametrize("precision", ["tf32", "bf16x3"])
@pytest.mark.parametrize("n,p", [((128, 128), 2), ((64, 1024), 1), ((1024, 256), 2), ((64, 64, 64), 2),
                                 ((128, 64, 256), 1)])
def test_tc_variant_matches_oracle(F, O, precision, n, p):
    pr = I.Problem(n=n, p=p)
    pr.dt = 6.0 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=80).astype(np.float32)
    ref, _ = O.step(pr, f0.astype(np.float64), 1)
    got = gpu_run(F, pr, f0, 1, precision)
    err = rel_linf(got, ref)
    assert err <= TOL[precision], err


@pytest.mark.parametrize("precision", ["tf32", "bf16x3"])
def test_tc_variant_2d_several_steps(F, O, precision):
    """2D steady state (spectra carried from step to step, every forward
    column transform through the tensor-core stage), ten steps against the
    oracle."""
    pr = I.Problem(n=(256, 128), p=2)
    pr.dt = 6.0 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=81).astype(np.float32)
    ref, _ = O.step(pr, f0.astype(np.float64), 10)
    assert rel_linf(gpu_run(F, pr, f0, 10, precision), ref) <= 10 * TOL[precision]


@pytest.mark.parametrize("precision", ["tf32", "bf16x3"])
def test_tc_variant_256_cube_and_mean(F, O, precision):
    pr = I.Problem(n=(256, 256, 256), p=2)
    pr.dt = 6.0 * I.fd_stable_dt(pr)
    f0 = I.noise_fields(pr, seed=0).astype(np.float32)
    ref, _ = O.step(pr, f0.astype(np.float64), 1)
    got = gpu_run(F, pr, f0, 1, precision)
    assert rel_linf(got, ref) <= TOL[precision]
    got20 = gpu_run(F, pr, f0, 20, precision)
    assert abs(got20[0].mean() - f0[0].astype(np.float64).mean()) <= 2e-7


def test_tc_rejects_small_axes(F):
    with pytest.raises(F.FSError) as ei:
        F.Plan(I.Problem(n=(32, 128), p=1, dt=1e-3), "tf32")
    assert ei.value.status == F.FS_ERR_UNSUPPORTED
