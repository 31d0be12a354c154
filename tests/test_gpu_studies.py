"""The configuration-level studies at small sizes: they run end to end on the
GPU and their results have the structure the method implies (FP32 close to
FP64, the spectral FS Laplacian the most accurate, finite costs)."""
import math

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def X():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_04322_gb300 import build as B
    from paper_2306_04322_gb300 import experiments
    B.build()
    return experiments


def test_precision_study_small(X):
    r = X.precision_study(40, n=64)
    assert max(r["f32"]["rel_linf_vs_f64"]) < 1e-3
    assert max(r["tf32"]["rel_linf_vs_f64"]) < 1e-2
    assert max(r["bf16x3"]["rel_linf_vs_f64"]) < 5e-2
    assert r["f64"]["ms_per_step"] > 0


def test_accuracy_study_small(X):
    r = X.accuracy_study(50, n=128)
    for k in ("FS_f64", "FS_f32", "FSFD2_f64", "FSFD4_f64", "FD_f64"):
        assert math.isfinite(r[k]["E_c"]) and math.isfinite(r[k]["E_eta"])
    # same dt and grid: the spectral Laplacian beats the O(dl^4) one, which beats O(dl^2)
    assert r["FS_f64"]["E_eta"] < r["FSFD4_f64"]["E_eta"] < r["FSFD2_f64"]["E_eta"]


def test_cost_study_small(X):
    r = X.cost_study(20, grids=[(64, 64), (16, 16, 16)])
    assert len(r["rows"]) == 4
    for row in r["rows"]:
        assert row["fs_ms_per_step"] > 0 and row["fd_ms_per_step"] > 0
