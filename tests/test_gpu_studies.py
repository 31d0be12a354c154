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


def test_table1_study_small(X):
    """The Table 1 study on small grids: the reference case is the reference
    run (E = 0), the time error grows with dt on the finest grid, FP32 stays
    close to FP64 over a short window, and every case (FS variants, explicit
    FD) yields finite errors."""
    from paper_2306_04322_gb300 import inputs as I
    fd = {n: 0.9 * I.fd_stable_dt(I.Problem(n=(n, n), dx=(200.0 / n,) * 2, p=4)) for n in (32, 64)}
    r = X.table1_study(t_span=0.05, grids=(32, 64), dts=(2.5e-4, 1e-3, 5e-3), ref_dt=2.5e-4, pre_n=256,
                       fd_dts=fd)
    rows = r["rows"]
    assert len(rows) == 2 * 3 * 3 + 2
    for row in rows:
        assert math.isfinite(row["E_c"]) and math.isfinite(row["E_eta"]) and row["E_c"] >= 0
    fs64 = {row["dt"]: row for row in rows if row["grid"] == 64 and row["scheme"] == "FS"}
    assert fs64[2.5e-4]["E_c"] == 0.0 and fs64[2.5e-4]["E_eta"] == 0.0
    assert fs64[1e-3]["E_eta"] < fs64[5e-3]["E_eta"]
    assert r["f32_floor"]["E_c"] < 1e-9 and r["f32_floor"]["E_eta"] < 1e-9
    assert {row["scheme"] for row in rows} == {"FS", "FSFD2", "FSFD4", "FD"}


def test_table2_study_small(X):
    """The Table 2 study on small cubes: every case yields finite errors and
    timings, the FS time error grows with dt on the finest grid, and the
    coarse grid's FS error is above the fine grid's."""
    from paper_2306_04322_gb300 import inputs as I
    fd = {n: 0.9 * I.fd_stable_dt(I.Problem(n=(n, n, n), dx=(100.0 / n,) * 3, p=4)) for n in (16, 32)}
    r = X.table2_study(t_span=0.05, grids=(16, 32), fs_dt=5e-3, ref_dt=1e-3, pre_n=128, fd_dts=fd)
    rows = r["rows"]
    assert len(rows) == 2 * 3 + 2
    for row in rows:
        assert "unstable" not in row, row
        assert math.isfinite(row["E_c"]) and math.isfinite(row["E_eta"]) and row["ms"] > 0
    fs = {row["grid"]: row for row in rows if row["scheme"] == "FS"}
    assert fs[16]["E_eta"] > fs[32]["E_eta"] > 0.0
    assert {row["scheme"] for row in rows} == {"FS", "FSFD2", "FSFD4", "FD"}


def test_slab_study_small(X):
    """The slab timing study on a small grid: per-rank times are positive and
    the exchange bytes follow the layout."""
    r = X.slab_study(steps=3, grids=(64,), ranks=(1, 2))
    rows = r["rows"]
    assert [row["ranks"] for row in rows] == [1, 2]
    for row in rows:
        assert row["row_ms_per_rank"] > 0 and row["col_ms_per_rank"] > 0 and row["plan_step_ms"] > 0
    assert rows[0]["exchange_bytes_per_rank"] == 0
    # R = 2, p = 2: (2 nf + 1) (R - 1) N s / R^2 = 7 * 64 * 64 * 4 / 4
    assert rows[1]["exchange_bytes_per_rank"] == 7 * 64 * 64 * 4 // 4
