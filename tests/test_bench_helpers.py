"""bench.py's roofline arithmetic on made-up timings (no GPU)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_step_entry_fractions():
    e = bench.step_entry(alg_bytes=54_525_952, comp_bytes=25_165_824, ms=0.05, peak=6790.0)
    assert e["algorithmic_GBps"] == pytest.approx(54_525_952 / 5e-5 / 1e9)
    assert e["compulsory_GBps"] == pytest.approx(25_165_824 / 5e-5 / 1e9)
    assert e["frac_algorithmic"] == pytest.approx(e["algorithmic_GBps"] / 6790.0)
    assert e["frac_compulsory"] < e["frac_algorithmic"]


def test_roofline_entry_picks_the_dominant_kernel():
    r = {"kern_ms": [2.0, 3.0], "kern_cnt": [10, 10]}
    e = bench.roofline_entry(["a", "b"], [1e8, 1e8], r, 6790.0, "measured")
    assert e["kernel"] == "b" and e["avg_launch_ms"] == pytest.approx(0.3)
    assert e["achieved"] == pytest.approx(1e8 / 3e-4 / 1e9)
    assert e["frac"] == pytest.approx(e["achieved"] / 6790.0)
    assert e["kernels"]["a"]["share"] == pytest.approx(0.4)


def test_traffic_table_lookup():
    assert bench.dram_traffic("fs_row_kernel", "f32") > 0
    assert bench.dram_traffic("fs_zstep_kernel", "f32", "traffic_3d_256_p2.txt") > 0
    assert bench.dram_traffic("no_such_kernel", "f32") is None
