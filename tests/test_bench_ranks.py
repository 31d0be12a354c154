"""The multi-rank path of bench.py on CPU: every rank runs an independent
replica (the step has no exchange between simulations), the job time is the
slowest rank's, the job value counts every rank's points; the reference arm
prints only on rank 0.  world_size 2, gloo backend, 127.0.0.1."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out_path):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.reduce_max(times[rank], dist, "cpu")
    v = bench.job_value(world, 1024 * 1024, 50, t)
    if rank == 0:
        with open(out_path, "w") as f:
            json.dump({"t": t, "v": v}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_slowest_rank_sets_the_job_time(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    times = [0.8, 1.3]
    out = str(tmp_path / "r.json")
    mp.start_processes(_rank_main, args=(2, _free_port(), times, out), nprocs=2, start_method="spawn")
    r = json.load(open(out))
    assert r["t"] == 1.3
    assert r["v"] == pytest.approx(2 * 1024 * 1024 * 50 / 1.3)


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(2.5, None) == 2.5
    assert bench.job_value(1, 100, 10, 2.0) == 500.0


def test_reference_arm_prints_on_rank_zero_only():
    """Rank 1 of a torchrun launch of the reference arm exits 0 without work
    or output."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "3", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
