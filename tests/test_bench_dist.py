"""The multi-rank path of bench.py on CPU (gloo, world size 2): every rank
solves its own replica, the timed region is the maximum over ranks and the
units are summed; --impl reference runs on rank 0 only."""
import os
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    res = bench.aggregate(100.0 + 50.0 * rank, 1000.0 * (rank + 1), dist)
    out[rank] = res
    dist.destroy_process_group()


def test_aggregate_max_time_and_summed_units():
    port = 29500 + os.getpid() % 1000
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn")
    for r in (0, 1):
        assert out[r]["max_ms"] == 150.0
        assert out[r]["units"] == 3000.0
        assert out[r]["world"] == 2
        assert abs(out[r]["per_s"] - 3000.0 / 0.150) < 1e-6


def test_aggregate_single_rank():
    import bench
    r = bench.aggregate(250.0, 500.0)
    assert r["world"] == 1 and r["max_ms"] == 250.0 and abs(r["per_s"] - 2000.0) < 1e-9


def test_reference_arm_under_torchrun_runs_on_rank0_only():
    env = dict(os.environ)
    port = str(29600 + os.getpid() % 1000)
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", port, "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--workload", "tsp20",
           "--ref-generations", "3"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=240)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    import json
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["cpu_baseline"]["kind"] == "oracle"
