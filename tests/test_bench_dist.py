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


# ------------------------------------------------------ bench option helpers
def test_extra_operator_masks_per_model():
    import bench
    import instances as I
    assert bench.extra_ops_mask(I.TSP, "three_opt,segment") == 1 << bench.O_THREE_OPT
    assert bench.extra_ops_mask(I.CVRPTW, "three_opt") == 1 << bench.O_THREE_OPT
    assert bench.extra_ops_mask(I.QAP, "three_opt") == 1 << bench.O_THREE_OPT
    assert bench.extra_ops_mask(I.KNAPSACK, "segment,three_opt") == 1 << bench.O_SEGMENT
    assert bench.extra_ops_mask(I.GAP, "segment") == 1 << bench.O_SEGMENT
    assert bench.extra_ops_mask(I.TSP, "") == 0
    assert bench.extra_ops_mask(I.CVRPTW, "rows") == 0x700       # row_swap, row_merge, row_split
    assert bench.extra_ops_mask(I.TSP, "rows") == 0
    with pytest.raises(SystemExit):
        bench.extra_ops_mask(I.TSP, "two_and_a_half_opt")


def test_solve_variant_applies_to_both_arms():
    import argparse
    import bench
    import instances as I
    args = argparse.Namespace(init_oversample=4, init_heuristic=1, islands="4,1000,2,3",
                              extra_ops="three_opt", cross=6554)
    cfg, desc = bench.solve_variant(args, I.TSP, dict(P=128, C=128, G=10), "w")
    assert cfg["init_oversample"] == 4 and cfg["init_heuristic"] == 1
    assert (cfg["islands"], cfg["migrate_period"], cfg["migrate_strategy"], cfg["migrate_n"]) == (4, 1000, 2, 3)
    assert cfg["extra_mask"] == 1 << bench.O_THREE_OPT and cfg["cross_q16"] == 6554
    assert "islands=4" in desc and "hybrid-3" in desc and "cross=0.100" in desc
    none = argparse.Namespace(init_oversample=1, init_heuristic=0, islands="", extra_ops="", cross=0)
    cfg2, desc2 = bench.solve_variant(none, I.TSP, dict(P=1), "w")
    assert cfg2 == dict(P=1) and desc2 == "w"


def test_cvrptw_objectives_of_a_separator_sequence():
    import numpy as np
    import bench
    # depot 0, customers 1..3; symbols 0..2 are customers, 3 and 4 separators
    d = np.array([[0, 10, 20, 15], [10, 0, 12, 25], [20, 12, 0, 8], [15, 25, 8, 0]], np.int32)
    inst = dict(n=3, mat0=d)
    # routes (1, 2) and (3), one empty route
    assert bench.cvrptw_objectives(inst, [0, 1, 3, 2, 4]) == {"distance": 42 + 30, "vehicles": 2,
                                                             "longest": 42}
    assert bench.cvrptw_objectives(inst, [3, 4, 2, 0, 1]) == {"distance": 15 + 25 + 12 + 20,
                                                             "vehicles": 1, "longest": 72}


def test_latency_by_class():
    import json
    import bench
    lats = [0.1, 0.2, 3.0, 0.3, 2.5, 0.4]
    cls = ["tsp", "gap", "cvrptw", "tsp", "cvrptw", "tsp"]
    out = bench.latency_by_class(lats, cls)
    assert sorted(out) == ["cvrptw", "gap", "tsp"]
    assert out["tsp"]["requests"] == 3 and out["tsp"]["latency_p50_s"] == 0.3
    assert abs(out["cvrptw"]["latency_p50_s"] - 2.75) < 1e-12
    assert out["gap"] == {"requests": 1, "latency_p50_s": 0.2, "latency_p99_s": 0.2}
    json.dumps(out)   # goes into the bench's JSON line
