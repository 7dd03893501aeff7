"""Benchmark: move evaluations per second of the population search on GB300.

Default workload (N=1): the large single permutation solve — TSP n=442 in 6
Gaussian clusters (sigma 40) plus 10% uniform noise over [0,4000]^2, int32
rounded-Euclidean matrix, population 128, 128 candidates per member per
generation, 2-opt / or-opt / insertion with the L1 priors, T0 = 100,
alpha = 0.999, 200,000 generations.  One step = one complete solve (init +
every generation + elite), through the library's C ABI.

Timing: W untimed warm-up steps, then K steps timed with CUDA events on the
stream the library launches on, an L2 flush (a 512 MB write) between steps,
a barrier + synchronize on both sides, max over ranks.  Clocks are sampled
with nvidia-smi during the timed region.  ``e2e`` repeats the step through the
public API from host buffers: problem creation (host->device copy of the
matrix), the solve and the read-back of the best solution (device->host).

--impl reference times the CPU oracle on the host cores on a bounded sample
(a prefix of the same solve), the only other place this file runs it.
Under torchrun every rank solves its own replica (seed 1 + rank).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import instances as I  # noqa: E402

TO, INS, OR = 1, 2, 3
O_THREE_OPT, O_SEGMENT = 6, 7     # operator slots of the C ABI (cgo_op)


def workload(name: str):
    if name == "tsp442":
        inst = I.tsp_clustered(442, 0)
        cfg = dict(P=128, C=128, G=200000, op_mask=(1 << TO) | (1 << OR) | (1 << INS))
        desc = "tsp442-clustered P=128 C=128 G=200000 ops=2opt/oropt/insert"
    elif name == "tsp20":
        inst = I.tsp_uniform(20, 0)
        cfg = dict(P=32, C=128, G=2000, op_mask=0b0111,
                   w_op=[21845, 21845, 21845, 0, 0, 0, 0, 0])
        desc = "tsp20-uniform P=32 C=128 G=2000 ops=swap/2opt/insert"
    elif name == "qap64":
        inst = I.qap_grid(64, 0)
        cfg = dict(P=256, C=128, G=100000, op_mask=1, w_op=[65536, 0, 0, 0, 0, 0, 0, 0])
        desc = "qap64-grid P=256 C=128 G=100000 ops=swap"
    elif name == "cvrptw100":
        inst = I.cvrptw(100, 0)
        cfg = dict(P=32, C=128, G=20000)
        desc = "cvrptw100-solomon-r P=32 C=128 G=20000 V=25 Q=200"
    elif name == "serve":
        return None, dict(P=32, C=128, G=20000), "serve-poisson200x60s mix+15%cvrptw P=32 C=128 G=20000"
    elif name == "batch512":
        return None, dict(P=32, C=128, G=20000), "batch512-mix P=32 C=128 G=20000"
    else:
        raise SystemExit("unknown workload " + name)
    return inst, cfg, desc


def lib_params(prob, cfg):
    p = prob.default_params()
    extra = cfg.get("extra_mask", 0)
    p.update({k: v for k, v in cfg.items() if k != "extra_mask"})
    p["op_mask"] |= extra
    return p


def solve_variant(args, model: int, cfg: dict, desc: str):
    """The single-solve options beyond the workload's own configuration
    (start pool, islands, extra operators), applied alike by both arms."""
    cfg = dict(cfg)
    if args.init_oversample > 1 or args.init_heuristic:
        cfg["init_oversample"] = args.init_oversample
        cfg["init_heuristic"] = args.init_heuristic
        desc += " start=K%d%s" % (args.init_oversample, "+heuristic" if args.init_heuristic else "")
    if args.islands:
        isl, per, strat, nmig = (int(x) for x in args.islands.split(","))
        cfg.update(islands=isl, migrate_period=per, migrate_strategy=strat, migrate_n=nmig)
        desc += " islands=%d period=%d %s" % (isl, per, ["ring", "top-%d" % nmig,
                                                          "hybrid-%d" % nmig][strat])
    if args.extra_ops:
        cfg["extra_mask"] = extra_ops_mask(model, args.extra_ops)
        desc += " +ops=" + args.extra_ops
    if args.cross:
        cfg["cross_q16"] = args.cross
        desc += " cross=%.3f" % (args.cross / 65536.0)
    return cfg, desc


def cvrptw_objectives(inst: dict, sol) -> dict:
    """Travel distance and vehicles used by a separator-encoded CVRPTW
    solution (for the report; the search's own cost adds the penalties)."""
    n, d = int(inst["n"]), np.asarray(inst["mat0"])
    dist, used, prev = 0, 0, 0
    for s in list(sol) + [n]:
        if s >= n:
            if prev:
                dist += int(d[prev][0])
                used += 1
            prev = 0
        else:
            dist += int(d[prev][s + 1])
            prev = s + 1
    return {"distance": dist, "vehicles": used}


def extra_ops_mask(model: int, extra: str) -> int:
    """Operator bits that --extra-ops adds for a model (QAP's GPU path is swap-only)."""
    bits = 0
    for name in filter(None, extra.split(",")):
        if name == "three_opt" and model in (I.TSP, I.CVRPTW):
            bits |= 1 << O_THREE_OPT
        elif name == "segment" and model in (I.KNAPSACK, I.GAP):
            bits |= 1 << O_SEGMENT
        elif name not in ("three_opt", "segment"):
            raise SystemExit("unknown operator " + name)
    return bits


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------- reference
def run_reference(args, rank, world):
    """CPU oracle on the host cores: each step runs a bounded prefix of the
    same solve (the oracle is deliberately slow)."""
    if rank != 0:
        return
    import oracle as O
    inst, cfg, desc = workload(args.workload)
    if inst is None:
        # batched / served workloads: a stratified sample of the instance mix
        insts = [dict(x, tag=i) for i, x in enumerate(I.batch_mix(512, 0))][::64]
        desc += " (oracle on every 64th instance)"
    else:
        if args.cvrptw_weights and inst["model"] == I.CVRPTW:
            wd, wv = (int(x) for x in args.cvrptw_weights.split(","))
            inst = dict(inst, weight_distance=wd, weight_vehicles=wv)
            desc += " weights=(%d,%d)" % (wd, wv)
        insts = [inst]
        cfg, desc = solve_variant(args, inst["model"], cfg, desc)
    plist = []
    for x in insts:
        p = O.default_params(x)
        p.update({k: v for k, v in cfg.items() if k not in ("G", "extra_mask")})
        p["op_mask"] |= cfg.get("extra_mask", 0)
        plist.append(p)
    gens = args.ref_generations
    cores = O.lib().orc_threads(0)
    for _ in range(args.warmup):
        for x, p in zip(insts, plist):
            O.solve(x, p, 1, max(1, gens // 4))
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for x, p in zip(insts, plist):
            O.solve(x, p, 1, gens)
        times.append(time.perf_counter() - t0)
    evals = cfg["P"] * cfg["C"] * gens * len(insts)
    value = evals * args.steps / sum(times)
    line = {"metric": "move_evals_per_s", "value": value, "unit": "evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": desc, "sample_generations": gens},
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cores, "kind": "oracle",
                             "sample": "first %d generations of the %s solve per step" % (gens, desc)},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(inst, cfg, desc, budget_s: float):
    """Time the oracle as it stands on a bounded prefix of the workload."""
    import oracle as O
    p = O.default_params(inst)
    p.update({k: v for k, v in cfg.items() if k not in ("G", "extra_mask")})
    p["op_mask"] |= cfg.get("extra_mask", 0)
    cores = O.lib().orc_threads(0)
    t0 = time.perf_counter()
    O.solve(inst, p, 1, 2)
    per_gen = (time.perf_counter() - t0) / 2
    gens = int(max(2, min(cfg["G"], budget_s / max(per_gen, 1e-6))))
    t0 = time.perf_counter()
    O.solve(inst, p, 1, gens)
    dt = time.perf_counter() - t0
    evals = cfg["P"] * cfg["C"] * gens
    # one host thread, on an eighth of the sample (same generations from 0)
    g1 = max(2, gens // 8)
    t0 = time.perf_counter()
    O.solve(inst, p, 1, g1, threads=1)
    dt1 = time.perf_counter() - t0
    return {"value": evals / dt, "unit": "evals/s", "cores": cores, "kind": "oracle",
            "sample": "first %d generations of the %s solve (%.1f s)" % (gens, desc, dt),
            "single_thread": {"value": cfg["P"] * cfg["C"] * g1 / dt1, "cores": 1,
                              "sample": "first %d generations (%.1f s)" % (g1, dt1)}}


# ------------------------------------------------------------------- ours
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tsp442")
    ap.add_argument("--ref-generations", type=int, default=100)
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--batch-class", default="mix")
    ap.add_argument("--wpm", type=int, default=0, help="warps per member override (batched)")
    ap.add_argument("--slice", type=int, default=2000)
    ap.add_argument("--init-oversample", type=int, default=1,
                    help="single solve: K of the oversampled start (1 = plain start)")
    ap.add_argument("--init-heuristic", type=int, default=0,
                    help="single solve: 1 = add the row/column-sum start permutations")
    ap.add_argument("--extra-ops", default="",
                    help="enable operators beyond the default mask where they apply: "
                         "'three_opt' (TSP, CVRPTW), 'segment' (seg_flip / seg_reset: knapsack, GAP)")
    ap.add_argument("--cvrptw-weights", default="",
                    help="cvrptw100: objective weights 'distance,vehicles' (0,0 = distance only)")
    ap.add_argument("--cross", type=int, default=0,
                    help="crossover probability per member and AOS window, Q16 (0 = off)")
    ap.add_argument("--islands", default="",
                    help="single solve: islands 'I,period,strategy,N' (strategy 0 ring, "
                         "1 top-N, 2 hybrid)")
    ap.add_argument("--launch", default="",
                    help="single solve: fixed launch shape 'warps,wpm,staging,gens_in_flight' "
                         "instead of the autotuner (profiling runs)")
    ap.add_argument("--seq-sample", type=int, default=24)
    ap.add_argument("--generations", type=int, default=0,
                    help="override G (small cases for profiler captures)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    from paper_2603_19163_gb300 import cgo

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    if args.workload in ("batch512", "serve"):
        fn = bench_batch if args.workload == "batch512" else bench_serve
        fn(args, rank, world, local, cgo, torch, dist, barrier)
        if world > 1:
            dist.destroy_process_group()
        return

    inst, cfg, desc = workload(args.workload)
    if args.generations > 0:
        cfg["G"] = args.generations
        desc = desc.replace("G=", "G(full)=") + " G=%d" % cfg["G"]
    inst = dict(inst, tag=0)
    if args.cvrptw_weights and inst["model"] == I.CVRPTW:
        wd, wv = (int(x) for x in args.cvrptw_weights.split(","))
        inst.update(weight_distance=wd, weight_vehicles=wv)
        desc += " weights=(%d,%d)" % (wd, wv)
    seed = 1 + rank
    stream = torch.cuda.Stream()
    cfg, desc = solve_variant(args, inst["model"], cfg, desc)
    prob = cgo.Problem(inst)
    params = lib_params(prob, cfg)
    from paper_2603_19163_gb300.autotune import Autotuner
    tuner = Autotuner(trial_generations=min(cfg["G"], 2000))
    if args.launch:
        shape = tuple(int(x) for x in args.launch.split(","))
        prob.set_launch(shape[0], staging=shape[2], wpm=shape[1], ns=shape[3])
    else:
        shape = tuner.tune_solve(prob, params, seed)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            prob.solve(params, seed, stream)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    if rank == 0:
        sampler.start()
    step_ms, kern_ms = [], []
    launches0 = cgo.kernel_launches()
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            flush.fill_(1)                       # evict L2 between steps
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            prob.solve(params, seed, stream)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            kern_ms.append(prob.last_kernel_time()[0])
    torch.cuda.synchronize()
    launches = cgo.kernel_launches() - launches0
    barrier()
    clocks = sampler.stop() if rank == 0 else None

    evals_rank = cfg["P"] * cfg["C"] * cfg["G"] * args.steps
    agg = aggregate(sum(step_ms), evals_rank, dist if world > 1 else None, "cuda")
    total_ms, value = agg["max_ms"], agg["per_s"]
    _, best_cost = prob.best()
    # the elite of the start population alone (no generation)
    p0 = cgo.Problem(inst)
    p0.solve(dict(params, G=0), seed, stream)
    _, start_cost = p0.best()
    p0.close()

    # end to end through the public API: host arrays in, best solution out
    e2e_ms = []
    h2d = sum(int(np.asarray(inst[k]).nbytes) for k in ("mat0", "mat1", "vec0", "vec1", "vec2", "vec3")
              if inst.get(k) is not None)
    d2h = 0
    for _ in range(max(1, min(args.steps, 3))):
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p2 = cgo.Problem(inst)
        p2.solve(params, seed, stream)
        sol, c = p2.best()
        e2e_ms.append(1000 * (time.perf_counter() - t0))
        d2h = int(sol.nbytes) + 8
        p2.close()
    e2e_t = torch.tensor([sum(e2e_ms) / len(e2e_ms)], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
    e2e_value = cfg["P"] * cfg["C"] * cfg["G"] * world / (float(e2e_t.item()) / 1000.0)

    if rank == 0:
        kms = sum(kern_ms) / len(kern_ms)
        evals_launch = cfg["P"] * cfg["C"] * cfg["G"]
        cv = inst["model"] == I.CVRPTW
        # the roofline model covers the TSP and QAP deltas; a CVRPTW delta is a
        # route walk of data-dependent length (reported without one)
        roof = None if cv else roofline(evals_launch, kms, prob, clocks)
        # mean steps per candidate: the roofline's figure (the open window's K
        # counts, 1.25 when the run ends on a window boundary)
        uk = prob.state()["u_k"]
        ek = roof["ops_per_eval_steps"] if roof else (
            (uk[0] + 2 * uk[1] + 3 * uk[2]) / sum(uk) if sum(uk) else 1.25)
        line = {"metric": "move_evals_per_s", "value": value, "unit": "evals/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int64",
                "data": "synthetic",
                "config": {"workload": desc, "l2": "flushed between steps (512 MB write)",
                           "launch": {"warps_per_cta": shape[0], "warps_per_member": shape[1],
                                      "staging": ["auto", "smem", "global"][shape[2]],
                                      "gens_in_flight": shape[3],
                                      "chosen_by": "fixed (--launch)" if args.launch else
                                      "autotuner (%d trial shapes)" % len(
                                          tuner.solve_shapes(params))},
                           "best_cost": int(best_cost), "start_best_cost": int(start_cost),
                           "gens_per_s": cfg["G"] / (total_ms / args.steps / 1000.0),
                           # operator applications: each evaluation applies k
                           # operators, E[k] from the run's last K counts
                           "operator_applications_per_s": value * ek},
                "e2e": {"value": e2e_value, "unit": "evals/s", "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "gpu_launches": launches,
                "clocks": clocks, "roofline": roof}
        if cv:
            line["config"]["elite_objectives"] = cvrptw_objectives(inst, prob.best()[0])
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(inst, cfg, desc, args.cpu_budget)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def bench_batch(args, rank, world, local, cgo, torch, dist, barrier):
    """512 uneven instances (40% TSP n~U[50,500], 40% knapsack n~U[100,2000],
    20% GAP n~U[50,300]) advanced together by the batched persistent kernel
    under a CUDA graph; one step = one cgo_solve_batch of all of them.  The
    one-launch-per-solve form (cgo_solve of each instance in turn, same P, C,
    G, seeds) is timed on every 8th instance."""
    _, cfg, desc = workload("batch512")
    G = args.generations if args.generations > 0 else cfg["G"]
    mix = [dict(x, tag=i) for i, x in enumerate(I.batch_mix(512, 0))]
    if args.batch_class != "mix":
        cls = {"tsp": I.TSP, "knapsack": I.KNAPSACK, "gap": I.GAP, "cvrptw": I.CVRPTW}[args.batch_class]
        if cls == I.CVRPTW:
            mix = [dict(x, tag=i) for i, x in enumerate(I.serving_pool(0)[512:])]
        else:
            mix = [x for x in mix if x["model"] == cls]
        desc = desc.replace("batch512-mix", "batch-%s%d" % (args.batch_class, len(mix)))
    probs = [cgo.Problem(x) for x in mix]
    params = []
    for pr, x in zip(probs, mix):
        q = pr.default_params()
        q.update(P=cfg["P"], C=cfg["C"], G=G)
        q["op_mask"] |= extra_ops_mask(x["model"], args.extra_ops)
        q["cross_q16"] = args.cross
        params.append(q)
    if args.extra_ops:
        desc += " +ops=" + args.extra_ops
    if args.cross:
        desc += " cross=%.3f" % (args.cross / 65536.0)
    seeds = [1000 * rank + 1 + i for i in range(len(mix))]
    if args.wpm:
        for pr in probs:
            pr.set_launch(0, 0, args.wpm)
        tuned = {"fixed_wpm": args.wpm}
    else:
        from paper_2603_19163_gb300.autotune import Autotuner
        tuned = {str(k): {"warps_per_member": v[0], "trial_evals_per_s": v[1]}
                 for k, v in Autotuner(trial_generations=min(G, 300)).tune_batch(
                     probs, params).items()}
    stream = torch.cuda.Stream()
    for _ in range(args.warmup):
        cgo.solve_batch(probs, params, seeds, stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    barrier()
    if rank == 0:
        sampler.start()
    ms = []
    launches0 = cgo.kernel_launches()
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cgo.solve_batch(probs, params, seeds, stream)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    launches = cgo.kernel_launches() - launches0
    barrier()
    clocks = sampler.stop() if rank == 0 else None
    # solution quality of the last step: the sum of the instances' best costs per model
    best_sum = {}
    for pr, x in zip(probs, mix):
        key = {I.TSP: "tsp", I.KNAPSACK: "knapsack", I.GAP: "gap", I.CVRPTW: "cvrptw"}[x["model"]]
        best_sum[key] = best_sum.get(key, 0) + int(pr.best()[1])
    t = torch.tensor([sum(ms)], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    evals = sum(q["P"] * q["C"] * q["G"] for q in params)
    value = evals * args.steps * world / (total_ms / 1000.0)
    solves_s = len(probs) * args.steps * world / (total_ms / 1000.0)
    # one launch per solve, on a stratified sample (every 8th instance)
    sample = list(range(0, len(probs), 8))
    for i in sample:
        probs[i].set_launch(0, 0, 0)        # one launch per solve: its own default shape
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in sample:
        probs[i].solve(params[i], seeds[i], stream)
    seq_s = time.perf_counter() - t0
    seq_solves_s = len(sample) / seq_s
    # end to end: create from host arrays (H2D), batch solve, read every best (D2H)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    p2 = [cgo.Problem(x) for x in mix]
    cgo.solve_batch(p2, params, seeds, stream)
    outs = [pp.best() for pp in p2]
    e2e_s = time.perf_counter() - t0
    h2d = sum(int(sum(np.asarray(x[k]).nbytes for k in ("mat0", "mat1", "vec0", "vec1", "vec2",
                                                         "vec3") if x.get(k) is not None))
              for x in mix)
    d2h = sum(int(o[0].nbytes) + 8 for o in outs)
    for pp in p2:
        pp.close()
    if rank == 0:
        line = {"metric": "move_evals_per_s", "value": value, "unit": "evals/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
                "config": {"workload": desc.replace("G=20000", "G=%d" % G),
                           "l2": "inputs > L2 in total (512 instances); no flush",
                           "solves_per_s_batched": solves_s,
                           "solves_per_s_one_launch_per_solve": seq_solves_s,
                           "batched_over_sequential": solves_s / seq_solves_s,
                           "sequential_sample": "%d of %d instances" % (len(sample), len(mix)),
                           "best_cost_sum_by_model": best_sum,
                           "autotuner": tuned},
                "e2e": {"value": evals * world / e2e_s, "unit": "evals/s",
                        "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "gpu_launches": launches, "clocks": clocks}
        print(json.dumps(line), flush=True)


def bench_serve(args, rank, world, local, cgo, torch, dist, barrier):
    """Serving: Poisson arrivals at 200 requests/s for 60 s (sizes from the
    batch mix, 15% CVRPTW with 100 customers); each request is created from
    host arrays when it arrives (host->device copy), submitted to the
    continuous-batching server and waited for; latency = completion - arrival.
    The one-launch-per-solve form is timed on sampled requests (cgo_solve of
    each in turn) and its queueing under the same arrival trace follows from
    the Lindley recursion W_i = max(0, W_(i-1) + S_(i-1) - A_i) with those
    measured service times."""
    import threading
    _, cfg, desc = workload("serve")
    G = args.generations if args.generations > 0 else cfg["G"]
    duration = args.serve_seconds
    pool = I.serving_pool(0)
    trace = I.poisson_arrivals(200.0, duration, 7)
    params_of = {}
    pop_of_model = {}      # the autotuner's population per class, once chosen

    def params_for(k):
        if k not in params_of:
            pr = cgo.Problem(dict(pool[k], tag=k))
            q = pr.default_params()
            q.update(P=pop_of_model.get(pool[k]["model"], cfg["P"]), C=cfg["C"], G=G)
            params_of[k] = q
            pr.close()
        return params_of[k]

    # autotuner: batched throughput per class (trial batches), then the
    # population per class from the load the trace offers
    from paper_2603_19163_gb300.autotune import Autotuner, population_for_load
    tuner = Autotuner(trial_generations=200)
    models = {}
    for k in set(k for _, k in trace):
        models.setdefault(pool[k]["model"], []).append(k)
    sample_probs, sample_params = [], []
    fill = 2 * torch.cuda.get_device_properties(local).multi_processor_count
    for mdl, ks in models.items():
        pick = ks[:: max(1, len(ks) // 8)][:8]
        for j in range(fill):           # a trial batch large enough to fill the GPU
            k = pick[j % len(pick)]
            sample_probs.append(cgo.Problem(dict(pool[k], tag=j)))
            sample_params.append(params_for(k))
    t_phase = time.perf_counter()
    tuned = tuner.tune_batch(sample_probs, sample_params, sample=fill)
    print("serve: autotune %.1f s" % (time.perf_counter() - t_phase), file=sys.stderr, flush=True)
    for pr in sample_probs:
        pr.close()
    share = {}
    for _, k in trace:
        share[pool[k]["model"]] = share.get(pool[k]["model"], 0) + 1.0 / len(trace)
    pops, load = population_for_load({m: tuned[m][1] for m in tuned}, share,
                                     len(trace) / duration, G, cfg["C"])
    wpm_of = {m: tuned[m][0] for m in tuned}
    pop_of_model.update(pops)
    for k in params_of:
        params_of[k]["P"] = pops[pool[k]["model"]]
    srv = cgo.Server(max_slots=4096, hbm_budget_bytes=96 << 30, slice_generations=args.slice)
    # warm-up: a few requests end to end
    def make(k, tag):
        pr = cgo.Problem(dict(pool[k], tag=tag))
        pr.set_launch(0, 0, wpm_of[pool[k]["model"]])
        return pr

    warm = [make(k, k) for k in (0, 1, 2, 512)]
    for pr, k in zip(warm, (0, 1, 2, 512)):
        srv.wait(srv.submit(pr, params_for(k), 1), -1)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    if rank == 0:
        sampler.start()
    probs = [None] * len(trace)
    tickets = [None] * len(trace)
    results = [None] * len(trace)
    launches0 = cgo.kernel_launches()
    t_start = time.perf_counter()

    def producer():
        for i, (ta, k) in enumerate(trace):
            now = time.perf_counter() - t_start
            if ta > now:
                time.sleep(ta - now)
            pr = make(k, i)
            probs[i] = pr
            tickets[i] = srv.submit(pr, params_for(k), 1 + i)

    th = threading.Thread(target=producer)
    th.start()
    stop_mon = [False]

    def monitor():
        while True:
            time.sleep(5.0)
            if stop_mon[0]:
                return
            print("serve: t=%.0f s %s" % (time.perf_counter() - t_start, srv.stats()),
                  file=sys.stderr, flush=True)

    mon = threading.Thread(target=monitor, daemon=True)
    mon.start()
    done_at = [0.0] * len(trace)
    for i in range(len(trace)):
        while tickets[i] is None:
            time.sleep(0.0005)
        cost, lat = srv.wait(tickets[i], -1)
        results[i] = (cost, lat)
        done_at[i] = time.perf_counter() - t_start
    th.join()
    launches = cgo.kernel_launches() - launches0
    stop_mon[0] = True
    wall = max(done_at) - trace[0][0]
    # every request's instance arrays go host -> device when it arrives; its
    # elite cost (int64) comes back when it completes
    h2d = sum(int(sum(np.asarray(pool[k][f]).nbytes for f in ("mat0", "mat1", "vec0", "vec1", "vec2",
                                                               "vec3") if pool[k].get(f) is not None))
              for _, k in trace)
    d2h = 8 * len(trace)
    print("serve: trace done %.1f s" % (time.perf_counter() - t_start), file=sys.stderr, flush=True)
    clocks = sampler.stop() if rank == 0 else None
    stats = srv.stats()
    srv.close()
    lats = np.array([r[1] for r in results])
    served_solves_s = len(trace) / wall
    evals = sum(params_for(k)["P"] * params_for(k)["C"] * G for _, k in trace)
    # one launch per solve: per-class service times measured on a stratified
    # sample of the trace's requests, queueing by the Lindley recursion
    def cls_of(k):
        return "cvrptw" if k >= 512 else ("tsp", "qap", "knapsack", "gap")[pool[k]["model"]]
    by_cls = {}
    for i, (_, k) in enumerate(trace):
        by_cls.setdefault(cls_of(k), []).append(i)
    per = max(2, args.seq_sample // max(1, len(by_cls)))
    service = {}
    for c, idx in by_cls.items():
        for i in idx[::max(1, len(idx) // per)][:per]:
            k = trace[i][1]
            pr = cgo.Problem(dict(pool[k], tag=i))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pr.solve(params_for(k), 1 + i)
            service.setdefault(c, []).append(time.perf_counter() - t0)
            pr.close()
    mean_cls = {c: float(np.mean(v)) for c, v in service.items()}
    overall = float(np.mean([mean_cls[cls_of(k)] for _, k in trace]))
    rng_pick = [x for v in service.values() for x in v]
    W, prev_t, prev_s, seq_lat = 0.0, None, 0.0, []
    for ta, k in trace:
        s_i = mean_cls[cls_of(k)]
        if prev_t is not None:
            W = max(0.0, W + prev_s - (ta - prev_t))
        seq_lat.append(W + s_i)
        prev_t, prev_s = ta, s_i
    seq_lat = np.array(seq_lat)
    seq_solves_s = 1.0 / overall
    for pr in probs + warm:
        if pr is not None:
            pr.close()
    if rank == 0:
        line = {"metric": "served_solves_per_s", "value": served_solves_s, "unit": "solves/s",
                "n_gpus": world, "steps": 1, "warmup": len(warm), "ms_per_step": 1000 * wall,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "int64", "data": "synthetic",
                "config": {"workload": desc.replace("G=20000", "G=%d" % G).replace(
                               "x60s", "x%ds" % int(duration)),
                           "requests": len(trace), "slice_generations": args.slice,
                           "autotuner": {"population_by_model": {str(m): v for m, v in pops.items()},
                                         "predicted_load": load,
                                         "warps_per_member_by_model": {str(m): v for m, v in wpm_of.items()},
                                         "trial_evals_per_s_by_model": {str(m): tuned[m][1] for m in tuned}},
                           "move_evals_per_s": evals / wall,
                           "latency_p50_s": float(np.percentile(lats, 50)),
                           "latency_p99_s": float(np.percentile(lats, 99)),
                           "latency_max_s": float(lats.max()),
                           "one_launch_per_solve": {
                               "solves_per_s": seq_solves_s,
                               "latency_p50_s": float(np.percentile(seq_lat, 50)),
                               "latency_p99_s": float(np.percentile(seq_lat, 99)),
                               "service_s_by_class": mean_cls,
                               "how": "per-class service times of %d sampled requests, Lindley "
                                      "recursion over the same arrivals" % len(rng_pick)},
                           "served_over_one_launch_per_solve": served_solves_s / seq_solves_s,
                           "server": stats},
                "e2e": {"value": served_solves_s, "unit": "solves/s",
                        "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "gpu_launches": launches, "clocks": clocks}
        print(json.dumps(line), flush=True)


def aggregate(local_ms: float, local_units: float, dist=None, device="cpu") -> dict:
    """Whole-job figures of a timed region over all ranks: the time is the
    maximum over ranks, the units (move evaluations, solves) their sum."""
    import torch
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    u = torch.tensor([local_units], dtype=torch.float64, device=device)
    world = 1
    if dist is not None and dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        world = dist.get_world_size()
    ms = float(t.item())
    return {"max_ms": ms, "units": float(u.item()), "per_s": float(u.item()) / (ms / 1000.0),
            "world": world}


# Issue-slot roofline of the evolve kernel: the kernel is bound by integer
# instruction issue and latency (instance data are staged in shared memory,
# nothing streams from HBM), so the peak is one instruction per lane per clock
# on every SM sub-partition: SMs x 128 lanes x f_max.  The algorithmic work of
# one move evaluation is counted in integer operations as stated in
# the design notes (Philox4x32-10 calls, roulette choices, position mapping,
# junction lookups and distance gathers), with the mean number of steps per
# candidate taken from the run's own K-step statistics.
OPS_PHILOX = 100          # 10 rounds x (2 mul.lo + 2 mul.hi + 4 xor + 2 key add)
OPS_STEP = 120            # TSP: roulette 10 + decode 15 + 10 lookups x 5 + 10 gathers x 4 + sums 5
OPS_CAND = 20             # K roulette, argmin share, stats
OPS_QAP_K = 17            # QAP, per k of the O(n) swap delta: 9 loads, 2 multiplies, 6 add/sub


# DRAM bytes (read + write) of one full launch of the single-solve kernel on
# the tsp442 workload, from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum, one pass; profiles/evolve_tsp442_g200000_dram.md),
# valid only for the kernel sources it was taken on.
TRAFFIC_BYTES = 1.28e6 + 89.86e3
TRAFFIC_SOURCES = "a9e1cac90c127137"


def kernel_sources_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("cgo_kernels.cu", "cgo_device.cuh", "cgo_internal.h"):
        with open(os.path.join(ROOT, "paper_2603_19163_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def roofline(evals_launch, kernel_ms, prob, clocks):
    import torch
    st = prob.state()
    uk = st["u_k"]
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    fmax = 2070.0
    try:
        pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        fmax = float(pk.get("sm_max_mhz", fmax))
    except (OSError, ValueError):
        pass
    # mean steps per candidate from the final window's K counts (fallback 1.25)
    tot = sum(uk)
    ek = (uk[0] + 2 * uk[1] + 3 * uk[2]) / tot if tot else 1.25
    model = int(prob.inst["model"])
    n = int(prob.inst["n"])
    qap = model == 1
    step_ops = 25 + OPS_QAP_K * n if qap else OPS_STEP
    ops_eval = ek * (OPS_PHILOX + step_ops) + OPS_CAND
    achieved = evals_launch * ops_eval / (kernel_ms / 1000.0) / 1e12
    peak = sms * 128 * fmax * 1e6 / 1e12
    traffic = TRAFFIC_BYTES if kernel_sources_hash() == TRAFFIC_SOURCES else None
    # the gather view: per counted step 8 tour positions and 8 distances
    # (algorithmic; the kernel executes all 3 steps of every candidate: 48),
    # against the random-gather rate measured on this GPU from a shared
    # buffer (the triangle and tours are staged in shared memory)
    from paper_2603_19163_gb300 import cgo
    g_peak, _ = cgo.gather_peak(0, 16)
    l2_peak, _ = cgo.gather_peak(1, 18)
    # (QAP: 9 shared loads per k of the O(n) delta)
    per_step = 9.0 * n + 2 if qap else 16.0
    gathers_eval = per_step * ek
    executed = per_step * (ek if qap else 3.0)
    g_achieved = evals_launch * gathers_eval / (kernel_ms / 1000.0)
    if not qap and kernel_sources_hash() != TRAFFIC_SOURCES:
        traffic = None
    if qap:
        traffic = None
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
            "frac": achieved / peak, "traffic": traffic,
            "kernel": "evolve_kernel<%s>" % ("QAP" if qap else "TSP,int16"), "kernel_ms": kernel_ms,
            "ops_per_eval": ops_eval, "ops_per_eval_steps": ek,
            "peak_basis": "%d SMs x 128 lanes x %.0f MHz" % (sms, fmax),
            "gather": {"achieved": g_achieved / 1e9, "peak": g_peak / 1e9, "unit": "G gathers/s",
                       "frac": g_achieved / g_peak, "gathers_per_eval": gathers_eval,
                       "executed_per_eval": executed,
                       "executed_frac": evals_launch * executed / (kernel_ms / 1000.0) / g_peak,
                       "peak_basis": "measured: random 16-bit gathers from a 128 KB shared buffer, "
                                     "one 1024-thread CTA per SM (cgo_gather_peak kind 0)",
                       "l2_random_gather_peak": l2_peak / 1e9}}


if __name__ == "__main__":
    main()
