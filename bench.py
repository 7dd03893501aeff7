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

With N=1 the line also carries the batched and served forms of the metric
(``config.batched``: the 512-instance uneven batch, solves/s against one
launch per solve on every 8th instance; ``config.served``: 10 s of the
200 requests/s Poisson trace through the continuous-batching server, p50/p99
latency, against one launch per solve replayed live on the trace's first
second and modelled over the whole trace), each with its own clock record.
The roofline counts the algorithmic distance gathers of the operators the
solve applied (whole-solve counts from the library) against the measured
shared-memory random-gather rate.

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
O_ROW_SWAP, O_ROW_MERGE, O_ROW_SPLIT = 8, 9, 10


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


LEX_NAMES = {"d": 0, "v": 1, "l": 2}      # distance, vehicles used, longest route


def cvrptw_variant(args, inst: dict, desc: str):
    """CVRPTW objective modes applied alike by both arms: weights
    'distance,vehicles', or the lexicographic mode 'd:tol,v:tol[,l:tol]'
    (objectives in priority order with their tolerances)."""
    if inst is None or inst["model"] != I.CVRPTW:
        return inst, desc
    if args.cvrptw_weights:
        wd, wv = (int(x) for x in args.cvrptw_weights.split(","))
        inst = dict(inst, weight_distance=wd, weight_vehicles=wv)
        desc += " weights=(%d,%d)" % (wd, wv)
    if args.cvrptw_longest:
        inst = dict(inst, weight_longest=args.cvrptw_longest)
        desc += " longest-route weight=%d" % args.cvrptw_longest
    if args.cvrptw_lex:
        lex = [(LEX_NAMES[t.split(":")[0]], int(t.split(":")[1])) for t in args.cvrptw_lex.split(",")]
        inst = dict(inst, lexicographic=lex)
        desc += " lexicographic=" + args.cvrptw_lex
    return inst, desc


def cvrptw_objectives(inst: dict, sol) -> dict:
    """Travel distance, vehicles used and the longest route's distance of a
    separator-encoded CVRPTW solution (for the report; the search's own cost
    adds the penalties)."""
    n, d = int(inst["n"]), np.asarray(inst["mat0"])
    dist, used, prev, rd, longest = 0, 0, 0, 0, 0
    for s in list(sol) + [n]:
        if s >= n:
            if prev:
                dist += int(d[prev][0])
                rd += int(d[prev][0])
                longest = max(longest, rd)
                used += 1
            prev, rd = 0, 0
        else:
            dist += int(d[prev][s + 1])
            rd += int(d[prev][s + 1])
            prev = s + 1
    return {"distance": dist, "vehicles": used, "longest": longest}


def extra_ops_mask(model: int, extra: str) -> int:
    """Operator bits that --extra-ops adds for a model (3-opt for the
    permutation models, the segment operator for binary and integer ones,
    the row level for CVRPTW)."""
    bits = 0
    for name in filter(None, extra.split(",")):
        if name == "three_opt" and model in (I.TSP, I.QAP, I.CVRPTW):
            bits |= 1 << O_THREE_OPT
        elif name == "segment" and model in (I.KNAPSACK, I.GAP):
            bits |= 1 << O_SEGMENT
        elif name == "rows" and model == I.CVRPTW:
            bits |= (1 << O_ROW_SWAP) | (1 << O_ROW_MERGE) | (1 << O_ROW_SPLIT)
        elif name not in ("three_opt", "segment", "rows"):
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
    pops = None
    if inst is None:
        # batched / served workloads: a stratified sample of the instance mix,
        # with the populations the batched arm's autotuner gives the classes
        mix = I.batch_mix(512, 0)
        insts = [dict(x, tag=i) for i, x in enumerate(mix)][::64]
        desc += " (oracle on every 64th instance)"
        if args.workload == "batch512" and args.batch_pop <= 0:
            from paper_2603_19163_gb300.autotune import batch_populations
            l2 = 126 << 20
            try:
                import torch
                if torch.cuda.is_available():
                    l2 = int(getattr(torch.cuda.get_device_properties(0), "L2_cache_size", l2))
            except ImportError:
                pass
            pops = batch_populations(mix, l2)[0]
    else:
        inst, desc = cvrptw_variant(args, inst, desc)
        insts = [inst]
        cfg, desc = solve_variant(args, inst["model"], cfg, desc)
    plist = []
    for x in insts:
        p = O.default_params(x)
        p.update({k: v for k, v in cfg.items() if k not in ("G", "extra_mask")})
        if pops is not None:
            p["P"] = pops[int(x["model"])]
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
    evals = sum(p["P"] for p in plist) * cfg["C"] * gens
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
    ap.add_argument("--batch-pop", type=int, default=0,
                    help="batched: one population for every class instead of the autotuner's")
    ap.add_argument("--slice", type=int, default=2000)
    ap.add_argument("--serve-fast-slice", type=int, default=20000,
                    help="serving: generations per slice of every class but the slowest, "
                         "at most the request budget (0 = --slice for every class)")
    ap.add_argument("--init-oversample", type=int, default=1,
                    help="single solve: K of the oversampled start (1 = plain start)")
    ap.add_argument("--init-heuristic", type=int, default=0,
                    help="single solve: 1 = add the row/column-sum start permutations")
    ap.add_argument("--extra-ops", default="",
                    help="enable operators beyond the default mask where they apply: "
                         "'three_opt' (TSP, QAP, CVRPTW), 'segment' (seg_flip / seg_reset: "
                         "knapsack, GAP), 'rows' (row_swap / row_merge / row_split: CVRPTW)")
    ap.add_argument("--cvrptw-weights", default="",
                    help="cvrptw100: objective weights 'distance,vehicles' (0,0 = distance only)")
    ap.add_argument("--cvrptw-longest", type=int, default=0,
                    help="cvrptw100: weight of the longest route's distance (0 = off)")
    ap.add_argument("--cvrptw-lex", default="",
                    help="cvrptw100: lexicographic mode, objectives in priority order with "
                         "tolerances, e.g. 'd:50,v:0' (d distance, v vehicles, l longest route)")
    ap.add_argument("--cross", type=int, default=0,
                    help="crossover probability per member and AOS window, Q16 (0 = off)")
    ap.add_argument("--islands", default="",
                    help="single solve: islands 'I,period,strategy,N' (strategy 0 ring, "
                         "1 top-N, 2 hybrid)")
    ap.add_argument("--launch", default="",
                    help="single solve: fixed launch shape 'warps,wpm,staging,gens_in_flight' "
                         "instead of the autotuner (profiling runs)")
    ap.add_argument("--seq-live-seconds", type=float, default=1.0,
                    help="serving: seconds of the trace replayed live by one launch per solve")
    ap.add_argument("--no-extras", action="store_true",
                    help="tsp442: leave out the batched and served results of the default line")
    ap.add_argument("--extra-steps", type=int, default=2,
                    help="tsp442 line: timed batches of the 512-instance mix")
    ap.add_argument("--extra-serve-seconds", type=float, default=10.0,
                    help="tsp442 line: seconds of the Poisson trace served")
    ap.add_argument("--generations", type=int, default=0,
                    help="override G (small cases for profiler captures)")
    ap.add_argument("--warm-start", type=int, default=0,
                    help="single solve: time G generations resumed from the state after this many "
                         "(a multiple of the AOS interval; profiles of the late phase)")
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
    inst, desc = cvrptw_variant(args, inst, desc)
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

    # --warm-start W: each timed solve resumes from the state after W
    # generations (the late phase of the search, where a long run spends
    # most of its time); the state is written before the timed region
    warm = None
    if args.warm_start > 0:
        prob.solve(dict(params, G=args.warm_start), seed, stream)
        warm = prob.state()
        desc += " resumed after %d generations" % args.warm_start

    def prepare():
        if warm is not None:
            prob.set_state(params, seed, warm)

    def run_step():
        if warm is None:
            prob.solve(params, seed, stream)
        else:
            prob.solve_continue(cfg["G"], stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            prepare()
            run_step()
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
            prepare()
            flush.fill_(1)                       # evict L2 between steps
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run_step()
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

    extras = {}
    if (world == 1 and args.workload == "tsp442" and not args.no_extras and args.generations == 0
            and args.warm_start == 0):
        # the batched and served forms of the metric (configs of the 512-instance
        # batch and the Poisson serving trace), each against one launch per solve
        t_x = time.perf_counter()
        b = batch_run(args, cgo, torch, local, args.extra_steps, 1, 20000)
        extras["batched"] = {k: b[k] for k in (
            "desc", "population", "solves_per_s", "evals_per_s", "one_launch_per_solve_solves_per_s",
            "batched_over_one_launch_per_solve", "same_final_costs", "one_launch_per_solve_sample",
            "autotuner", "clocks", "gpu_launches", "steps", "total_ms")}
        sv = serve_run(args, cgo, torch, local, args.extra_serve_seconds, 20000,
                       args.seq_live_seconds)
        extras["served"] = {k: v for k, v in sv.items() if k not in ("h2d_bytes", "d2h_bytes")}
        extras["seconds"] = time.perf_counter() - t_x

    if rank == 0:
        kms = sum(kern_ms) / len(kern_ms)
        cv = inst["model"] == I.CVRPTW
        # the roofline model covers the TSP and QAP deltas; a CVRPTW delta is a
        # route walk of data-dependent length (reported without one)
        roof = None if cv else roofline(kms, prob, clocks)
        # mean steps per candidate over the whole solve (measured counts)
        mix = op_mix(prob.op_counts())
        ek = mix["steps_per_eval"]
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
                           # operators, E[k] counted over the whole solve
                           "operator_applications_per_s": value * ek,
                           "op_mix": mix},
                "e2e": {"value": e2e_value, "unit": "evals/s", "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "gpu_launches": launches,
                "clocks": clocks, "roofline": roof}
        if cv:
            line["config"]["elite_objectives"] = cvrptw_objectives(inst, prob.best()[0])
        line["config"].update({k: v for k, v in extras.items()})
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(inst, cfg, desc, args.cpu_budget)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def batch_run(args, cgo, torch, local, steps, warmup, G, rank=0, world=1, dist=None,
              barrier=lambda: None) -> dict:
    """512 uneven instances (40% TSP n~U[50,500], 40% knapsack n~U[100,2000],
    20% GAP n~U[50,300]) advanced together by the batched persistent kernel
    under a CUDA graph; one step = one cgo_solve_batch of all of them.  The
    one-launch-per-solve form (cgo_solve of each instance in turn, same P, C,
    G, seeds, each with its own default launch shape) runs on every 8th
    instance; both forms reach the same final costs (bit-identical results)."""
    _, cfg, desc = workload("batch512")
    mix = [dict(x, tag=i) for i, x in enumerate(I.batch_mix(512, 0))]
    if args.batch_class != "mix":
        cls = {"tsp": I.TSP, "knapsack": I.KNAPSACK, "gap": I.GAP, "cvrptw": I.CVRPTW}[args.batch_class]
        if cls == I.CVRPTW:
            mix = [dict(x, tag=i) for i, x in enumerate(I.serving_pool(0)[512:])]
        else:
            mix = [x for x in mix if x["model"] == cls]
        desc = desc.replace("batch512-mix", "batch-%s%d" % (args.batch_class, len(mix)))
    probs = [cgo.Problem(x) for x in mix]
    # population per model class: fixed, or the autotuner's L2-aware rule
    from paper_2603_19163_gb300.autotune import batch_populations
    if args.batch_pop > 0:
        pops, ws = {int(x["model"]): args.batch_pop for x in mix}, None
    else:
        l2 = int(getattr(torch.cuda.get_device_properties(local), "L2_cache_size", 126 << 20))
        pops, ws = batch_populations(mix, l2)
    params = []
    for pr, x in zip(probs, mix):
        q = pr.default_params()
        q.update(P=pops[int(x["model"])], C=cfg["C"], G=G)
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
    for _ in range(warmup):
        cgo.solve_batch(probs, params, seeds, stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    barrier()
    if rank == 0:
        sampler.start()
    ms = []
    launches0 = cgo.kernel_launches()
    for _ in range(steps):
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
    best_sum, batched_best = {}, []
    for pr, x in zip(probs, mix):
        key = {I.TSP: "tsp", I.KNAPSACK: "knapsack", I.GAP: "gap", I.CVRPTW: "cvrptw"}[x["model"]]
        c = int(pr.best()[1])
        batched_best.append(c)
        best_sum[key] = best_sum.get(key, 0) + c
    t = torch.tensor([sum(ms)], dtype=torch.float64, device="cuda")
    if dist is not None and world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    evals = sum(q["P"] * q["C"] * q["G"] for q in params)
    value = evals * steps * world / (total_ms / 1000.0)
    solves_s = len(probs) * steps * world / (total_ms / 1000.0)
    # one launch per solve, on a stratified sample (every 8th instance)
    sample = list(range(0, len(probs), 8))
    for i in sample:
        probs[i].set_launch(0, 0, 0)        # one launch per solve: its own default shape
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in sample:
        probs[i].solve(params[i], seeds[i], stream)
    seq_s = time.perf_counter() - t0
    same = all(int(probs[i].best()[1]) == batched_best[i] for i in sample)
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
    for pp in p2 + probs:
        pp.close()
    pop_note = {"population_by_model": {str(m): v for m, v in pops.items()},
                "rule": ("fixed (--batch-pop)" if ws is None else
                         "L2-aware: largest per class whose batch working set fits L2 (%.1f MB)"
                         % (ws / 2 ** 20))}
    return {"desc": desc.replace("G=20000", "G=%d" % G).replace("P=32 ", ""), "value": value,
            "total_ms": total_ms, "population": pop_note,
            "steps": steps, "evals_per_s": value, "solves_per_s": solves_s,
            "one_launch_per_solve_solves_per_s": seq_solves_s,
            "batched_over_one_launch_per_solve": solves_s / seq_solves_s,
            "same_final_costs": same,
            "one_launch_per_solve_sample": "%d of %d instances (every 8th)" % (len(sample), len(mix)),
            "best_cost_sum_by_model": best_sum, "autotuner": tuned, "clocks": clocks,
            "gpu_launches": launches, "e2e_evals_per_s": evals * world / e2e_s,
            "h2d_bytes": h2d, "d2h_bytes": d2h}


def bench_batch(args, rank, world, local, cgo, torch, dist, barrier):
    G = args.generations if args.generations > 0 else workload("batch512")[1]["G"]
    r = batch_run(args, cgo, torch, local, args.steps, args.warmup, G, rank, world, dist, barrier)
    if rank == 0:
        line = {"metric": "move_evals_per_s", "value": r["value"], "unit": "evals/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": r["total_ms"] / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
                "config": {"workload": r["desc"],
                           "l2": "inputs > L2 in total (512 instances); no flush",
                           "solves_per_s_batched": r["solves_per_s"],
                           "solves_per_s_one_launch_per_solve": r["one_launch_per_solve_solves_per_s"],
                           "batched_over_sequential": r["batched_over_one_launch_per_solve"],
                           "same_final_costs": r["same_final_costs"],
                           "sequential_sample": r["one_launch_per_solve_sample"],
                           "best_cost_sum_by_model": r["best_cost_sum_by_model"],
                           "population": r["population"],
                           "autotuner": r["autotuner"]},
                "e2e": {"value": r["e2e_evals_per_s"], "unit": "evals/s",
                        "h2d_bytes_per_step": r["h2d_bytes"], "d2h_bytes_per_step": r["d2h_bytes"]},
                "gpu_launches": r["gpu_launches"], "clocks": r["clocks"]}
        print(json.dumps(line), flush=True)


def latency_by_class(lats, classes) -> dict:
    """Requests, p50 and p99 latency (s) per request class."""
    out = {}
    for c in sorted(set(classes)):
        v = np.array([x for x, k in zip(lats, classes) if k == c], dtype=np.float64)
        out[c] = {"requests": int(v.size), "latency_p50_s": float(np.percentile(v, 50)),
                  "latency_p99_s": float(np.percentile(v, 99))}
    return out


def lindley(trace, service_of) -> np.ndarray:
    """Latencies of one server taking requests first come, first served:
    W_i = max(0, W_(i-1) + S_(i-1) - A_i) (Lindley), latency = W_i + S_i."""
    W, prev_t, prev_s, out = 0.0, None, 0.0, []
    for ta, k in trace:
        s_i = service_of(k)
        if prev_t is not None:
            W = max(0.0, W + prev_s - (ta - prev_t))
        out.append(W + s_i)
        prev_t, prev_s = ta, s_i
    return np.array(out)


def serve_run(args, cgo, torch, local, duration, G, seq_live_s, rank=0) -> dict:
    """Serving: Poisson arrivals at 200 requests/s (sizes from the batch mix,
    15% CVRPTW with 100 customers); each request is created from host arrays
    when it arrives (host->device copy), submitted to the continuous-batching
    server and waited for; latency = completion - arrival.  The
    one-launch-per-solve form replays the first seq_live_s seconds of the
    same trace for real (one worker, first come first served, cgo_solve of
    each request with its own default launch shape); its measured service
    times per class also drive the Lindley recursion over the whole trace."""
    import threading
    _, cfg, desc = workload("serve")
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
        pick = sorted(ks)[:: max(1, len(ks) // 8)][:8]
        for j in range(fill):           # a trial batch large enough to fill the GPU
            k = pick[j % len(pick)]
            sample_probs.append(cgo.Problem(dict(pool[k], tag=j)))
            sample_params.append(params_for(k))
    tuned = tuner.tune_batch(sample_probs, sample_params, sample=fill)
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
    # generations per slice: the class that advances slowest per request
    # keeps --slice; the others take --serve-fast-slice (the autotuner's rule)
    from paper_2603_19163_gb300.autotune import slices_by_class
    slice_by_model = {int(m): v for m, v in slices_by_class(
        {m: tuned[m][1] for m in tuned}, pops, cfg["C"], G, args.slice,
        args.serve_fast_slice).items()}
    srv = cgo.Server(max_slots=4096, hbm_budget_bytes=96 << 30, slice_generations=args.slice,
                     slice_by_model=slice_by_model)

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
    done_at = [0.0] * len(trace)
    for i in range(len(trace)):
        while tickets[i] is None:
            time.sleep(0.0005)
        cost, lat = srv.wait(tickets[i], -1)
        results[i] = (cost, lat)
        done_at[i] = time.perf_counter() - t_start
    th.join()
    launches = cgo.kernel_launches() - launches0
    wall = max(done_at) - trace[0][0]
    clocks = sampler.stop() if rank == 0 else None
    stats = srv.stats()
    srv.close()
    # every request's instance arrays go host -> device when it arrives; its
    # elite cost (int64) comes back when it completes
    h2d = sum(int(sum(np.asarray(pool[k][f]).nbytes for f in ("mat0", "mat1", "vec0", "vec1", "vec2",
                                                               "vec3") if pool[k].get(f) is not None))
              for _, k in trace)
    lats = np.array([r[1] for r in results])
    served_solves_s = len(trace) / wall
    evals = sum(params_for(k)["P"] * params_for(k)["C"] * G for _, k in trace)

    def cls_of(k):
        return "cvrptw" if k >= 512 else ("tsp", "qap", "knapsack", "gap")[pool[k]["model"]]

    # one launch per solve, live: the trace's first seq_live_s seconds
    live = [(i, ta, k) for i, (ta, k) in enumerate(trace) if ta < trace[0][0] + seq_live_s]
    seq_lat, service, same = [], {}, True
    torch.cuda.synchronize()
    t_live = time.perf_counter() - trace[0][0]
    for i, ta, k in live:
        now = time.perf_counter() - t_live
        if ta > now:
            time.sleep(ta - now)
        pr = cgo.Problem(dict(pool[k], tag=i))
        t0 = time.perf_counter()
        pr.solve(params_for(k), 1 + i)
        c = int(pr.best()[1])
        t1 = time.perf_counter()
        service.setdefault(cls_of(k), []).append(t1 - t0)
        seq_lat.append(t1 - t_live - ta)
        same = same and c == int(results[i][0])
        pr.close()
    seq_lat = np.array(seq_lat)
    mean_cls = {c: float(np.mean(v)) for c, v in service.items()}
    overall = float(np.mean([mean_cls.get(cls_of(k), max(mean_cls.values())) for _, k in trace]))
    model_lat = lindley(trace, lambda k: mean_cls.get(cls_of(k), max(mean_cls.values())))
    model_prefix = lindley([(ta, k) for _, ta, k in live],
                           lambda k: mean_cls.get(cls_of(k), max(mean_cls.values())))
    served_prefix = np.array([results[i][1] for i, _, _ in live])
    for pr in probs + warm:
        if pr is not None:
            pr.close()
    return {"desc": desc.replace("G=20000", "G=%d" % G).replace("x60s", "x%ds" % int(duration)),
            "requests": len(trace), "wall_s": wall, "solves_per_s": served_solves_s,
            "move_evals_per_s": evals / wall,
            "latency_p50_s": float(np.percentile(lats, 50)),
            "latency_p99_s": float(np.percentile(lats, 99)),
            "latency_max_s": float(lats.max()),
            "latency_by_class": latency_by_class(lats, [cls_of(k) for _, k in trace]),
            "slice_generations": args.slice,
            "slice_by_model": {str(m): v for m, v in slice_by_model.items()},
            "autotuner": {"population_by_model": {str(m): v for m, v in pops.items()},
                          "predicted_load": load,
                          "warps_per_member_by_model": {str(m): v for m, v in wpm_of.items()},
                          "trial_evals_per_s_by_model": {str(m): tuned[m][1] for m in tuned}},
            "one_launch_per_solve": {
                "live": {"requests": len(live), "arrivals_s": seq_live_s,
                         "solves_per_s": len(live) / float(sum(sum(v) for v in service.values())),
                         "latency_p50_s": float(np.percentile(seq_lat, 50)),
                         "latency_p99_s": float(np.percentile(seq_lat, 99)),
                         "served_latency_p50_s_same_requests": float(np.percentile(served_prefix, 50)),
                         "served_latency_p99_s_same_requests": float(np.percentile(served_prefix, 99)),
                         "lindley_p50_s_same_requests": float(np.percentile(model_prefix, 50)),
                         "lindley_p99_s_same_requests": float(np.percentile(model_prefix, 99)),
                         "same_final_costs": same},
                "modelled_whole_trace": {"solves_per_s": 1.0 / overall,
                                         "latency_p50_s": float(np.percentile(model_lat, 50)),
                                         "latency_p99_s": float(np.percentile(model_lat, 99)),
                                         "service_s_by_class": mean_cls,
                                         "how": "Lindley recursion over the whole trace with the "
                                                "live run's mean service time per class"}},
            "served_over_one_launch_per_solve": served_solves_s * overall,
            "server": stats, "clocks": clocks, "gpu_launches": launches,
            "h2d_bytes": h2d, "d2h_bytes": 8 * len(trace)}


def bench_serve(args, rank, world, local, cgo, torch, dist, barrier):
    G = args.generations if args.generations > 0 else workload("serve")[1]["G"]
    r = serve_run(args, cgo, torch, local, args.serve_seconds, G, args.seq_live_seconds, rank)
    if rank == 0:
        cfg = {k: v for k, v in r.items()
               if k not in ("desc", "clocks", "gpu_launches", "h2d_bytes", "d2h_bytes", "wall_s")}
        cfg["workload"] = r["desc"]
        line = {"metric": "served_solves_per_s", "value": r["solves_per_s"], "unit": "solves/s",
                "n_gpus": world, "steps": 1, "warmup": 4, "ms_per_step": 1000 * r["wall_s"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "int64", "data": "synthetic", "config": cfg,
                "e2e": {"value": r["solves_per_s"], "unit": "solves/s",
                        "h2d_bytes_per_step": r["h2d_bytes"], "d2h_bytes_per_step": r["d2h_bytes"]},
                "gpu_launches": r["gpu_launches"], "clocks": r["clocks"]}
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


# Roofline of the evolve kernel.  The hot-path table's measure is the
# distance gathers a move's delta needs (algorithmic, per operator
# application): swap 8, 2-opt 4, insertion 6, or-opt 6, 3-opt 6 entries of
# D; a QAP swap reads about 8n entries of F and D.  The operator mix and the
# steps per candidate come from the run's own counts (cgo_op_counts: every
# operator application of the whole solve).  The denominator is the random
# 16-bit gather rate of shared memory measured on this GPU by the library's
# microbenchmark (the triangle of D is staged in shared memory); the L2
# random-gather rate is reported beside it.  The integer-issue view counts
# the algorithmic integer operations of an evaluation against one
# instruction per lane per clock on every SM sub-partition.
D_GATHERS = {0: 8, 1: 4, 2: 6, 3: 6, 6: 6}
OPS_PHILOX = 100          # 10 rounds x (2 mul.lo + 2 mul.hi + 4 xor + 2 key add)
OPS_STEP = 120            # TSP: roulette 10 + decode 15 + 10 lookups x 5 + 10 gathers x 4 + sums 5
OPS_CAND = 20             # K roulette, argmin share, stats
OPS_QAP_K = 17            # QAP, per k of the O(n) swap delta: 9 loads, 2 multiplies, 6 add/sub


# DRAM bytes (read + write) of one full launch of the single-solve kernel on
# the tsp442 workload, from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum, one pass; profiles/evolve_tsp442_g200000_dram.md),
# valid only for the kernel sources it was taken on.
TRAFFIC_BYTES = 1269760 + 95232
TRAFFIC_SOURCES = "cbb57a7683deef50"


def kernel_sources_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("cgo_kernels.cu", "cgo_device.cuh", "cgo_internal.h"):
        with open(os.path.join(ROOT, "paper_2603_19163_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def op_mix(counts: dict) -> dict:
    """Measured operator mix and steps per candidate from whole-solve counts."""
    u, uk = counts["u_op"], counts["u_k"]
    apps, cands = sum(u), sum(uk)
    names = {0: "swap", 1: "2opt", 2: "insert", 3: "oropt", 4: "flip", 5: "reset", 6: "3opt",
             7: "segment", 8: "row_swap", 9: "row_merge", 10: "row_split"}
    return {"evals": cands, "applications": apps,
            "steps_per_eval": (uk[0] + 2 * uk[1] + 3 * uk[2]) / cands if cands else 0.0,
            "k_share": [x / cands for x in uk] if cands else [],
            "op_share": {names[i]: u[i] / apps for i in range(len(u)) if u[i]} if apps else {}}


def roofline(kernel_ms, prob, clocks):
    import torch
    from paper_2603_19163_gb300 import cgo
    counts = prob.op_counts()
    mix = op_mix(counts)
    evals = mix["evals"]
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    fmax = 2070.0
    try:
        pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        fmax = float(pk.get("sm_max_mhz", fmax))
    except (OSError, ValueError):
        pass
    model, n = int(prob.inst["model"]), int(prob.inst["n"])
    qap = model == 1
    sec = kernel_ms / 1000.0
    # algorithmic gathers of the whole launch, from the counted applications
    if qap:
        gathers = 8.0 * n * counts["u_op"][0]
    else:
        gathers = float(sum(D_GATHERS.get(i, 0) * counts["u_op"][i] for i in range(8)))
    # what the kernel executes: TSP evaluates all three steps of every
    # candidate (8 distance gathers and 8 tour reads each); QAP only the k
    # steps that count
    executed_d = 8.0 * n * counts["u_op"][0] if qap else 24.0 * evals
    g_peak, _ = cgo.gather_peak(0, 16)
    l2_peak, _ = cgo.gather_peak(1, 18)
    ek = mix["steps_per_eval"]
    step_ops = 25 + OPS_QAP_K * n if qap else OPS_STEP
    ops_eval = ek * (OPS_PHILOX + step_ops) + OPS_CAND
    alu_peak = sms * 128 * fmax * 1e6
    traffic = TRAFFIC_BYTES if (not qap and kernel_sources_hash() == TRAFFIC_SOURCES) else None
    achieved = gathers / sec
    return {"bound": "gather", "achieved": achieved / 1e9, "peak": g_peak / 1e9,
            "unit": "G gathers/s", "frac": achieved / g_peak, "traffic": traffic,
            "kernel": "evolve_kernel<%s>" % ("QAP" if qap else "TSP,int16"),
            "kernel_ms": kernel_ms, "evals_per_launch": evals,
            "gathers_per_launch": gathers, "gathers_per_eval": gathers / evals,
            "gathers_per_application": ("8n per QAP swap" if qap else
                                        "swap 8, 2opt 4, insert 6, oropt 6, 3opt 6"),
            "op_mix": mix,
            "peak_basis": "measured on this GPU: random 16-bit gathers from a 128 KB shared "
                          "buffer, one 1024-thread CTA per SM (cgo_gather_peak kind 0)",
            "executed_gathers_per_eval": executed_d / evals,
            "executed_frac": executed_d / sec / g_peak,
            "l2_random_gather_peak": l2_peak / 1e9,
            "alu": {"achieved": evals * ops_eval / sec / 1e12, "peak": alu_peak / 1e12,
                    "unit": "T int-ops/s", "frac": evals * ops_eval / sec / alu_peak,
                    "ops_per_eval": ops_eval,
                    "peak_basis": "%d SMs x 128 lanes x %.0f MHz" % (sms, fmax)}}


if __name__ == "__main__":
    main()
