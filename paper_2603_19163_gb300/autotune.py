"""Autotuner: launch shapes and serving populations, chosen by measurement.

Search results never depend on the launch shape (warps per member, members
per CTA, staging mode), so the tuner simply times short trial runs through
the C ABI and keeps the fastest shape; choices are cached by a shape key.
For serving it also picks the population per instance class: the largest
population from a ladder whose predicted device load at the offered arrival
rate stays under a utilisation target (the largest classes are halved first),
using the batched throughput measured per class.  For a batch it picks the
population per class by the L2-aware rule (batch_populations).
"""
from __future__ import annotations

import time

import numpy as np

from . import cgo as C

SMEM, GLOBAL = 1, 2


def _key(prob: "C.Problem", params: dict) -> tuple:
    inst = prob.inst
    return (int(inst["model"]), int(inst["n"]), int(inst.get("m", 0)), int(params["P"]),
            int(params["C"]))


class Autotuner:
    def __init__(self, trial_generations: int = 200):
        self.trial = int(trial_generations)
        self.cache_solve: dict = {}
        self.cache_batch: dict = {}
        self.log: list = []

    # ------------------------------------------------------------- single
    def solve_shapes(self, params: dict) -> list[tuple[int, int, int, int]]:
        """(warps per CTA, warps per member generation, staging, generations
        in flight) candidates for a single solve."""
        out = []
        xf = int(params.get("islands", 1)) > 1 or int(params.get("cross_q16", 0)) > 0
        for wpm in (4, 2, 1):
            if wpm * 32 > max(32, params["C"]) * 2:
                continue
            for ns in (4, 3, 2, 1):
                if ns >= 2 and params["C"] > 32 * wpm:
                    continue
                if ns > 2 and (wpm != 4 or xf):
                    continue
                for mpc in (1, 2):
                    if wpm * ns * mpc <= (16 if ns > 2 else 8) and (ns <= 2 or mpc == 1):
                        for staging in (SMEM, GLOBAL):
                            out.append((wpm * ns * mpc, wpm, staging, ns))
        return out

    def tune_solve(self, prob: "C.Problem", params: dict, seed: int = 1) -> tuple[int, int, int, int]:
        """Pick (warps per CTA, warps per member generation, staging,
        generations in flight) for cgo_solve of this problem and apply it;
        returns the choice.  Each shape is timed on the same stretch of the
        search, taken after a warm start of a tenth of the budget (the
        acceptance rate, and with it the cost of a generation, changes as the
        temperature falls)."""
        key = _key(prob, params)
        if key not in self.cache_solve:
            G = int(params["G"])
            warm = min(G // 10, 20000)
            trial = max(1, min(self.trial, G - warm))
            prob.set_launch(0, 0, 0, 0)
            prob.solve(dict(params, G=warm), seed)
            start = prob.state()
            best = None
            for shape in self.solve_shapes(params):
                try:
                    prob.set_launch(shape[0], staging=shape[2], wpm=shape[1], ns=shape[3])
                    prob.set_state(params, seed, start)
                    prob.solve_continue(trial)
                    ms, gens = prob.last_kernel_time()
                except C.CgoError:
                    continue
                rate = gens / max(ms, 1e-6)
                self.log.append(("solve", key, shape, rate))
                if best is None or rate > best[0]:
                    best = (rate, shape)
            if best is None:
                raise RuntimeError("no launch shape runs for %r" % (key,))
            self.cache_solve[key] = best[1]
        shape = self.cache_solve[key]
        prob.set_launch(shape[0], staging=shape[2], wpm=shape[1], ns=shape[3])
        return shape

    # ------------------------------------------------------------ batched
    def tune_batch(self, probs: list, params: list, sample: int = 16, seed0: int = 1) -> dict:
        """Pick warps per member for every model class of a batch (trial
        batches of a sample of each class) and apply it to every problem;
        returns {model: (wpm, evals_per_s)}."""
        classes: dict = {}
        for i, pr in enumerate(probs):
            classes.setdefault(int(pr.inst["model"]), []).append(i)
        out = {}
        for model, idx in classes.items():
            pick = idx[:: max(1, len(idx) // sample)][:sample]
            key = (model, len(pick), tuple(sorted(set(params[i]["P"] for i in pick))))
            if key not in self.cache_batch:
                best = None
                for wpm in (1, 2, 4):
                    sub = [probs[i] for i in pick]
                    for pr in sub:
                        pr.set_launch(0, 0, wpm)
                    trial = [dict(params[i], G=self.trial) for i in pick]
                    evals = sum(t["P"] * t["C"] * t["G"] for t in trial)
                    C.solve_batch(sub, trial, [seed0 + i for i in pick])    # warm
                    t0 = time.perf_counter()
                    C.solve_batch(sub, trial, [seed0 + i for i in pick])
                    rate = evals / (time.perf_counter() - t0)
                    self.log.append(("batch", key, wpm, rate))
                    if best is None or rate > best[1]:
                        best = (wpm, rate)
                self.cache_batch[key] = best
            wpm, rate = self.cache_batch[key]
            for i in idx:
                probs[i].set_launch(0, 0, wpm)
            out[model] = (wpm, rate)
        return out


def population_for_load(class_rate: dict, share: dict, arrivals_per_s: float,
                        generations: int, candidates: int, ladder=(32, 16, 8),
                        utilisation: float = 0.8) -> tuple[dict, float]:
    """Serving populations: start every class at the top of the ladder and,
    while the predicted device load (fraction of one GPU) exceeds the target,
    step down the class that contributes most.  class_rate: measured batched
    move evaluations per second of each class; share: its fraction of
    arrivals.  Returns ({class: P}, predicted load)."""
    P = {c: ladder[0] for c in class_rate}

    def load_of(c):
        return arrivals_per_s * share[c] * P[c] * candidates * generations / class_rate[c]

    while True:
        load = sum(load_of(c) for c in P)
        if load <= utilisation:
            return P, load
        c = max((c for c in P if P[c] > ladder[-1]), key=load_of, default=None)
        if c is None:
            return P, load
        P[c] = ladder[ladder.index(P[c]) + 1]


def slices_by_class(class_rate: dict, population: dict, candidates: int, generations: int,
                    base: int, fast: int) -> dict:
    """Serving slice lengths: every bucket advances in each slice and the
    slice lasts as long as its slowest bucket, so the class that advances
    slowest per request (class_rate / (population x candidates), request
    generations per second of a full batch) keeps `base` generations a slice
    and every other class takes `fast` (at most the request budget
    `generations`), finishing in fewer slices.  fast <= 0: `base` for all.
    Returns {class: generations per slice}."""
    speed = {c: class_rate[c] / (population[c] * candidates) for c in class_rate}
    slowest = min(speed, key=speed.get) if speed else None
    return {c: (base if c == slowest or fast <= 0 else min(generations, fast)) for c in speed}


def instance_data_bytes(inst: dict) -> int:
    """Device bytes of an instance's data as the library holds them (the
    caller's arrays, plus the int16 or int32 upper triangle of a TSP)."""
    b = sum(int(np.asarray(inst[k]).nbytes) for k in ("mat0", "mat1", "vec0", "vec1", "vec2", "vec3")
            if inst.get(k) is not None)
    if int(inst["model"]) == 0:
        n = int(inst["n"])
        b += n * (n + 1) // 2 * (2 if int(np.abs(np.asarray(inst["mat0"])).max()) < 32768 else 4)
    return b


def state_bytes(length: int, P: int) -> int:
    """Device bytes of a population's search state: current and best
    solutions (int32), current and best costs (int64)."""
    return 2 * P * length * 4 + 16 * P


def batch_populations(insts: list, l2_bytes: int, ladder=(64, 32, 16, 8)) -> tuple[dict, int]:
    """Populations of a batch by model class, L2-aware (the paper's adaptive
    population sizing, Sec. "Adaptive Population Sizing": the population is
    cut to the largest size whose working set the L2 cache sustains, in
    powers of two).  For a batch the working set is every instance's data
    plus every population's state, all resident across the time slices:
    start every class at the top of the ladder and, while the total exceeds
    L2, halve the class whose populations hold the most state.  Returns
    ({model: P}, working-set bytes)."""
    data = sum(instance_data_bytes(x) for x in insts)
    lens = {}
    for x in insts:
        n = int(x["n"])
        ln = n + int(x.get("vehicles", 1)) - 1 if int(x["model"]) == 4 else n
        lens.setdefault(int(x["model"]), []).append(ln)
    P = {m: ladder[0] for m in lens}

    def state_of(m):
        return sum(state_bytes(ln, P[m]) for ln in lens[m])

    while True:
        total = data + sum(state_of(m) for m in P)
        if total <= l2_bytes:
            return P, total
        m = max((m for m in P if P[m] > ladder[-1]), key=state_of, default=None)
        if m is None:
            return P, total
        P[m] = ladder[ladder.index(P[m]) + 1]
