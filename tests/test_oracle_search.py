"""Pins of the oracle's search as a whole (no GPU).

- brute-force optima of tiny instances of every model are reached by the
  search in all five of the paper's seeds (the style of Table "generality");
- state invariants: tracked costs equal full re-evaluation, bests are bests,
  solutions stay in their domain;
- resumability: running G1 then G2 generations equals running G1+G2;
- determinism across thread counts;
- stagnation reset and elite injection behave as stated in Sec. 4.2.3 and
  Sec. 3.4.3.
"""
import itertools

import numpy as np
import pytest

import instances as I
import oracle as O
from conftest import SEEDS


def equal_weights(p, ops):
    w = [0] * O.NOPS
    for o in ops:
        w[o] = 65536 // len(ops)
    p["w_op"] = w
    p["op_mask"] = sum(1 << o for o in ops)
    return p


# ------------------------------------------------ independent brute force
def bf_tsp(D):
    n = len(D)
    best = None
    for perm in itertools.permutations(range(1, n)):
        t = (0,) + perm
        c = sum(int(D[t[k]][t[(k + 1) % n]]) for k in range(n))
        best = c if best is None else min(best, c)
    return best


def bf_qap(F, D):
    n = len(F)
    best = None
    F = np.asarray(F, np.int64)
    D = np.asarray(D, np.int64)
    for perm in itertools.permutations(range(n)):
        p = np.array(perm)
        c = int((F * D[np.ix_(p, p)]).sum())
        best = c if best is None else min(best, c)
    return best


def bf_knapsack(w, v, cap):
    n = len(w)
    best = 0
    for bits in range(1 << n):
        x = [(bits >> i) & 1 for i in range(n)]
        W = sum(a * b for a, b in zip(w, x))
        if W <= cap:
            best = max(best, sum(a * b for a, b in zip(v, x)))
    return -best


def bf_gap(c, r, cap, lam):
    m, n = c.shape
    best = None
    for x in itertools.product(range(m), repeat=n):
        cost = sum(int(c[x[j], j]) for j in range(n))
        for a in range(m):
            load = sum(int(r[a, j]) for j in range(n) if x[j] == a)
            cost += lam * max(0, load - int(cap[a]))
        best = cost if best is None else min(best, cost)
    return best


def bf_cvrptw(inst, wd=1, wv=0, wl=0):
    """Brute-force optimum of the separator encoding; wd, wv, wl weigh
    distance, the vehicles used (routes that visit a customer) and the
    longest route's distance."""
    n, V = inst["n"], inst["vehicles"]
    d, dem, rdy, due, svc = (inst[k] for k in ("mat0", "vec0", "vec1", "vec2", "vec3"))
    Q = inst["capacity"]
    best = None
    for perm in itertools.permutations(range(n + V - 1)):
        routes, cur = [], []
        for s in perm:
            if s >= n:
                routes.append(cur)
                cur = []
            else:
                cur.append(s + 1)
        routes.append(cur)
        dist = excess = late = used = longest = 0
        for rt in routes:
            if not rt:
                continue
            used += 1
            t, load, prev, rd = 0, 0, 0, 0
            for c in rt:
                dist += int(d[prev][c])
                rd += int(d[prev][c])
                t = max(t + int(d[prev][c]), int(rdy[c]))
                late += max(0, t - int(due[c]))
                t += int(svc[c])
                load += int(dem[c])
                prev = c
            dist += int(d[prev][0])
            rd += int(d[prev][0])
            longest = max(longest, rd)
            t += int(d[prev][0])
            late += max(0, t - int(due[0]))
            excess += max(0, load - Q)
        cost = wd * dist + 100 * excess + 100 * late + wv * used + wl * longest
        best = cost if best is None else min(best, cost)
    return best


def _run(inst, p, seed, G):
    return O.solve(inst, p, seed, G, threads=2)


@pytest.mark.parametrize("seed", SEEDS)
def test_tsp_reaches_bruteforce_optimum(seed):
    inst = I.tsp_uniform(8, 100)
    opt = bf_tsp(inst["mat0"])
    p = O.default_params(inst)
    p.update(P=8, C=32)
    st = _run(inst, p, seed, 300)
    assert st["best_cost"].min() == opt


def test_asymmetric_tsp_cost_follows_the_tour_direction():
    # an asymmetric matrix: a tour and its reverse cost differently, each the
    # sum of its directed edges
    inst = I.tsp_asym(7, 3)
    D = inst["mat0"]
    t = [0, 3, 1, 6, 2, 5, 4]
    fwd = sum(int(D[t[k]][t[(k + 1) % 7]]) for k in range(7))
    bwd = sum(int(D[t[(k + 1) % 7]][t[k]]) for k in range(7))
    assert fwd != bwd
    assert O.cost(inst, t) == fwd
    assert O.cost(inst, t[::-1]) == bwd


@pytest.mark.parametrize("seed", SEEDS)
def test_asymmetric_tsp_reaches_bruteforce_optimum(seed):
    # every permutation operator, 2-opt and 3-opt included, on a matrix where
    # reversing a piece changes its inner edges
    inst = I.tsp_asym(8, 102)
    opt = bf_tsp(inst["mat0"])
    p = equal_weights(O.default_params(inst),
                      [O.SWAP, O.TWO_OPT, O.INSERT, O.OR_OPT, O.THREE_OPT])
    p.update(P=8, C=32)
    st = _run(inst, p, seed, 300)
    assert st["best_cost"].min() == opt
    x = st["best_sol"][int(np.argmin(st["best_cost"]))]
    assert O.cost(inst, x) == opt


@pytest.mark.parametrize("seed", SEEDS)
def test_qap_reaches_bruteforce_optimum(seed):
    inst = I.qap_random(7, 101)            # asymmetric, non-zero diagonals
    opt = bf_qap(inst["mat0"], inst["mat1"])
    p = equal_weights(O.default_params(inst), [O.SWAP, O.TWO_OPT, O.INSERT, O.OR_OPT])
    p.update(P=8, C=32)
    st = _run(inst, p, seed, 300)
    assert st["best_cost"].min() == opt


@pytest.mark.parametrize("seed", SEEDS)
def test_knapsack_reaches_bruteforce_optimum(seed):
    inst = I.knapsack(12, 102)
    opt = bf_knapsack(inst["vec0"].tolist(), inst["vec1"].tolist(), inst["capacity"])
    p = O.default_params(inst)
    p.update(P=8, C=32)
    st = _run(inst, p, seed, 300)
    assert st["best_cost"].min() == opt


@pytest.mark.parametrize("seed", SEEDS)
def test_gap_reaches_bruteforce_optimum(seed):
    inst = I.gap(7, 103, m=3)
    lam = 1 + int(inst["mat0"].max())
    opt = bf_gap(inst["mat0"], inst["mat1"], inst["vec0"], lam)
    p = O.default_params(inst)
    p.update(P=8, C=32)
    st = _run(inst, p, seed, 300)
    assert st["best_cost"].min() == opt


@pytest.mark.parametrize("seed", SEEDS)
@pytest.mark.parametrize("model", ["knapsack", "gap"])
def test_segment_operators_alone_reach_bruteforce_optimum(seed, model):
    """seg_flip (binary) and seg_reset (integer) as the only operator: every
    assignment stays reachable (a segment of 2 and one of 3 overlapping in
    all but one element change a single element), so the optimum is found."""
    if model == "knapsack":
        inst = I.knapsack(12, 102)
        opt = bf_knapsack(inst["vec0"].tolist(), inst["vec1"].tolist(), inst["capacity"])
    else:
        inst = I.gap(7, 103, m=3)
        opt = bf_gap(inst["mat0"], inst["mat1"], inst["vec0"], 1 + int(inst["mat0"].max()))
    p = equal_weights(O.default_params(inst), [O.SEGMENT])
    p.update(P=8, C=32)
    st = _run(inst, p, seed, 400)
    assert st["best_cost"].min() == opt


@pytest.mark.parametrize("seed", SEEDS)
@pytest.mark.parametrize("wd,wv", [(1, 10 ** 6), (10 ** 6, 1), (2, 35)])
def test_cvrptw_weighted_objectives_reach_bruteforce_optimum(seed, wd, wv):
    """Weighted distance and vehicle count (Sec. 6.8): a vehicle weight above
    any distance difference orders vehicles first (lexicographic), a distance
    weight above any vehicle count orders distance first; both and a mixed
    weighting reach the brute-force optimum of the weighted cost."""
    inst = dict(I.cvrptw(5, 104, vehicles=3, capacity=60, box=60, horizon=300, width=80),
                weight_distance=wd, weight_vehicles=wv)
    opt = bf_cvrptw(inst, wd, wv)
    p = O.default_params(inst)
    p.update(P=8, C=32)
    st = _run(inst, p, seed, 400)
    assert st["best_cost"].min() == opt


@pytest.mark.parametrize("seed", SEEDS)
@pytest.mark.parametrize("wd,wv,wl", [(1, 0, 3), (1, 10 ** 4, 2), (0, 0, 1)])
def test_cvrptw_longest_route_reaches_bruteforce_optimum(seed, wd, wv, wl):
    """The tri-objective VRP of Sec. 6.8 (distance, vehicles, longest route)
    as weights: the longest route's distance enters the cost with weight wl;
    the search reaches the brute-force optimum of the weighted cost (wd = 0
    takes the default distance weight 1)."""
    inst = dict(I.cvrptw(5, 104, vehicles=3, capacity=60, box=60, horizon=300, width=80),
                weight_distance=wd, weight_vehicles=wv, weight_longest=wl)
    opt = bf_cvrptw(inst, wd or 1, wv, wl)
    p = O.default_params(inst)
    p.update(P=8, C=32)
    st = _run(inst, p, seed, 400)
    assert st["best_cost"].min() == opt


@pytest.mark.parametrize("seed", SEEDS)
def test_cvrptw_reaches_bruteforce_optimum(seed):
    inst = I.cvrptw(5, 104, vehicles=2, capacity=60, box=60, horizon=300, width=80)
    opt = bf_cvrptw(inst)
    p = O.default_params(inst)
    p.update(P=8, C=32)
    st = _run(inst, p, seed, 300)
    assert st["best_cost"].min() == opt


# ------------------------------------------------------------ invariants
MODELS = {
    "tsp": lambda: I.tsp_uniform(13, 1),
    "qap": lambda: I.qap_random(9, 2),
    "knapsack": lambda: I.knapsack(40, 3),
    "gap": lambda: I.gap(30, 4, m=5),
    "cvrptw": lambda: I.cvrptw(12, 5, vehicles=3, capacity=100),
}


def check_state(inst, st):
    for p in range(st["P"]):
        assert O.valid(inst, st["cur"][p])
        assert O.valid(inst, st["best_sol"][p])
        assert O.cost(inst, st["cur"][p]) == st["cost"][p]
        assert O.cost(inst, st["best_sol"][p]) == st["best_cost"][p]
        assert st["best_cost"][p] <= st["cost"][p]


@pytest.mark.parametrize("name", sorted(MODELS))
def test_state_invariants_and_resume(name):
    inst = MODELS[name]()
    p = O.default_params(inst)
    p.update(P=6, C=40, U=7, elite_period=14)
    a = O.Solver(inst, p, 77)
    check_state(inst, a.state())
    bests = [a.state()["best_cost"].copy()]
    for G in (5, 9, 13, 1):
        a.run(G, threads=3)
        st = a.state()
        check_state(inst, st)
        assert (st["best_cost"] <= bests[-1]).all()
        bests.append(st["best_cost"].copy())
    b = O.Solver(inst, p, 77).run(28, threads=1).state()
    sa = a.state()
    for k in sa:
        if isinstance(sa[k], np.ndarray):
            assert (sa[k] == b[k]).all(), k
        else:
            assert sa[k] == b[k], k


def test_greedy_never_worsens():
    inst = I.tsp_uniform(15, 6)
    p = O.default_params(inst)
    p.update(P=4, C=16, T0=0)
    s = O.Solver(inst, p, 5)
    prev = s.state()["cost"].copy()
    for _ in range(30):
        s.run(1)
        cur = s.state()["cost"]
        assert (cur <= prev).all()
        prev = cur.copy()


def test_stagnation_resets_k_weights():
    # every tour of 3 cities (symmetric D) has the same length: the elite can
    # never improve, so each AOS update counts one more stagnant update and
    # the 5th resets w_K to (0.8, 0.15, 0.05)
    inst = I.tsp_uniform(3, 7)
    p = O.default_params(inst)
    p.update(P=3, C=8, U=10, stag_limit=5)
    s = O.Solver(inst, p, 1)
    s.run(40)
    st = s.state()
    assert st["stag"] == 4
    assert st["w_k"] != [52429, 9830, 3277]
    s.run(10)
    st = s.state()
    assert st["stag"] == 0 and st["w_k"] == [52429, 9830, 3277]


def test_elite_injection_replaces_worst():
    inst = I.tsp_uniform(25, 8)
    p0 = O.default_params(inst)
    p0.update(P=8, C=16, U=5, elite_period=0)
    p1 = dict(p0, elite_period=5)
    a = O.Solver(inst, p0, 3).run(5).state()
    b = O.Solver(inst, p1, 3).run(5).state()
    e = int(np.argmin(a["best_cost"]))            # lowest index on ties
    wv = int(np.argmax(a["cost"]))
    assert (b["cur"][wv] == a["best_sol"][e]).all()
    assert b["cost"][wv] == a["best_cost"][e]
    for q in range(8):
        if q != wv:
            assert (b["cur"][q] == a["cur"][q]).all() and b["cost"][q] == a["cost"][q]
    assert b["best_cost"][wv] == min(a["best_cost"][wv], a["best_cost"][e])


def test_thread_count_does_not_change_results():
    inst = I.gap(40, 9, m=6)
    p = O.default_params(inst)
    p.update(P=16, C=64)
    a = O.solve(inst, p, 11, 25, threads=1)
    b = O.solve(inst, p, 11, 25, threads=4)
    for k in ("cur", "cost", "best_sol", "best_cost"):
        assert (a[k] == b[k]).all()
    assert a["w_op"] == b["w_op"] and a["w_k"] == b["w_k"] and a["T"] == b["T"]


def test_default_priors_by_scale():
    # Table "weight_preset": or-opt prior 0.80 / 0.70 / 0.30 and 3-opt prior
    # 0.50 / 0.30 / 0.05 by scale, the O(1) operators 1.0, normalised to Q16
    # over the default mask (3-opt off by default, its prior kept on the same
    # scale for callers that enable it)
    for n, oro, tro in ((50, 52429, 32768), (200, 45875, 19661), (442, 19661, 3277)):
        inst = I.tsp_uniform(n, 10)
        p = O.default_params(inst)
        S = 3 * 65536 + oro
        assert p["w_op"][:4] == [(65536 << 16) // S] * 3 + [(oro << 16) // S]
        assert p["w_op"][4:] == [0, 0, (tro << 16) // S, 0, 0, 0, 0]   # no row level for TSP
        assert not (p["op_mask"] >> O.THREE_OPT) & 1
        assert p["w_k"] == [52429, 9830, 3277]
    # the segment operators of the binary and integer sets take the
    # segment-level (or-opt) preset, off by default: the element operator
    # alone normalises to 1.0
    for n, seg in ((60, 52429), (180, 45875), (600, 19661)):
        for inst in (I.knapsack(n, 11), I.gap(n, 12, m=4)):
            p = O.default_params(inst)
            el = O.FLIP if inst["model"] == 2 else O.PERTURB
            assert p["w_op"][el] == 65536 and p["w_op"][O.SEGMENT] == (seg << 16) // 65536
            assert not (p["op_mask"] >> O.SEGMENT) & 1


def test_init_distributions():
    # Fisher-Yates with j uniform in [0, i] gives every permutation of 3
    # elements with probability 1/6 (an off-by-one, j in [0, i-1], would give
    # only the two cyclic ones); binary bits are fair; integers are uniform
    inst = I.tsp_uniform(3, 11)
    p = O.default_params(inst)
    p.update(P=6000)
    st = O.Solver(inst, p, 99).state()
    counts = {}
    for row in st["cur"]:
        counts[tuple(row)] = counts.get(tuple(row), 0) + 1
    assert len(counts) == 6
    assert all(abs(c / 6000 - 1 / 6) < 0.025 for c in counts.values())
    kp = I.knapsack(50, 12)
    p = O.default_params(kp)
    p.update(P=200)
    st = O.Solver(kp, p, 5).state()
    assert abs(st["cur"].mean() - 0.5) < 0.02
    gp = I.gap(50, 13, m=7)
    p = O.default_params(gp)
    p.update(P=200)
    st = O.Solver(gp, p, 5).state()
    h = np.bincount(st["cur"].reshape(-1), minlength=7) / st["cur"].size
    assert st["cur"].min() == 0 and st["cur"].max() == 6
    assert np.abs(h - 1 / 7).max() < 0.02
