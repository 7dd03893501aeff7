"""Search quality against exact optima (no GPU).

- TSP n = 20 of the plain single-solve workload (integer coordinates in
  [0, 1000]^2, P = 32, C = 128, swap / 2-opt / insertion at equal weight,
  2000 generations, the paper's seeds of Sec. 6.1): the Held-Karp optimum.
- 0-1 knapsack (weights and values in [1, 1000], capacity half the weight
  sum): the exact dynamic program.

Each exact solver is pinned by brute force on tiny instances first.  The GPU
path reproduces the oracle bit for bit, so the gaps hold for it too.
"""
import itertools

import numpy as np
import pytest

import instances as I
import oracle as O

SEEDS = (1, 42, 123, 456, 789, 2024)


def held_karp(D) -> int:
    """Shortest tour by dynamic programming over subsets (Held and Karp,
    1962): dp[S][j] = shortest path from city 0 through the set S ending at
    j, built by subset size."""
    D = np.asarray(D, np.int64)
    n = len(D)
    m = n - 1                            # cities 1 .. n-1 are bits 0 .. m-1
    full, inf = 1 << m, 1 << 60
    dp = np.full((full, m), inf, np.int64)
    for j in range(m):
        dp[1 << j, j] = D[0, j + 1]
    size = np.array([bin(x).count("1") for x in range(full)])
    masks = np.arange(full)
    for k in range(2, m + 1):
        layer = masks[size == k]
        for j in range(m):
            S = layer[(layer >> j) & 1 == 1]
            dp[S, j] = (dp[S ^ (1 << j)] + D[1:, j + 1][None, :]).min(axis=1)
    return int((dp[full - 1] + D[1:, 0]).min())


def knapsack_dp(w, v, cap) -> int:
    """Largest value within the capacity, dp[c] over capacities item by item."""
    dp = np.zeros(cap + 1, np.int64)
    for wi, vi in zip(w, v):
        wi, vi = int(wi), int(vi)
        if wi <= cap:
            dp[wi:] = np.maximum(dp[wi:], dp[:cap + 1 - wi] + vi)
    return int(dp[cap])


def test_held_karp_equals_brute_force():
    for idx in range(4):
        D = I.tsp_uniform(8, 700 + idx)["mat0"].tolist()
        bf = min(sum(D[p[i]][p[(i + 1) % 8]] for i in range(8))
                 for p in ([0] + list(q) for q in itertools.permutations(range(1, 8))))
        assert held_karp(D) == bf


def test_knapsack_dp_equals_brute_force():
    for idx in range(4):
        inst = I.knapsack(12, 710 + idx)
        w, v, cap = inst["vec0"], inst["vec1"], int(inst["capacity"])
        bf = max(sum(int(v[i]) for i in range(12) if (s >> i) & 1)
                 for s in range(1 << 12) if sum(int(w[i]) for i in range(12) if (s >> i) & 1) <= cap)
        assert knapsack_dp(w, v, cap) == bf


def test_tsp20_workload_reaches_the_held_karp_optimum():
    inst = I.tsp_uniform(20, 0)
    opt = held_karp(inst["mat0"])
    p = O.default_params(inst)
    p.update(P=32, C=128, op_mask=0b0111, w_op=[21845, 21845, 21845] + [0] * (O.NOPS - 3))
    for seed in SEEDS:
        st = O.solve(inst, p, seed, 2000)
        assert int(st["best_cost"].min()) == opt, seed


@pytest.mark.parametrize("n,idx", [(100, 800), (100, 801), (200, 800), (200, 801)])
def test_knapsack_gap_to_the_exact_optimum(n, idx):
    inst = I.knapsack(n, idx)
    opt = knapsack_dp(inst["vec0"], inst["vec1"], int(inst["capacity"]))
    p = O.default_params(inst)
    p.update(P=32, C=128)
    st = O.solve(inst, p, 1, 2000)
    best = -int(st["best_cost"].min())          # the search minimises -value (+ penalty)
    x = st["best_sol"][int(np.argmin(st["best_cost"]))]
    assert int(np.dot(x, inst["vec0"])) <= int(inst["capacity"])   # feasible
    assert best <= opt
    assert (opt - best) / opt <= 0.005                             # within 0.5%
