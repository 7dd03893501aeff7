"""Oracle pins for the oversampled and heuristic starts (Sec. 3.4.1-3.4.2).

The start permutations are checked against numpy's stable argsort of the row
and column sums; the oversampled population against the plain start of a
population K times larger (the same random starts), ordered by numpy's
lexicographic sort of (cost, index)."""
import numpy as np
import pytest

import instances as I
import oracle as O
from helpers import params_for


def expected_perms(inst):
    mats = {0: ["mat0"], 1: ["mat0", "mat1"]}.get(inst["model"], [])
    out = []
    for k in mats:
        M = np.asarray(inst[k], np.int64)
        for s in (M.sum(1), M.sum(0)):
            out.append(np.argsort(s, kind="stable"))
            out.append(np.argsort(-s, kind="stable"))
    return np.array(out, dtype=np.int32).reshape(len(out), inst["n"]) if out else np.zeros((0, inst["n"]), np.int32)


@pytest.mark.parametrize("maker", [lambda: I.tsp_uniform(31, 1), lambda: I.tsp_clustered(442, 0),
                                   lambda: I.qap_random(17, 2), lambda: I.qap_grid(64, 0)])
def test_heuristic_permutations_are_sorted_row_and_column_sums(maker):
    inst = maker()
    got = O.heuristic_perms(inst)
    want = expected_perms(inst)
    assert got.shape == want.shape == (4 * (1 + (inst["model"] == 1)), inst["n"])
    assert (got == want).all()
    for p in got:
        assert O.valid(inst, p)


def test_heuristic_permutations_only_for_square_matrices():
    for inst in (I.knapsack(50, 3), I.gap(30, 4, m=5), I.cvrptw(12, 5, vehicles=3, capacity=60)):
        assert O.heuristic_perms(inst).shape[0] == 0


def pool_order(costs):
    idx = np.arange(len(costs))
    return np.lexsort((idx, np.asarray(costs)))


@pytest.mark.parametrize("maker,K", [(lambda: I.tsp_uniform(40, 6), 4), (lambda: I.knapsack(70, 7), 3),
                                     (lambda: I.gap(25, 8, m=4), 2), (lambda: I.qap_random(11, 9), 5),
                                     (lambda: I.cvrptw(14, 10, vehicles=4, capacity=70), 4)])
def test_oversampled_start_keeps_the_cheapest_of_k_times_p(maker, K):
    inst = maker()
    P = 6
    big = O.solve(inst, params_for(inst, P=K * P), 3, 0)           # the K*P random starts
    st = O.solve(inst, params_for(inst, P=P, init_oversample=K), 3, 0)
    order = pool_order(big["cost"])[:P]
    assert (st["cur"] == big["cur"][order]).all()
    assert (st["best_sol"] == st["cur"]).all()
    assert (st["cost"] == big["cost"][order]).all() and (st["best_cost"] == st["cost"]).all()
    assert st["elite_prev"] == st["best_cost"].min()


@pytest.mark.parametrize("K", [1, 2])
def test_heuristic_starts_join_the_pool(K):
    inst = I.tsp_clustered(120, 11)
    P = 5
    rnd = O.solve(inst, params_for(inst, P=K * P), 4, 0)
    H = expected_perms(inst)
    pool = np.concatenate([rnd["cur"], H])
    costs = np.concatenate([rnd["cost"], [O.cost(inst, h) for h in H]])
    order = pool_order(costs)[:P]
    st = O.solve(inst, params_for(inst, P=P, init_oversample=K, init_heuristic=1), 4, 0)
    assert (st["cur"] == pool[order]).all()
    assert (st["cost"] == costs[order]).all()
    # on a clustered instance the sorted-row-sum tours beat every random one
    assert order[0] >= K * P


def test_plain_start_is_unchanged_by_k_one():
    inst = I.tsp_uniform(25, 12)
    a = O.solve(inst, params_for(inst, P=7), 9, 0)
    b = O.solve(inst, params_for(inst, P=7, init_oversample=1, init_heuristic=0), 9, 0)
    assert (a["cur"] == b["cur"]).all() and (a["cost"] == b["cost"]).all()
