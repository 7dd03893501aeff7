"""GPU parity of the batched persistent kernel (cgo_solve_batch).

A batch mixes models, sizes, populations and parameters; every problem's
final state must equal the CPU oracle's for the same inputs and seed, and
equal cgo_solve of that problem alone, bit for bit.  Time slices that cut AOS
windows in the middle must not change anything.
"""
import numpy as np
import pytest

import instances as I
import oracle as O
from helpers import assert_same_counts, assert_same_state, oracle_run, params_for

pytestmark = pytest.mark.gpu
SW = O.SWAP


@pytest.fixture(scope="module")
def cgo():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_19163_gb300 import cgo as C
    C.lib()
    return C


def mixed_batch():
    items = []
    for i, n in enumerate((9, 24, 57, 130)):
        items.append((dict(I.tsp_uniform(n, 200 + i), tag=i), dict(P=8 + 3 * i, C=64, G=37 + 11 * i)))
    items.append((dict(I.tsp_uniform(40, 210, box=90000), tag=9), dict(P=6, C=40, G=29)))  # int32 triangle
    items.append((dict(I.qap_random(10, 220), tag=10), dict(P=5, C=48, G=23, ops=[SW])))
    items.append((dict(I.qap_grid(16, 221), tag=11), dict(P=12, C=128, G=17, ops=[SW])))
    for i, n in enumerate((3, 70, 400)):
        items.append((dict(I.knapsack(n, 230 + i), tag=20 + i), dict(P=7 + i, C=96, G=31 + 5 * i, U=6)))
    for i, (n, m) in enumerate(((12, 3), (60, 10))):
        items.append((dict(I.gap(n, 240 + i, m=m), tag=30 + i), dict(P=9, C=80, G=41, U=4,
                                                                        elite_period=8)))
    items.append((dict(I.tsp_uniform(20, 250), tag=40), dict(P=4, C=32, G=0)))  # init only
    items.append((dict(I.cvrptw(25, 251, vehicles=5, capacity=120), tag=41), dict(P=8, C=64, G=33)))
    # oversampled and heuristic starts (Sec. 3.4.1-3.4.2)
    items.append((dict(I.tsp_clustered(90, 252), tag=42),
                  dict(P=6, C=64, G=21, init_oversample=3, init_heuristic=1)))
    items.append((dict(I.qap_random(12, 253), tag=43),
                  dict(P=5, C=48, G=19, ops=[SW], init_oversample=2, init_heuristic=1)))
    items.append((dict(I.knapsack(80, 254), tag=44), dict(P=7, C=64, G=15, init_oversample=4)))
    # 3-opt with the other permutation operators
    items.append((dict(I.tsp_uniform(70, 255), tag=45),
                  dict(P=6, C=96, G=23, ops=[0, 1, 2, 3, O.THREE_OPT])))
    items.append((dict(I.cvrptw(22, 256, vehicles=5, capacity=100), tag=46),
                  dict(P=5, C=64, G=19, ops=[0, 1, 2, 3, O.THREE_OPT])))
    # islands and migration (Sec. 3.4.3), members in one CTA
    items.append((dict(I.tsp_uniform(50, 257), tag=47),
                  dict(P=12, C=64, G=31, U=5, islands=4, migrate_period=10, migrate_strategy=2,
                       migrate_n=2, elite_period=15)))
    items.append((dict(I.gap(30, 258, m=5), tag=48),
                  dict(P=9, C=48, G=22, U=3, islands=3, migrate_period=6, migrate_strategy=1,
                       migrate_n=3)))
    # seg_flip / seg_reset beside the element operators
    items.append((dict(I.knapsack(150, 259), tag=49),
                  dict(P=8, C=64, G=25, ops=[O.FLIP, O.SEGMENT])))
    items.append((dict(I.gap(40, 260, m=6), tag=50),
                  dict(P=6, C=64, G=23, ops=[O.PERTURB, O.SEGMENT], w_k=[20000, 30000, 15536])))
    # crossover (with islands on one of them)
    items.append((dict(I.tsp_uniform(45, 261), tag=51),
                  dict(P=10, C=64, G=27, U=3, cross_q16=40000, islands=2, migrate_period=9)))
    items.append((dict(I.knapsack(90, 262), tag=52), dict(P=7, C=48, G=21, U=7, cross_q16=65536)))
    items.append((dict(I.cvrptw(16, 263, vehicles=4, capacity=80), tag=53),
                  dict(P=6, C=48, G=20, U=4, cross_q16=65536)))
    # the row level of CVRPTW (routes as rows), with and without the others
    items.append((dict(I.cvrptw(20, 265, vehicles=6, capacity=80), tag=55),
                  dict(P=6, C=64, G=26, U=4, ops=[O.SWAP, O.TWO_OPT, O.INSERT] + [O.ROW_SWAP_OP, O.ROW_MERGE_OP, O.ROW_SPLIT_OP])))
    items.append((dict(I.cvrptw(12, 266, vehicles=7, capacity=60), tag=56),
                  dict(P=5, C=48, G=21, ops=[O.ROW_SWAP_OP, O.ROW_MERGE_OP, O.ROW_SPLIT_OP], w_k=[20000, 30000, 15536])))
    # the longest route as a third objective
    items.append((dict(I.cvrptw(16, 267, vehicles=5, capacity=80), tag=57, weight_longest=4),
                  dict(P=6, C=48, G=23, U=4)))
    # weighted CVRPTW objectives (vehicles first)
    items.append((dict(I.cvrptw(18, 264, vehicles=5, capacity=90), tag=54, weight_vehicles=10 ** 6),
                  dict(P=6, C=48, G=22)))
    # asymmetric TSP (the full matrix, piece deltas) and QAP with every
    # permutation operator
    items.append((dict(I.tsp_asym(35, 268), tag=58), dict(P=6, C=64, G=27, U=4, cross_q16=30000)))
    items.append((dict(I.tsp_asym(80, 269, skew=50000), tag=59),
                  dict(P=5, C=48, G=19, ops=[0, 1, 2, 3, O.THREE_OPT])))
    items.append((dict(I.qap_random(13, 270), tag=60), dict(P=5, C=48, G=21, ops=[0, 1, 2, 3, O.THREE_OPT])))
    # CVRPTW's lexicographic mode
    items.append((dict(I.cvrptw(18, 271, vehicles=5, capacity=90), tag=61,
                       lexicographic=[(O.LEX_VEHICLES, 0), (O.LEX_DISTANCE, 30)]),
                  dict(P=6, C=48, G=24, U=4, cross_q16=30000)))
    items.append((dict(I.cvrptw(15, 272, vehicles=4, capacity=80), tag=62,
                       lexicographic=[(O.LEX_DISTANCE, 20), (O.LEX_VEHICLES, 0), (O.LEX_LONGEST, 5)]),
                  dict(P=5, C=64, G=21)))
    return items


def run_batch(C, items, seeds):
    probs = [C.Problem(inst) for inst, _ in items]
    params = [params_for(inst, **over) for inst, over in items]
    C.solve_batch(probs, params, seeds)
    return probs, params


@pytest.mark.parametrize("slice_len", [2000, 7])
def test_batch_matches_oracle(cgo, slice_len):
    cgo.lib().cgo_debug_inject(None, 3, slice_len)
    try:
        items = mixed_batch()
        seeds = [100 + i for i in range(len(items))]
        probs, params = run_batch(cgo, items, seeds)
        for (inst, _), prob, p, seed in zip(items, probs, params, seeds):
            o = oracle_run(inst, p, seed, p["G"])
            where = "model %d n %d slice %d" % (inst["model"], inst["n"], slice_len)
            assert_same_state(prob.state(), o, where)
            assert_same_counts(prob, o, where)
    finally:
        cgo.lib().cgo_debug_inject(None, 3, 2000)


def test_batch_equals_alone(cgo):
    items = mixed_batch()[:6]
    seeds = [7 * i + 1 for i in range(len(items))]
    probs, params = run_batch(cgo, items, seeds)
    for (inst, _), prob, p, seed in zip(items, probs, params, seeds):
        alone = cgo.Problem(inst)
        alone.solve(p, seed)
        assert_same_state(prob.state(), alone.state(), "alone vs batch")
        assert prob.best()[1] == alone.best()[1]


def test_batch_then_continue(cgo):
    """A batched solve leaves a normal state: continuing it alone equals the
    oracle run for the total generations."""
    inst = dict(I.tsp_uniform(33, 260), tag=3)
    p = params_for(inst, P=10, C=64, G=25)
    prob = cgo.Problem(inst)
    cgo.solve_batch([prob], [p], [5])
    prob.solve_continue(14)
    assert_same_state(prob.state(), oracle_run(inst, p, 5, 39), "batch + continue")


def test_batch_rejects_repeated_handles(cgo):
    inst = I.tsp_uniform(10, 261)
    prob = cgo.Problem(inst)
    p = params_for(inst, P=4, C=8, G=3)
    with pytest.raises(cgo.CgoError) as e:
        cgo.solve_batch([prob, prob], [p, p], [1, 2])
    assert e.value.status == cgo.ERR_BUSY


def test_config4_mix_sample_prefix(cgo):
    """Instances of the uneven 512-instance mix (TSP n~U[50,500], knapsack
    n~U[100,2000], GAP n~U[50,300]) in one batch, over a prefix of the
    generation budget, against the oracle."""
    mix = I.batch_mix(512, 0)
    pick = [0, 1, 2, 3, 5, 8, 13, 21, 34, 55]
    items = [(mix[i], dict(P=32, C=128, G=12)) for i in pick]
    seeds = [1 + i for i in pick]
    probs, params = run_batch(cgo, items, seeds)
    for (inst, _), prob, p, seed in zip(items, probs, params, seeds):
        assert_same_state(prob.state(), oracle_run(inst, p, seed, p["G"]),
                          "mix model %d n %d" % (inst["model"], inst["n"]))
