"""Full-size runs, in the launch shapes the benchmark times, checked through
properties that hold at any size (the oracle cannot replay 200,000
generations of a 128-member population in a test): every member's current
and best solution is valid and its cost is the oracle's cost of that
solution, best <= current, the elite is the lowest best (lowest index on
ties), the generation counter and temperature are those of G coolings, and
the AOS weights are normalised Q16 values within their clamps.  Plus a TSP
too large for shared memory, where the triangle is read through L2, compared
with the oracle over a short prefix."""
import numpy as np
import pytest

import instances as I
import oracle as O
from helpers import assert_same_state, oracle_run, params_for

pytestmark = pytest.mark.gpu

TO, INS, OR = O.TWO_OPT, O.INSERT, O.OR_OPT


@pytest.fixture(scope="module")
def cgo():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_19163_gb300 import cgo as C
    return C


def cooled(T0: int, alpha: int, G: int) -> int:
    T = T0
    for _ in range(G):
        T = (T * alpha) >> 32
        if T == 0:
            break
    return T


def check_state(inst, p, st, best, where):
    P, G = p["P"], p["G"]
    assert st["g"] == G, where
    assert st["T"] == cooled(p["T0"], p["alpha"], G), where
    for q in range(P):
        cur, bs = st["cur"][q], st["best_sol"][q]
        assert O.valid(inst, cur) and O.valid(inst, bs), "%s member %d" % (where, q)
        assert O.cost(inst, cur) == st["cost"][q], "%s member %d cost" % (where, q)
        assert O.cost(inst, bs) == st["best_cost"][q], "%s member %d best" % (where, q)
        assert st["best_cost"][q] <= st["cost"][q], where
    e = int(np.argmin(st["best_cost"]))
    sol, c = best
    assert c == st["best_cost"][e] and (np.asarray(sol) == st["best_sol"][e]).all(), where
    # weights: after the last update the enabled operators' Q16 weights sum
    # to 2^16 less at most one unit each (floor division); disabled ones are 0
    on = [(p["op_mask"] >> i) & 1 for i in range(len(st["w_op"]))]
    w = [x for x, e in zip(st["w_op"], on) if e]
    assert all(x > 0 for x in w) and all(x == 0 for x, e in zip(st["w_op"], on) if not e), where
    assert 65536 - len(w) <= sum(w) <= 65536, (where, w)
    assert 65536 - 3 <= sum(st["w_k"]) <= 65536, (where, st["w_k"])


def test_tsp442_full_run(cgo):
    """The benchmark's single solve: n=442 clustered, P=128, C=128, 200,000
    generations, 4 warps per generation, two generations in flight."""
    inst = I.tsp_clustered(442, 0)
    p = params_for(inst, P=128, C=128, G=200000, op_mask=(1 << TO) | (1 << OR) | (1 << INS))
    prob = cgo.Problem(inst)
    prob.set_launch(8, 1, 4, 2)
    prob.solve(p, 1)
    assert prob.get_launch() == (8, 4, 1, 2)
    check_state(inst, p, prob.state(), prob.best(), "tsp442")


def test_qap64_full_run(cgo):
    inst = I.qap_grid(64, 0)
    p = params_for(inst, P=256, C=128, G=100000, ops=[O.SWAP])
    prob = cgo.Problem(inst)
    prob.solve(p, 1)
    check_state(inst, p, prob.state(), prob.best(), "qap64")


def test_batch512_full_run_sample(cgo):
    """The 512-instance batch at 20,000 generations; a stratified sample of
    32 instances checked member by member."""
    mix = [dict(x, tag=i) for i, x in enumerate(I.batch_mix(512, 0))]
    probs = [cgo.Problem(x) for x in mix]
    params = []
    for pr in probs:
        q = pr.default_params()
        q.update(P=32, C=128, G=20000)
        params.append(q)
    seeds = [1 + i for i in range(len(mix))]
    cgo.solve_batch(probs, params, seeds)
    for i in range(0, 512, 16):
        check_state(mix[i], params[i], probs[i].state(), probs[i].best(), "batch %d" % i)


def test_tsp442_islands_crossover_full_run(cgo):
    """The n=442 solve at 20,000 generations with every population step on:
    4 islands with hybrid migration every 1,000 generations, crossover at
    probability 0.1 per window, elite injection every 500 generations, and
    3-opt beside the benchmark's operators."""
    inst = I.tsp_clustered(442, 0)
    p = params_for(inst, P=128, C=128, G=20000,
                   op_mask=(1 << TO) | (1 << OR) | (1 << INS) | (1 << O.THREE_OPT),
                   islands=4, migrate_period=1000, migrate_strategy=2, migrate_n=4,
                   cross_q16=6554, elite_period=500)
    prob = cgo.Problem(inst)
    prob.solve(p, 3)
    check_state(inst, p, prob.state(), prob.best(), "tsp442 islands+crossover")


def test_batch_extra_operators_and_crossover_sample(cgo):
    """A 64-instance slice of the batch mix at 5,000 generations with the
    segment operators, 3-opt, crossover and ring migration enabled."""
    mix = [dict(x, tag=i) for i, x in enumerate(I.batch_mix(512, 0)[:64])]
    probs = [cgo.Problem(x) for x in mix]
    params = []
    for pr, x in zip(probs, mix):
        q = pr.default_params()
        extra = {I.TSP: 1 << O.THREE_OPT, I.KNAPSACK: 1 << O.SEGMENT, I.GAP: 1 << O.SEGMENT}
        q.update(P=32, C=128, G=5000, cross_q16=20000, islands=4, migrate_period=500)
        q["op_mask"] |= extra.get(x["model"], 0)
        params.append(q)
    cgo.solve_batch(probs, params, [7 + i for i in range(len(mix))])
    for i in range(0, 64, 4):
        check_state(mix[i], params[i], probs[i].state(), probs[i].best(), "batch %d" % i)


def test_tsp_beyond_shared_memory(cgo):
    """n = 1,500: the int16 triangle (2.25 MB) does not fit shared memory and
    is read through L2; the search matches the oracle over a prefix."""
    inst = I.tsp_uniform(1500, 77)
    p = params_for(inst, P=4, C=64, G=6, U=3)
    prob = cgo.Problem(inst)
    prob.solve(p, 5)
    assert prob.get_launch()[2] == 2          # staged through L2
    assert_same_state(prob.state(), oracle_run(inst, p, 5, 6), "tsp1500")


def test_atsp442_full_run(cgo):
    """An asymmetric n = 442 matrix in the benchmark's shape (P = 128, C = 128,
    20,000 generations, every permutation operator): the full matrix (390 KB
    of int16) is read through L2, each member keeps its edge-cost prefix
    sums, and every member's cost is the oracle's directed tour cost."""
    inst = I.tsp_asym(442, 5)
    p = params_for(inst, P=128, C=128, G=20000,
                   op_mask=(1 << O.SWAP) | (1 << TO) | (1 << OR) | (1 << INS) | (1 << O.THREE_OPT))
    prob = cgo.Problem(inst)
    prob.solve(p, 2)
    assert prob.get_launch()[2] == 2          # staged through L2
    check_state(inst, p, prob.state(), prob.best(), "atsp442")


def test_cvrptw100_lexicographic_full_run(cgo):
    """The 100-customer CVRPTW workload (P = 32, C = 128, 20,000 generations)
    in the lexicographic mode with every objective (vehicles, then distance
    with tolerance 50, then the longest route), the row level on: each
    member's cost is the oracle's key of its routes."""
    inst = dict(I.cvrptw(100, 0), lexicographic=[(O.LEX_VEHICLES, 0), (O.LEX_DISTANCE, 50),
                                                 (O.LEX_LONGEST, 0)])
    p = params_for(inst, P=32, C=128, G=20000)
    p["op_mask"] = ((1 << O.SWAP) | (1 << TO) | (1 << INS) | (1 << OR) | (1 << O.ROW_SWAP_OP) |
                    (1 << O.ROW_MERGE_OP) | (1 << O.ROW_SPLIT_OP))
    prob = cgo.Problem(inst)
    prob.solve(p, 4)
    check_state(inst, p, prob.state(), prob.best(), "cvrptw100 lexicographic")


def test_qap64_block_moves_full_run(cgo):
    """QAP n = 64 (P = 256, 2,000 generations) with every permutation
    operator: the block moves' exact deltas keep every cost the oracle's."""
    inst = I.qap_grid(64, 0)
    p = params_for(inst, P=256, C=128, G=2000, ops=[O.SWAP, TO, INS, OR, O.THREE_OPT])
    prob = cgo.Problem(inst)
    prob.solve(p, 1)
    check_state(inst, p, prob.state(), prob.best(), "qap64 block moves")
