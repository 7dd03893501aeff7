"""GPU tests of the serving loop (continuous batching).

Requests of different models and sizes arrive while others are resident;
each result must be the same as solving it alone (and as the CPU oracle),
whatever the mix, the admission order, the slice length or the memory
budget.
"""
import threading
import time

import pytest

import instances as I
import oracle as O
from helpers import assert_same_state, oracle_run, params_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cgo():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_19163_gb300 import cgo as C
    C.lib()
    return C


def request_mix():
    return [
        (dict(I.tsp_uniform(30, 300), tag=1), dict(P=8, C=64, G=45)),
        (dict(I.knapsack(120, 301), tag=2), dict(P=6, C=96, G=33, U=4)),
        (dict(I.gap(40, 302, m=6), tag=3), dict(P=9, C=64, G=27, elite_period=10)),
        (dict(I.cvrptw(20, 303, vehicles=4, capacity=100), tag=4), dict(P=5, C=48, G=38)),
        (dict(I.qap_random(9, 304), tag=5), dict(P=7, C=40, G=21, ops=[O.SWAP])),
        (dict(I.tsp_uniform(90, 305), tag=6), dict(P=4, C=128, G=52)),
        (dict(I.tsp_uniform(12, 306), tag=7), dict(P=3, C=32, G=0)),
        (dict(I.knapsack(7, 307), tag=8), dict(P=2, C=16, G=9)),
        # oversampled and heuristic starts
        (dict(I.tsp_clustered(70, 308), tag=9), dict(P=5, C=64, G=31, init_oversample=4,
                                                     init_heuristic=1)),
        (dict(I.gap(25, 309, m=4), tag=10), dict(P=6, C=48, G=22, init_oversample=3)),
        # islands with ring migration
        (dict(I.tsp_uniform(40, 310), tag=11), dict(P=8, C=64, G=29, U=4, islands=4,
                                                    migrate_period=8, migrate_strategy=0)),
        # segment operators
        (dict(I.gap(35, 311, m=5), tag=12), dict(P=6, C=48, G=26, ops=[O.PERTURB, O.SEGMENT])),
        # crossover
        (dict(I.tsp_uniform(35, 312), tag=13), dict(P=6, C=48, G=24, U=4, cross_q16=50000)),
        # weighted CVRPTW objectives
        (dict(I.cvrptw(16, 313, vehicles=4, capacity=80), tag=14, weight_distance=2,
              weight_vehicles=300), dict(P=5, C=48, G=21)),
        # the longest route as a third objective
        (dict(I.cvrptw(15, 315, vehicles=5, capacity=80), tag=16, weight_longest=6),
         dict(P=5, C=48, G=22)),
        # the row level (routes as rows) beside the permutation operators
        (dict(I.cvrptw(18, 314, vehicles=6, capacity=80), tag=15),
         dict(P=6, C=64, G=26, U=4, ops=[O.SWAP, O.INSERT, O.OR_OPT] + [O.ROW_SWAP_OP, O.ROW_MERGE_OP, O.ROW_SPLIT_OP])),
        # asymmetric TSP; QAP with block moves
        (dict(I.tsp_asym(40, 316), tag=17), dict(P=6, C=64, G=25, U=4)),
        (dict(I.qap_random(10, 317), tag=18), dict(P=5, C=48, G=23, ops=[O.TWO_OPT, O.INSERT, O.OR_OPT])),
        # CVRPTW's lexicographic mode
        (dict(I.cvrptw(16, 318, vehicles=4, capacity=80), tag=19,
              lexicographic=[(O.LEX_VEHICLES, 0), (O.LEX_DISTANCE, 25)]), dict(P=5, C=48, G=22)),
    ]


def serve(C, items, slice_len, hbm_budget=8 << 30, stagger=0.0):
    srv = C.Server(max_slots=6, hbm_budget_bytes=hbm_budget, slice_generations=slice_len)
    probs, params, tickets = [], [], []
    for k, (inst, over) in enumerate(items):
        prob = C.Problem(inst)
        p = params_for(inst, **over)
        tickets.append(srv.submit(prob, p, 50 + k))
        probs.append(prob)
        params.append(p)
        if stagger and k % 3 == 2:
            time.sleep(stagger)
    results = [srv.wait(t, 60000) for t in tickets]
    stats = srv.stats()
    srv.close()
    return probs, params, results, stats


@pytest.mark.parametrize("slice_len", [2000, 7])
def test_served_results_equal_oracle(cgo, slice_len):
    items = request_mix()
    probs, params, results, stats = serve(cgo, items, slice_len, stagger=0.01)
    assert stats["completed"] == len(items)
    for k, ((inst, _), prob, p, (cost, lat)) in enumerate(zip(items, probs, params, results)):
        st = prob.state()
        assert_same_state(st, oracle_run(inst, p, 50 + k, p["G"]), "request %d" % k)
        assert cost == st["best_cost"].min() and lat >= 0.0


def test_slice_length_per_model(cgo):
    """Models that advance by different numbers of generations per slice
    (longer, shorter and the default) reach the same states as the oracle."""
    items = request_mix()
    srv = cgo.Server(max_slots=8, slice_generations=9,
                     slice_by_model={I.TSP: 40, I.KNAPSACK: 3, I.CVRPTW: 17})
    probs, params, tickets = [], [], []
    for k, (inst, over) in enumerate(items):
        prob = cgo.Problem(inst)
        p = params_for(inst, **over)
        tickets.append(srv.submit(prob, p, 50 + k))
        probs.append(prob)
        params.append(p)
    for t in tickets:
        srv.wait(t, 60000)
    stats = srv.stats()
    srv.close()
    assert stats["completed"] == len(items)
    for k, ((inst, _), prob, p) in enumerate(zip(items, probs, params)):
        assert_same_state(prob.state(), oracle_run(inst, p, 50 + k, p["G"]), "request %d" % k)


def test_slice_by_model_validated(cgo):
    with pytest.raises(Exception):
        cgo.Server(max_slots=2, slice_generations=5, slice_by_model={I.GAP: -1})


def test_served_equals_alone_under_tight_memory(cgo):
    """A budget that fits one request at a time serialises admission;
    results do not change."""
    items = request_mix()[:5]
    probs, params, results, stats = serve(cgo, items, 13, hbm_budget=1)
    for k, ((inst, _), prob, p) in enumerate(zip(items, probs, params)):
        alone = cgo.Problem(inst)
        alone.solve(p, 50 + k)
        assert_same_state(prob.state(), alone.state(), "request %d" % k)


def test_concurrent_clients(cgo):
    srv = cgo.Server(max_slots=16, slice_generations=11)
    items = [(dict(I.tsp_uniform(15 + 3 * k, 320 + k), tag=k), dict(P=4, C=32, G=30 + k))
             for k in range(12)]
    out = {}

    def client(lo, hi):
        for k in range(lo, hi):
            inst, over = items[k]
            prob = cgo.Problem(inst)
            p = params_for(inst, **over)
            t = srv.submit(prob, p, k + 1)
            out[k] = (prob, p, srv.wait(t, 60000))

    ths = [threading.Thread(target=client, args=(i * 4, i * 4 + 4)) for i in range(3)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    srv.close()
    for k, (inst, _) in enumerate(items):
        prob, p, _ = out[k]
        assert_same_state(prob.state(), oracle_run(inst, p, k + 1, p["G"]), "client req %d" % k)


def test_submit_errors(cgo):
    srv = cgo.Server(max_slots=2, smem_budget_bytes=1024, slice_generations=5)
    inst = I.tsp_uniform(40, 330)
    prob = cgo.Problem(inst)
    with pytest.raises(cgo.CgoError) as e:
        srv.submit(prob, params_for(inst, P=4, C=32, G=10), 1)
    assert e.value.status == cgo.ERR_UNSUPPORTED
    srv.close()
    srv = cgo.Server(max_slots=2, slice_generations=5)
    t = srv.submit(prob, params_for(inst, P=4, C=32, G=200), 1)
    with pytest.raises(cgo.CgoError) as e:
        prob.solve(params_for(inst, P=4, C=32, G=1), 1)       # in use by the server
    assert e.value.status == cgo.ERR_BUSY
    srv.wait(t, 60000)
    with pytest.raises(cgo.CgoError) as e:
        srv.wait(t, 10)                                        # already collected
    assert e.value.status == cgo.ERR_INVALID
    srv.close()
