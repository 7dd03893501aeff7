"""GPU parity: the CUDA search (through the C ABI) against the CPU oracle.

Every case runs the same instance, parameters and seed on both sides and
compares the complete search state bit for bit: current and best solutions,
current and best costs, temperature, both AOS weight levels, stagnation
counter, the elite cost of the last update and the counts of the open AOS
window.  The work is integer, so the tolerance is zero.
"""
import numpy as np
import pytest

import instances as I
import oracle as O
from conftest import SEEDS
from helpers import assert_same_counts, assert_same_state, oracle_run, params_for

pytestmark = pytest.mark.gpu

SW, TO, INS, OR, TH = O.SWAP, O.TWO_OPT, O.INSERT, O.OR_OPT, O.THREE_OPT


@pytest.fixture(scope="module")
def cgo():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_19163_gb300 import cgo as C
    C.lib()
    return C


def run_both(C, inst, params, seed, warps=0, staging=0, wpm=0, ns=0):
    prob = C.Problem(inst)
    prob.set_launch(warps, staging, wpm, ns)
    prob.solve(params, seed)
    g = prob.state()
    o = oracle_run(inst, params, seed, params["G"])
    return prob, g, o


# --------------------------------------------------------------------- TSP
@pytest.mark.parametrize("ns", [1, 2])
@pytest.mark.parametrize("seed", SEEDS)
def test_tsp_n20_config(cgo, seed, ns):
    """TSP n=20, P=32, C=128, swap/2-opt/insertion at equal weight, T0=100,
    alpha=0.999, 2000 generations; one or two generations in flight."""
    inst = I.tsp_uniform(20, 0)
    p = params_for(inst, P=32, C=128, G=2000, ops=[SW, TO, INS])
    prob, g, o = run_both(cgo, inst, p, seed, ns=ns)
    assert prob.get_launch()[3] == ns
    assert_same_state(g, o, "tsp20 seed %d ns %d" % (seed, ns))
    assert_same_counts(prob, o, "tsp20 seed %d ns %d" % (seed, ns))
    assert sum(prob.op_counts()["u_k"]) == 32 * 128 * 2000


@pytest.mark.parametrize("n", [2, 3, 4, 5, 7, 33])
def test_tsp_small_n_all_ops(cgo, n):
    inst = I.tsp_uniform(n, 10 + n)
    p = params_for(inst, P=5, C=40, G=37, U=3, ops=[SW, TO, INS, OR, TH])
    _, g, o = run_both(cgo, inst, p, 3)
    assert_same_state(g, o, "n=%d" % n)


@pytest.mark.parametrize("ns,C", [(1, 100), (2, 64), (1, 300)])
def test_three_opt_tsp_and_cvrptw(cgo, ns, C):
    """3-opt (segment exchange) with the other operators, alone and composed,
    on TSP and on the routing model's separator sequence."""
    for inst in (I.tsp_clustered(90, 60), I.cvrptw(30, 61, vehicles=6, capacity=90)):
        for ops in ([TH], [SW, TO, INS, OR, TH]):
            p = params_for(inst, P=6, C=C, G=27, U=5, ops=ops, T0=30 << 32)
            _, g, o = run_both(cgo, inst, p, 5, ns=ns)
            assert_same_state(g, o, "model %d ops %s ns %d" % (inst["model"], ops, ns))


@pytest.mark.parametrize("op", [SW, TO, INS, OR, TH])
@pytest.mark.parametrize("kw", [(65536, 0, 0), (0, 65536, 0), (0, 0, 65536)])
def test_tsp_each_op_each_k(cgo, op, kw):
    inst = I.tsp_uniform(17, 21)
    p = params_for(inst, P=4, C=64, G=30, U=5, ops=[op], w_k=list(kw), stag_limit=0)
    _, g, o = run_both(cgo, inst, p, 9)
    assert_same_state(g, o, "op %d k %s" % (op, kw))


@pytest.mark.parametrize("C", [1, 31, 32, 33, 100, 257])
def test_tsp_candidate_counts(cgo, C):
    inst = I.tsp_uniform(29, 22)
    p = params_for(inst, P=6, C=C, G=23, U=4)
    _, g, o = run_both(cgo, inst, p, 5)
    assert_same_state(g, o, "C=%d" % C)


@pytest.mark.parametrize("P,warps,wpm", [(1, 0, 0), (3, 1, 1), (17, 2, 1), (9, 4, 2), (40, 8, 4),
                                         (64, 0, 0), (33, 8, 2), (5, 4, 4)])
def test_tsp_population_and_launch_shape(cgo, P, warps, wpm):
    """Results do not depend on warps per member or members per CTA."""
    inst = I.tsp_uniform(24, 23)
    p = params_for(inst, P=P, C=100, G=21, U=7, elite_period=14)
    _, g, o = run_both(cgo, inst, p, 8, warps=warps, wpm=wpm)
    assert_same_state(g, o, "P=%d warps=%d wpm=%d" % (P, warps, wpm))


@pytest.mark.parametrize("T0", [0, 40 << 32, 1 << 44])
@pytest.mark.parametrize("C,wpm,warps", [(1, 1, 0), (29, 1, 2), (32, 1, 8), (33, 2, 4), (64, 2, 8),
                                         (100, 4, 8)])
def test_two_generations_in_flight(cgo, C, wpm, warps, T0):
    """Generation g + 1 evaluated beside g: its result stands when g keeps
    the solution and is redone when g accepts (acceptance rare, mixed and
    almost certain across T0), over odd window lengths, windows that cross
    32-generation blocks and launches that end mid-window."""
    inst = I.tsp_uniform(37, 80)
    p = params_for(inst, P=9, C=C, G=45, U=7, elite_period=14, T0=T0, ops=[SW, TO, INS, OR])
    prob, g, o = run_both(cgo, inst, p, 11, warps=warps, wpm=wpm, ns=2)
    assert prob.get_launch()[3] == 2
    assert_same_state(g, o, "C=%d wpm=%d T0=%d" % (C, wpm, T0))
    prob.solve_continue(13)
    prob.solve_continue(1)
    prob.solve_continue(22)
    assert_same_state(prob.state(), oracle_run(inst, p, 11, 81), "continued")


def test_two_generations_in_flight_every_model(cgo):
    for inst, ops in ((I.tsp_uniform(31, 81), None), (I.qap_random(11, 82), [SW]),
                      (I.knapsack(90, 83), None), (I.gap(45, 84, m=7), None),
                      (I.cvrptw(14, 85, vehicles=4, capacity=80), None)):
        for T0 in (0, 30 << 32):
            over = dict(P=6, C=61, G=33, U=5, elite_period=10, T0=T0)
            if ops:
                over["ops"] = ops
            p = params_for(inst, **over)
            prob, g, o = run_both(cgo, inst, p, 4, wpm=2, ns=2)
            assert prob.get_launch()[3] == 2
            assert_same_state(g, o, "model %d T0 %d" % (inst["model"], T0))


@pytest.mark.parametrize("ns", [3, 4])
@pytest.mark.parametrize("T0", [0, 40 << 32, 1 << 44])
@pytest.mark.parametrize("C", [1, 77, 128])
def test_deep_generations_in_flight(cgo, ns, T0, C):
    """Three or four generations evaluated against the same solution and
    decided in order (later ones redone after an accepted move), over odd
    windows, windows across 32-generation blocks and split launches."""
    inst = I.tsp_uniform(37, 87)
    p = params_for(inst, P=9, C=C, G=45, U=7, elite_period=14, T0=T0, ops=[SW, TO, INS, OR])
    prob, g, o = run_both(cgo, inst, p, 11, wpm=4, ns=ns)
    assert prob.get_launch()[3] == ns and prob.get_launch()[0] == 4 * ns
    assert_same_state(g, o, "ns=%d C=%d T0=%d" % (ns, C, T0))
    prob.solve_continue(13)
    prob.solve_continue(1)
    prob.solve_continue(22)
    o81 = oracle_run(inst, p, 11, 81)
    assert_same_state(prob.state(), o81, "continued")
    assert_same_counts(prob, o81, "ns=%d" % ns)


@pytest.mark.parametrize("ns", [3, 4])
def test_deep_generations_every_model(cgo, ns):
    for inst, ops in ((I.tsp_uniform(31, 88), None), (I.qap_random(11, 89), [SW]),
                      (I.knapsack(90, 90), None), (I.gap(45, 91, m=7), None),
                      (I.cvrptw(14, 92, vehicles=4, capacity=80), None),
                      (I.tsp_clustered(90, 93), [SW, TO, INS, OR, TH])):
        for T0 in (0, 30 << 32):
            over = dict(P=6, C=128, G=33, U=5, elite_period=10, T0=T0)
            if ops:
                over["ops"] = ops
            p = params_for(inst, **over)
            prob, g, o = run_both(cgo, inst, p, 4, wpm=4, ns=ns)
            assert prob.get_launch()[3] == ns
            assert_same_state(g, o, "model %d T0 %d ns %d" % (inst["model"], T0, ns))


def test_deep_generations_limits(cgo):
    inst = I.tsp_uniform(20, 94)
    prob = cgo.Problem(inst)
    with pytest.raises(cgo.CgoError):
        prob.set_launch(0, 0, 2, 3)              # 3 in flight take 4 warps per generation
    with pytest.raises(cgo.CgoError):
        prob.set_launch(20, 0, 4, 4)             # beyond 16 warps per CTA
    prob.set_launch(0, 0, 4, 3)
    with pytest.raises(cgo.CgoError):            # more candidates than lanes
        prob.solve(params_for(inst, P=4, C=129, G=5), 1)
    with pytest.raises(cgo.CgoError):            # crossover kernels take at most two
        prob.solve(params_for(inst, P=4, C=128, G=5, cross_q16=30000), 1)


def test_two_generations_need_one_candidate_per_lane(cgo):
    inst = I.tsp_uniform(20, 86)
    p = params_for(inst, P=4, C=65, G=5)
    prob = cgo.Problem(inst)
    prob.set_launch(0, 0, 2, 2)
    with pytest.raises(cgo.CgoError):
        prob.solve(p, 1)


@pytest.mark.parametrize("wpm", [1, 2, 4])
def test_every_model_every_group_width(cgo, wpm):
    for inst, ops in ((I.tsp_uniform(31, 70), None), (I.qap_random(11, 71), [SW]),
                      (I.knapsack(90, 72), None), (I.gap(45, 73, m=7), None)):
        over = dict(P=6, C=150, G=26, U=5, elite_period=10)
        if ops:
            over["ops"] = ops
        p = params_for(inst, **over)
        _, g, o = run_both(cgo, inst, p, 4, wpm=wpm)
        assert_same_state(g, o, "model %d wpm %d" % (inst["model"], wpm))


KERNEL_TABLE_MODELS = [
    ("tsp int16", lambda: I.tsp_uniform(31, 74)),
    ("tsp int32", lambda: I.tsp_uniform(31, 75, box=90000)),
    ("atsp int16", lambda: I.tsp_asym(23, 76)),
    ("atsp int32", lambda: I.tsp_asym(23, 77, skew=60000)),
    ("qap", lambda: I.qap_random(11, 78)),
    ("cvrptw", lambda: I.cvrptw(14, 79, vehicles=4, capacity=80)),
    ("knapsack", lambda: I.knapsack(60, 80)),
    ("gap", lambda: I.gap(30, 81, m=5)),
]
# (warps per member, generations in flight, candidates): every launch shape
KERNEL_TABLE_SHAPES = [(1, 1, 150), (2, 1, 150), (4, 1, 150), (1, 2, 32), (2, 2, 64), (4, 2, 128),
                       (4, 3, 128), (4, 4, 128)]


@pytest.mark.parametrize("name,maker", KERNEL_TABLE_MODELS, ids=[m[0] for m in KERNEL_TABLE_MODELS])
def test_every_kernel_set_and_shape(cgo, name, maker):
    """Each model and matrix width, with no population step, crossover alone
    and islands with crossover, in every launch shape its kernels are built
    for: the host finds the kernel (built in one of the parallel units) and
    the search equals the oracle's.  Three and four generations in flight
    exist without population steps only, and not for the asymmetric TSP."""
    inst = maker()
    for xf, extra in ((0, {}), (1, dict(cross_q16=40000)),
                      (2, dict(cross_q16=40000, islands=2, migrate_period=5))):
        for wpm, ns, C in KERNEL_TABLE_SHAPES:
            p = params_for(inst, P=6, C=C, G=12, U=5, elite_period=10, **extra)
            prob = cgo.Problem(inst)
            prob.set_launch(wpm * ns, 0, wpm, ns)
            built = ns <= 2 or (xf == 0 and "atsp" not in name)
            if not built:
                with pytest.raises(cgo.CgoError) as e:
                    prob.solve(p, 3)
                assert e.value.status == cgo.ERR_UNSUPPORTED
                continue
            prob.solve(p, 3)
            assert prob.get_launch()[1:4:2] == (wpm, ns)
            assert_same_state(prob.state(), oracle_run(inst, p, 3, 12),
                              "%s xf %d wpm %d ns %d" % (name, xf, wpm, ns))


@pytest.mark.parametrize("staging", [1, 2])
def test_tsp_staging_modes(cgo, staging):
    inst = I.tsp_uniform(60, 24)
    p = params_for(inst, P=8, C=64, G=40)
    _, g, o = run_both(cgo, inst, p, 2, staging=staging)
    assert_same_state(g, o, "staging %d" % staging)


# ------------------------------------------------------- asymmetric TSP
@pytest.mark.parametrize("ns", [1, 2])
@pytest.mark.parametrize("n,skew", [(2, 50), (3, 50), (4, 300), (5, 300), (9, 300), (40, 300),
                                    (40, 60000)])
def test_atsp_all_operators(cgo, n, skew, ns):
    """TSP of an asymmetric matrix: every operator alone and composed, the
    candidate's tour as pieces of the current one over prefix sums of its
    forward and backward edge costs; 16-bit and (skew 60000) 32-bit entries."""
    inst = I.tsp_asym(n, 40 + n, skew=skew)
    assert (inst["mat0"] != inst["mat0"].T).any()
    p = params_for(inst, P=5, C=40, G=37, U=3, ops=[SW, TO, INS, OR, TH], T0=60 << 32)
    _, g, o = run_both(cgo, inst, p, 3, wpm=2 if ns == 2 else 0, ns=ns)
    assert_same_state(g, o, "atsp n=%d skew=%d ns=%d" % (n, skew, ns))


@pytest.mark.parametrize("op", [SW, TO, INS, OR, TH])
@pytest.mark.parametrize("kw", [(65536, 0, 0), (0, 65536, 0), (0, 0, 65536)])
def test_atsp_each_op_each_k(cgo, op, kw):
    inst = I.tsp_asym(17, 41)
    p = params_for(inst, P=4, C=64, G=30, U=5, ops=[op], w_k=list(kw), stag_limit=0)
    prob, g, o = run_both(cgo, inst, p, 9)
    assert_same_state(g, o, "atsp op %d k %s" % (op, kw))
    assert_same_counts(prob, o, "atsp op %d k %s" % (op, kw))


@pytest.mark.parametrize("staging", [1, 2])
@pytest.mark.parametrize("warps,wpm", [(0, 0), (2, 1), (8, 2), (8, 4)])
def test_atsp_staging_and_launch_shape(cgo, staging, warps, wpm):
    """The full matrix in shared or in global memory; one to eight member
    groups per CTA; elite injection, crossover, heuristic starts and islands
    (each rebuilds the prefix sums of the members it replaces)."""
    inst = I.tsp_asym(60, 42)
    p = params_for(inst, P=12, C=96, G=41, U=4, elite_period=8, cross_q16=40000,
                   init_heuristic=1, islands=3, migrate_period=8, migrate_strategy=1, migrate_n=2)
    _, g, o = run_both(cgo, inst, p, 4, warps=warps, staging=staging, wpm=wpm)
    assert_same_state(g, o, "atsp staging %d warps %d wpm %d" % (staging, warps, wpm))


def test_atsp_large_global_matrix(cgo):
    """n = 300: the 180 KB matrix of 16-bit entries; continued launches."""
    inst = I.tsp_asym(300, 43)
    p = params_for(inst, P=16, C=128, G=25, U=5)
    prob, g, o = run_both(cgo, inst, p, 6)
    assert_same_state(g, o, "atsp300")
    prob.solve_continue(14)
    assert_same_state(prob.state(), oracle_run(inst, p, 6, 39), "atsp300 continued")


def test_tsp_wide_distances_int32_triangle(cgo):
    inst = I.tsp_uniform(30, 25, box=100000)     # distances > 32767
    assert inst["mat0"].max() > 32767
    p = params_for(inst, P=8, C=64, G=40)
    _, g, o = run_both(cgo, inst, p, 4)
    assert_same_state(g, o, "int32 triangle")


@pytest.mark.parametrize("T0", [0, 1 << 32, 1 << 60])
def test_tsp_temperature_limits(cgo, T0):
    inst = I.tsp_uniform(19, 26)
    p = params_for(inst, P=6, C=32, G=30, T0=T0)
    _, g, o = run_both(cgo, inst, p, 6)
    assert_same_state(g, o, "T0=%d" % T0)


def test_tsp_stagnation_and_injection(cgo):
    inst = I.tsp_uniform(3, 27)                  # the elite never improves
    p = params_for(inst, P=5, C=8, G=70, U=5, stag_limit=2, elite_period=10)
    _, g, o = run_both(cgo, inst, p, 1)
    assert_same_state(g, o, "stagnation")
    inst = I.tsp_uniform(40, 28)
    p = params_for(inst, P=12, C=32, G=60, U=4, elite_period=8, stag_limit=1)
    _, g, o = run_both(cgo, inst, p, 7, warps=4)
    assert_same_state(g, o, "injection")


def test_tsp442_clustered_prefix(cgo):
    """The large single solve (n=442 clustered, P=128, 2-opt/or-opt/insertion
    with the 'Large' or-opt prior), launched as the benchmark launches it,
    compared over the first 60 generations."""
    inst = I.tsp_clustered(442, 0)
    p = params_for(inst, P=128, C=128, G=60, op_mask=(1 << TO) | (1 << OR) | (1 << INS))
    _, g, o = run_both(cgo, inst, p, 1)
    assert_same_state(g, o, "tsp442")
    for ns in (3, 4):
        _, g, _ = run_both(cgo, inst, p, 1, wpm=4, ns=ns)
        assert_same_state(g, o, "tsp442 ns %d" % ns)


# --------------------------------------------------------------------- QAP
@pytest.mark.parametrize("n", [3, 5, 9, 20])
def test_qap_asymmetric_diagonal(cgo, n):
    inst = I.qap_random(n, 30 + n)
    p = params_for(inst, P=6, C=40, G=25, U=5, ops=[SW])
    _, g, o = run_both(cgo, inst, p, 11)
    assert_same_state(g, o, "qap n=%d" % n)


@pytest.mark.parametrize("hi", [50, 200000])
def test_qap_wide_entries_take_64_bit_deltas(cgo, hi):
    """Small entries take the 32-bit swap delta, large ones the 64-bit one;
    both match the oracle."""
    inst = I.qap_random(23, 45, lo=-hi, hi=hi)
    p = params_for(inst, P=7, C=70, G=21, U=4, ops=[SW], T0=1 << 40)
    _, g, o = run_both(cgo, inst, p, 13)
    assert_same_state(g, o, "qap entries up to %d" % hi)


def test_qap64_grid_prefix(cgo):
    inst = I.qap_grid(64, 0)
    p = params_for(inst, P=256, C=128, G=8, ops=[SW])
    _, g, o = run_both(cgo, inst, p, 1)
    assert_same_state(g, o, "qap64")


@pytest.mark.parametrize("ops", [[TO], [INS], [OR], [TH], [SW, TO, INS, OR, TH]])
@pytest.mark.parametrize("kw", [(65536, 0, 0), (0, 0, 65536), None])
def test_qap_every_permutation_operator(cgo, ops, kw):
    """QAP with 2-opt, insertion, or-opt and 3-opt beside the swap: a block
    move's exact delta over the positions it changes (asymmetric F and D with
    a nonzero diagonal), alone and in k-step composites."""
    inst = I.qap_random(11, 39)
    over = dict(P=5, C=40, G=19, U=4, ops=ops, T0=20 << 32)
    if kw:
        over.update(w_k=list(kw), stag_limit=0)
    p = params_for(inst, **over)
    for ns, wpm in ((1, 1), (2, 2)):
        _, g, o = run_both(cgo, inst, p, 6, wpm=wpm, ns=ns)
        assert_same_state(g, o, "qap ops %s k %s ns %d" % (ops, kw, ns))


def test_qap_grid_block_moves(cgo):
    inst = I.qap_grid(36, 5)
    p = params_for(inst, P=8, C=64, G=12, ops=[SW, TO, INS, OR])
    _, g, o = run_both(cgo, inst, p, 2)
    assert_same_state(g, o, "qap36 block moves")


# ---------------------------------------------------------------- knapsack
@pytest.mark.parametrize("n,kw", [(2, None), (3, (0, 0, 65536)), (50, None), (200, (0, 65536, 0))])
def test_knapsack(cgo, n, kw):
    inst = I.knapsack(n, 40 + n)
    over = dict(P=7, C=70, G=33, U=6)
    if kw:
        over["w_k"] = list(kw)
    p = params_for(inst, **over)
    _, g, o = run_both(cgo, inst, p, 12)
    assert_same_state(g, o, "knapsack n=%d" % n)


def test_knapsack2000_prefix(cgo):
    inst = I.knapsack(2000, 49)
    p = params_for(inst, P=32, C=128, G=20)
    _, g, o = run_both(cgo, inst, p, 3)
    assert_same_state(g, o, "knapsack2000")


# --------------------------------------------------------------------- GAP
@pytest.mark.parametrize("n,m,kw", [(2, 2, None), (30, 5, (0, 0, 65536)), (80, 10, None)])
def test_gap(cgo, n, m, kw):
    inst = I.gap(n, 50 + n, m=m)
    over = dict(P=6, C=64, G=31, U=5, elite_period=10)
    if kw:
        over["w_k"] = list(kw)
    p = params_for(inst, **over)
    _, g, o = run_both(cgo, inst, p, 13)
    assert_same_state(g, o, "gap n=%d m=%d" % (n, m))


def test_gap300_prefix(cgo):
    inst = I.gap(300, 59, m=10)
    p = params_for(inst, P=32, C=128, G=20)
    _, g, o = run_both(cgo, inst, p, 3)
    assert_same_state(g, o, "gap300")


# ------------------------------------- seg_flip / seg_reset (segment level)
SEGMENT_K = [(65536, 0, 0), (0, 65536, 0), (0, 0, 65536), None]


@pytest.mark.parametrize("kw", SEGMENT_K)
@pytest.mark.parametrize("n", [2, 3, 5, 40, 300])
def test_knapsack_seg_flip(cgo, n, kw):
    """Segments of 2..5 items (clamped to n), alone and beside the flip, with
    one, two or three steps (overlapping segments of one candidate)."""
    inst = I.knapsack(n, 70 + n)
    for ops in ([O.SEGMENT], [O.FLIP, O.SEGMENT]):
        over = dict(P=6, C=80, G=29, U=4, ops=ops)
        if kw:
            over["w_k"] = list(kw)
        p = params_for(inst, **over)
        _, g, o = run_both(cgo, inst, p, 14)
        assert_same_state(g, o, "knapsack n=%d ops %s kw %s" % (n, ops, kw))


@pytest.mark.parametrize("kw", SEGMENT_K)
@pytest.mark.parametrize("n,m", [(2, 2), (4, 3), (7, 2), (30, 5), (120, 12)])
def test_gap_seg_reset(cgo, n, m, kw):
    inst = I.gap(n, 90 + n, m=m)
    for ops in ([O.SEGMENT], [O.PERTURB, O.SEGMENT]):
        over = dict(P=6, C=64, G=27, U=3, ops=ops, elite_period=9)
        if kw:
            over["w_k"] = list(kw)
        p = params_for(inst, **over)
        _, g, o = run_both(cgo, inst, p, 15)
        assert_same_state(g, o, "gap n=%d m=%d ops %s kw %s" % (n, m, ops, kw))


@pytest.mark.parametrize("ns,wpm", [(2, 1), (2, 2), (1, 4)])
def test_segment_operators_launch_shapes(cgo, ns, wpm):
    for inst, ops in ((I.knapsack(500, 97), [O.FLIP, O.SEGMENT]),
                      (I.gap(200, 98, m=8), [O.PERTURB, O.SEGMENT])):
        p = params_for(inst, P=9, C=32 * wpm, G=41, U=5, ops=ops)
        prob, g, o = run_both(cgo, inst, p, 16, wpm=wpm, ns=ns)
        assert prob.get_launch()[3] == ns
        assert_same_state(g, o, "model %d ns %d wpm %d" % (inst["model"], ns, wpm))


def test_segment_operator_needs_two_elements(cgo):
    inst = I.knapsack(1, 99)
    p = params_for(inst, P=3, C=8, G=5, ops=[O.SEGMENT])
    with pytest.raises(cgo.CgoError) as e:
        cgo.Problem(inst).solve(p, 1)
    assert e.value.status == cgo.ERR_INVALID


# ------------------------------------------------------------------ CVRPTW
@pytest.mark.parametrize("n,V,kw", [(2, 1, None), (5, 2, None), (12, 3, (0, 0, 65536)),
                                    (30, 6, None)])
def test_cvrptw(cgo, n, V, kw):
    inst = I.cvrptw(n, 80 + n, vehicles=V, capacity=60, box=60, horizon=400, width=80)
    over = dict(P=6, C=64, G=29, U=5, elite_period=10)
    if kw:
        over["w_k"] = list(kw)
    p = params_for(inst, **over)
    _, g, o = run_both(cgo, inst, p, 17)
    assert_same_state(g, o, "cvrptw n=%d V=%d" % (n, V))


@pytest.mark.parametrize("wd,wv", [(1, 10 ** 6), (10 ** 6, 1), (3, 40)])
@pytest.mark.parametrize("ns", [1, 2])
def test_cvrptw_weighted_objectives(cgo, wd, wv, ns):
    """Distance and vehicles used weighted (Sec. 6.8): vehicles first,
    distance first and a mixed weighting, every permutation operator."""
    for n, V in ((8, 3), (30, 6)):
        inst = dict(I.cvrptw(n, 340 + n, vehicles=V, capacity=70), weight_distance=wd,
                    weight_vehicles=wv)
        p = params_for(inst, P=8, C=64, G=33, U=4, ops=[SW, TO, INS, OR, TH], elite_period=8)
        _, g, o = run_both(cgo, inst, p, 17, ns=ns)
        assert_same_state(g, o, "n %d wd %d wv %d ns %d" % (n, wd, wv, ns))


def test_cvrptw_weights_validated(cgo):
    base = I.cvrptw(6, 349, vehicles=2, capacity=60)
    for bad in (dict(weight_distance=-1), dict(weight_vehicles=-5), dict(weight_distance=1 << 58)):
        with pytest.raises(cgo.CgoError) as e:
            cgo.Problem(dict(base, **bad))
        assert e.value.status == cgo.ERR_INVALID, bad


@pytest.mark.parametrize("C,wpm,kw", [(150, 1, None), (150, 2, (20000, 30000, 15536)),
                                       (100, 4, None), (300, 1, (0, 0, 65536)), (256, 1, (0, 65536, 0))])
def test_cvrptw_candidates_per_lane(cgo, C, wpm, kw):
    """Several candidates per lane: one-step candidates in place, multi-step
    ones gathered over the warp (up to 8 per lane), else one by one."""
    inst = I.cvrptw(40, 91, vehicles=9, capacity=90)
    over = dict(P=5, C=C, G=31, U=6, elite_period=12, T0=20 << 32)
    if kw:
        over["w_k"] = list(kw)
    p = params_for(inst, **over)
    _, g, o = run_both(cgo, inst, p, 23, wpm=wpm, ns=1)
    assert_same_state(g, o, "cvrptw C=%d wpm=%d" % (C, wpm))


@pytest.mark.parametrize("C,U,ops,extra", [
    (128, 5, None, {}),                                   # four per lane, default operators
    (128, 5, [TO], {}),                                   # reversals alone: every walk class
    (256, 5, [TO, INS], {}),                              # eight per lane, byte counts at their bound
    (256, 6, [TO, INS], {}),                              # eight per lane, full-width counts
    (64, 5, [SW, INS, OR], {"weight_longest": 2}),        # longest route: any one-step move gathers
    (96, 4, [SW, TO, INS, OR], {"lexicographic": [(1, 0), (2, 10), (0, 20)]}),
])
def test_cvrptw_gathered_walk_classes(cgo, C, U, ops, extra):
    """Several candidates per lane on 100 customers and 25 routes (sequences
    of 124 symbols): candidates whose routes span more than 24 positions
    (multi-step hulls, reversals, and with the longest route any move) are
    evaluated after the in-place ones, gathered over the warp in three
    classes, so a lane may evaluate twice its share in one generation."""
    inst = dict(I.cvrptw(100, 97, vehicles=25, capacity=200), **extra)
    over = dict(P=4, C=C, G=25, U=U, T0=30 << 32)
    if ops:
        over["ops"] = ops
    p = params_for(inst, **over)
    prob, g, o = run_both(cgo, inst, p, 19, wpm=1, ns=1)
    where = "C %d U %d ops %s %s" % (C, U, ops, sorted(extra))
    assert_same_state(g, o, where)
    assert_same_counts(prob, o, where)


def test_cvrptw100_prefix(cgo):
    """The serving workload's routing class: 100 customers, 25 vehicles."""
    inst = I.cvrptw(100, 90)
    p = params_for(inst, P=16, C=128, G=15)
    _, g, o = run_both(cgo, inst, p, 2)
    assert_same_state(g, o, "cvrptw100")


# ------------------------------------------------- oversampled / heuristic start
@pytest.mark.parametrize("K,heur", [(2, 0), (4, 0), (1, 1), (3, 1), (64, 1)])
def test_pool_start_every_model(cgo, K, heur):
    """Sec. 3.4.1-3.4.2: the P cheapest of K*P random starts (plus the
    row/column-sum permutations for TSP and QAP) start the search."""
    cases = [(I.tsp_clustered(60, 300), None), (I.qap_random(13, 301), [SW]),
             (I.knapsack(70, 302), None), (I.gap(30, 303, m=5), None),
             (I.cvrptw(16, 304, vehicles=4, capacity=80), None)]
    for inst, ops in cases:
        P = 3 if K == 64 else 7
        over = dict(P=P, C=48, G=13, U=4, init_oversample=K, init_heuristic=heur)
        if ops:
            over["ops"] = ops
        p = params_for(inst, **over)
        _, g, o = run_both(cgo, inst, p, 9)
        assert_same_state(g, o, "model %d K %d heur %d" % (inst["model"], K, heur))


def test_pool_start_init_only_and_limits(cgo):
    inst = I.tsp_clustered(200, 305)
    p = params_for(inst, P=20, C=32, G=0, init_oversample=5, init_heuristic=1)
    prob, g, o = run_both(cgo, inst, p, 2)
    assert_same_state(g, o, "init only")
    prob2 = cgo.Problem(inst)
    for bad in (dict(init_oversample=65), dict(init_oversample=64, P=257), dict(init_heuristic=2)):
        with pytest.raises(cgo.CgoError) as e:
            prob2.solve(dict(p, **bad), 1)
        assert e.value.status == cgo.ERR_INVALID


# ------------------------------------------------------ islands and migration
ISLAND_CASES = [(I.tsp_uniform(30, 310), None), (I.qap_random(11, 311), [SW]),
                (I.knapsack(60, 312), None), (I.gap(25, 313, m=4), None),
                (I.cvrptw(14, 314, vehicles=4, capacity=70), None)]


@pytest.mark.parametrize("strategy,n", [(0, 1), (1, 1), (1, 3), (2, 2)])
@pytest.mark.parametrize("ns", [1, 2])
def test_islands_every_model(cgo, strategy, n, ns):
    """Sec. 3.4.3: ring, top-N and hybrid migration between 3 islands of 4
    members every 2 AOS windows, elite injection at every third window (both
    at generation 30)."""
    for inst, ops in ISLAND_CASES:
        over = dict(P=12, C=64, G=37, U=5, islands=3, migrate_period=10, migrate_strategy=strategy,
                    migrate_n=n, elite_period=15)
        if ops:
            over["ops"] = ops
        p = params_for(inst, **over)
        _, g, o = run_both(cgo, inst, p, 4, ns=ns)
        assert_same_state(g, o, "model %d strategy %d n %d ns %d" % (inst["model"], strategy, n, ns))


@pytest.mark.parametrize("warps,wpm", [(1, 1), (2, 1), (8, 2), (8, 4)])
def test_islands_across_ctas(cgo, warps, wpm):
    """Islands whose members sit in different CTAs (one to eight member groups
    per CTA), so that migration crosses the cooperative grid barrier."""
    inst = I.tsp_clustered(60, 315)
    for strategy, n in ((0, 1), (1, 4), (2, 2)):
        p = params_for(inst, P=48, C=96, G=61, U=4, islands=6, migrate_period=12,
                       migrate_strategy=strategy, migrate_n=n, elite_period=8)
        _, g, o = run_both(cgo, inst, p, 11, warps=warps, wpm=wpm)
        assert_same_state(g, o, "strategy %d warps %d wpm %d" % (strategy, warps, wpm))


def test_islands_degenerate_shapes(cgo):
    """One member per island (ring: each member takes its predecessor's best)
    and top-N with N = P/I (every member of every island is replaced)."""
    inst = I.tsp_uniform(25, 316)
    for over in (dict(P=5, islands=5, migrate_strategy=0), dict(P=6, islands=2, migrate_strategy=1, migrate_n=3),
                 dict(P=8, islands=8, migrate_strategy=2, migrate_n=1)):
        p = params_for(inst, C=40, G=25, U=3, migrate_period=3, **over)
        _, g, o = run_both(cgo, inst, p, 6)
        assert_same_state(g, o, str(over))


# ----------------------------------------------- lexicographic CVRPTW (R37)
LEX_MODES = [[(0, 0), (1, 0)], [(0, 50), (1, 0)], [(1, 0), (0, 100)], [(0, 0), (1, 0), (2, 0)],
             [(1, 0), (0, 30), (2, 20)], [(2, 15)]]


@pytest.mark.parametrize("ns", [1, 2])
@pytest.mark.parametrize("lex", LEX_MODES)
def test_cvrptw_lexicographic_mode(cgo, lex, ns):
    """The lexicographic mode (penalty first, then each objective in buckets
    of width tolerance + 1): the kernels' packed route cost turned into the
    order's key for every candidate; the element operators, 3-opt and the
    row level, at every k level, one and two generations in flight."""
    inst = dict(I.cvrptw(30, 70, vehicles=6, capacity=90), lexicographic=lex)
    ops = [SW, TO, INS, OR, TH, O.ROW_SWAP_OP, O.ROW_MERGE_OP, O.ROW_SPLIT_OP]
    p = params_for(inst, P=6, C=64, G=31, U=4, ops=ops, T0=30 << 32)
    prob, g, o = run_both(cgo, inst, p, 5, wpm=2 if ns == 2 else 0, ns=ns)
    assert_same_state(g, o, "lex %s ns %d" % (lex, ns))
    assert_same_counts(prob, o, "lex %s ns %d" % (lex, ns))


def test_cvrptw_lexicographic_population_steps(cgo):
    """With crossover (children costed as keys), islands and injection."""
    inst = dict(I.cvrptw(25, 71, vehicles=5, capacity=100), lexicographic=[(1, 0), (0, 40)])
    p = params_for(inst, P=12, C=64, G=37, U=3, cross_q16=50000, islands=3, migrate_period=6,
                   migrate_strategy=1, migrate_n=2, elite_period=9, init_oversample=2)
    _, g, o = run_both(cgo, inst, p, 8)
    assert_same_state(g, o, "lex population steps")


def test_cvrptw_lexicographic_invalid(cgo):
    base = I.cvrptw(12, 72, vehicles=3, capacity=80)
    for lex, extra in (([(0, 0), (0, 5)], {}), ([(3, 0)], {}), ([(0, -1)], {}),
                       ([(0, 0)], dict(weight_vehicles=5)), ([(0, 0)] * 4, {})):
        with pytest.raises(cgo.CgoError) as e:
            cgo.Problem(dict(base, lexicographic=lex, **extra))
        assert e.value.status == cgo.ERR_INVALID, lex
    # objectives too wide for the packed cost
    wide = dict(I.cvrptw(30, 73, vehicles=6, capacity=90, box=1000000, horizon=10 ** 9),
                lexicographic=[(0, 0), (1, 0), (2, 0)])
    with pytest.raises(cgo.CgoError) as e:
        cgo.Problem(wide)
    assert e.value.status == cgo.ERR_UNSUPPORTED


# ------------------------------------------------------------------ crossover
CROSS_CASES = [(I.tsp_uniform(30, 320), None), (I.qap_random(11, 321), None),
               (I.tsp_asym(30, 329), None),
               (I.knapsack(60, 322), None), (I.gap(25, 323, m=4), None),
               (I.cvrptw(14, 324, vehicles=4, capacity=70), None)]


@pytest.mark.parametrize("q16", [65536, 30000])
@pytest.mark.parametrize("ns", [1, 2])
def test_crossover_every_model(cgo, q16, ns):
    """Order crossover (permutations) and uniform crossover (binary,
    integer) at every AOS window end, certain or with probability 0.46;
    elite injection in the same windows as every third crossover."""
    for inst, ops in CROSS_CASES:
        over = dict(P=8, C=64, G=37, U=5, cross_q16=q16, elite_period=15)
        if ops:
            over["ops"] = ops
        p = params_for(inst, **over)
        _, g, o = run_both(cgo, inst, p, 5, ns=ns)
        assert_same_state(g, o, "model %d q16 %d ns %d" % (inst["model"], q16, ns))


@pytest.mark.parametrize("warps,wpm", [(1, 1), (2, 1), (8, 2), (8, 4)])
def test_crossover_across_ctas_with_islands(cgo, warps, wpm):
    """Partners in other CTAs; migration and crossover in the same windows."""
    inst = I.tsp_clustered(80, 325)
    p = params_for(inst, P=24, C=96, G=49, U=4, cross_q16=50000, islands=4, migrate_period=8,
                   migrate_strategy=2, migrate_n=2, elite_period=12)
    _, g, o = run_both(cgo, inst, p, 12, warps=warps, wpm=wpm)
    assert_same_state(g, o, "warps %d wpm %d" % (warps, wpm))
    inst = I.knapsack(300, 326)
    p = params_for(inst, P=20, C=64, G=31, U=3, cross_q16=65536, ops=[O.FLIP, O.SEGMENT])
    _, g, o = run_both(cgo, inst, p, 13, warps=warps, wpm=wpm)
    assert_same_state(g, o, "knapsack warps %d wpm %d" % (warps, wpm))


def test_crossover_edge_cases(cgo):
    """One member (nothing to cross with), two members (each other's only
    partner), a permutation of length 2 and a launch that ends mid-window."""
    for inst, P, G in ((I.tsp_uniform(12, 327), 1, 20), (I.tsp_uniform(12, 328), 2, 20),
                       (I.tsp_uniform(2, 329), 3, 15), (I.gap(9, 330, m=3), 5, 23)):
        p = params_for(inst, P=P, C=16, G=G, U=5, cross_q16=65536)
        _, g, o = run_both(cgo, inst, p, 14)
        assert_same_state(g, o, "n %d P %d" % (inst["n"], P))
    prob = cgo.Problem(I.tsp_uniform(12, 331))
    with pytest.raises(cgo.CgoError) as e:
        prob.solve(params_for(I.tsp_uniform(12, 331), P=4, C=16, G=5, cross_q16=65537), 1)
    assert e.value.status == cgo.ERR_INVALID


@pytest.mark.parametrize("ns,warps,wpm", [(1, 0, 0), (2, 4, 2), (1, 8, 1)])
def test_crossover_parent_rows_across_launches(cgo, ns, warps, wpm):
    """Crossover parents are each member's best as it stood before the
    window's crossovers.  Many windows in which bests fall by moves, by
    children, by migrants and by injected elites, in launches that end
    inside windows and at their ends (each launch starts its parent rows
    afresh), with one and two generations in flight."""
    for inst in (I.tsp_clustered(70, 332), I.cvrptw(15, 333, vehicles=4, capacity=80),
                 I.knapsack(90, 334)):
        p = params_for(inst, P=16, C=64, G=33, U=3, cross_q16=52000, elite_period=9, islands=4,
                       migrate_period=6, migrate_strategy=2, migrate_n=2, T0=50 << 32)
        prob, g, o = run_both(cgo, inst, p, 15, warps=warps, wpm=wpm, ns=ns)
        assert_same_state(g, o, "model %d ns %d" % (inst["model"], ns))
        G = 33
        for extra in (1, 2, 3, 7, 12):
            prob.solve_continue(extra)
            G += extra
            assert_same_state(prob.state(), oracle_run(inst, p, 15, G),
                              "model %d ns %d G %d" % (inst["model"], ns, G))


def test_islands_invalid_parameters(cgo):
    inst = I.tsp_uniform(20, 317)
    p = params_for(inst, P=12, C=32, G=10, U=5, islands=3, migrate_period=10)
    prob = cgo.Problem(inst)
    for bad, status in ((dict(islands=5), cgo.ERR_INVALID), (dict(migrate_period=7), cgo.ERR_UNSUPPORTED),
                        (dict(migrate_strategy=3), cgo.ERR_INVALID),
                        (dict(migrate_strategy=1, migrate_n=0), cgo.ERR_INVALID),
                        (dict(migrate_strategy=1, migrate_n=5), cgo.ERR_INVALID)):
        with pytest.raises(cgo.CgoError) as e:
            prob.solve(dict(p, **bad), 1)
        assert e.value.status == status, bad
    # islands without a migration period is one population
    q = dict(p, migrate_period=0)
    _, g, o = run_both(cgo, inst, q, 2)
    assert_same_state(g, o, "no migration")


# ------------------------------------------------------------ row level
ROWS = [O.ROW_SWAP_OP, O.ROW_MERGE_OP, O.ROW_SPLIT_OP]


@pytest.mark.parametrize("ns", [1, 2])
@pytest.mark.parametrize("kw", [(65536, 0, 0), (0, 65536, 0), (0, 0, 65536), None])
@pytest.mark.parametrize("ops", [ROWS, [SW, TO, INS, OR, TH] + ROWS, [INS, O.ROW_SPLIT_OP],
                                 [O.ROW_SWAP_OP], [O.ROW_MERGE_OP, TO]])
def test_cvrptw_row_operators(cgo, ns, kw, ops):
    """The row level of CVRPTW's separator sequence (row_swap, row_merge,
    row_split; Table "operators"), alone and composed with the permutation
    operators in k-step moves: a row step after earlier steps finds its
    routes in the sequence those steps left."""
    inst = I.cvrptw(20, 95, vehicles=7, capacity=70)
    over = dict(P=6, C=64, G=30, U=5, ops=ops, T0=30 << 32)
    if kw:
        over.update(w_k=list(kw), stag_limit=0)
    p = params_for(inst, **over)
    prob, g, o = run_both(cgo, inst, p, 7, wpm=2, ns=ns)
    where = "ops %s k %s ns %d" % (ops, kw, ns)
    assert_same_state(g, o, where)
    assert_same_counts(prob, o, where)


@pytest.mark.parametrize("n,V", [(3, 2), (6, 6), (30, 3), (40, 12)])
def test_cvrptw_row_operators_sizes(cgo, n, V):
    """Two routes, more routes than customers (many empty routes), long
    routes; several candidates per lane and the deep generations."""
    inst = I.cvrptw(n, 96 + n, vehicles=V, capacity=90)
    for C, wpm, ns in ((150, 1, 1), (128, 4, 2), (128, 4, 3)):
        p = params_for(inst, P=5, C=C, G=23, U=4, ops=[SW, INS, OR] + ROWS)
        prob, g, o = run_both(cgo, inst, p, 3, wpm=wpm, ns=ns)
        assert_same_state(g, o, "n %d V %d C %d ns %d" % (n, V, C, ns))


@pytest.mark.parametrize("ns", [1, 2])
@pytest.mark.parametrize("wd,wv,wl", [(1, 0, 3), (2, 500, 1), (1, 0, 40)])
def test_cvrptw_longest_route(cgo, ns, wd, wv, wl):
    """The longest route (Sec. 6.8's third objective) as a weighted term:
    its delta takes the routes outside the changed span from prefix and
    suffix maxima of the route cache and walks the changed span whole."""
    inst = dict(I.cvrptw(25, 98, vehicles=6, capacity=90), weight_distance=wd, weight_vehicles=wv,
                weight_longest=wl)
    for ops in (None, [SW, TO, INS, OR, TH] + ROWS):
        over = dict(P=6, C=64, G=31, U=5, T0=40 << 32)
        if ops:
            over["ops"] = ops
        p = params_for(inst, **over)
        prob, g, o = run_both(cgo, inst, p, 2, wpm=2, ns=ns)
        assert_same_state(g, o, "wl %d ops %s ns %d" % (wl, ops, ns))


def test_earlier_descriptor_size_is_accepted(cgo):
    import ctypes
    inst = I.cvrptw(12, 99, vehicles=3, capacity=80)
    desc = cgo.cgo_problem_desc()
    keep = []
    for f in ("mat0", "vec0", "vec1", "vec2", "vec3"):
        a = np.ascontiguousarray(np.asarray(inst[f], np.int32).reshape(-1))
        keep.append(a)
        setattr(desc, f, a.ctypes.data)
    desc.struct_size = cgo.cgo_problem_desc.weight_longest.offset
    desc.encoding, desc.model, desc.n = 0, 4, 12
    desc.capacity, desc.vehicles = int(inst["capacity"]), 3
    desc.weight_longest = 99                      # beyond the earlier size: ignored
    h = ctypes.c_void_p()
    cgo.check(cgo.lib().cgo_problem_create(ctypes.byref(desc), ctypes.byref(h)), "create")
    q = cgo.params_struct(params_for(inst, P=4, C=32, G=11))
    cgo.check(cgo.lib().cgo_solve(h, ctypes.byref(q), 3, None), "solve")
    c = ctypes.c_int64()
    cgo.check(cgo.lib().cgo_best(h, None, 0, ctypes.byref(c)), "best")
    o = oracle_run(inst, params_for(inst, P=4, C=32, G=11), 3, 11)
    assert c.value == int(o["best_cost"].min())
    cgo.lib().cgo_problem_destroy(h)


def test_earlier_struct_sizes_are_accepted(cgo):
    """cgo_params / cgo_state of the size before the row level was appended:
    solves run with the row operators off; a state without the row level is
    refused only while row operators are on."""
    import ctypes
    inst = I.cvrptw(15, 97, vehicles=4, capacity=80)
    prob = cgo.Problem(inst)
    v1 = (cgo.cgo_params.row_w0_q16.offset + 7) & ~7     # the earlier sizeof
    q = cgo.cgo_params()
    q.struct_size = v1
    cgo.check(cgo.lib().cgo_params_default(prob.h, ctypes.byref(q)), "default")
    assert q.struct_size == v1 and list(q.row_w0_q16) == [0, 0, 0]
    q.generations = 17
    cgo.check(cgo.lib().cgo_solve(prob.h, ctypes.byref(q), 5, None), "solve")
    p = params_for(inst, P=32, C=128, G=17)
    assert_same_state(prob.state(), oracle_run(inst, p, 5, 17), "v1 params")
    # the full defaults carry the row priors, off in the mask
    full = prob.default_params()
    assert full["w_op"][8:] == [full["w_op"][0]] * 3 and not full["op_mask"] >> 8
    bad = cgo.cgo_params()
    bad.struct_size = v1 - 4
    with pytest.raises(cgo.CgoError):
        cgo.check(cgo.lib().cgo_solve(prob.h, ctypes.byref(bad), 5, None), "solve")


# ----------------------------------------------------- state and resume
@pytest.mark.parametrize("maker", [lambda: I.tsp_uniform(25, 60), lambda: I.knapsack(60, 61),
                                   lambda: I.gap(40, 62, m=6), lambda: I.qap_random(8, 63),
                                   lambda: I.cvrptw(15, 68, vehicles=4, capacity=80)])
def test_split_solve_and_checkpoint_resume(cgo, maker):
    inst = maker()
    ops = [SW] if inst["model"] == 1 else None
    p = params_for(inst, P=9, C=40, G=13, U=4, elite_period=8, **({"ops": ops} if ops else {}))
    prob = cgo.Problem(inst)
    prob.solve(p, 21)
    prob.solve_continue(6)
    prob.solve_continue(15)
    g = prob.state()
    o = oracle_run(inst, p, 21, 34)
    assert_same_state(g, o, "split")
    assert_same_counts(prob, o, "split")
    # checkpoint at g=34, resume on a fresh handle
    prob2 = cgo.Problem(inst)
    prob2.set_state(p, 21, g)
    prob2.solve_continue(9)
    prob.solve_continue(9)
    assert_same_state(prob2.state(), prob.state(), "resume")
    o43 = oracle_run(inst, p, 21, 43)
    assert_same_state(prob.state(), o43, "resume vs oracle")
    assert_same_counts(prob, o43, "split, 43 generations")


def test_best_rows_are_the_routes(cgo):
    """The elite as a multi-row solution: CVRPTW's routes as rows, equal to
    decoding the separator sequence; other models have one row."""
    inst = I.cvrptw(16, 70, vehicles=5, capacity=80)
    prob = cgo.Problem(inst)
    prob.solve(params_for(inst, P=6, C=48, G=15, ops=[SW, INS] + ROWS), 3)
    seq, c = prob.best()
    rows, c2 = prob.best_rows()
    want, cur = [], []
    for s in seq.tolist():
        if s >= 16:
            want.append(cur)
            cur = []
        else:
            cur.append(s)
    want.append(cur)
    assert rows == want and c2 == c and len(rows) == 5
    assert sorted(x for r in rows for x in r) == list(range(16))
    t = cgo.Problem(I.tsp_uniform(12, 71))
    t.solve(params_for(I.tsp_uniform(12, 71), P=4, C=32, G=5), 1)
    assert t.best_rows()[0] == [t.best()[0].tolist()]


def test_state_blob_round_trip(cgo):
    """The opaque checkpoint: export, import on a fresh handle, resume; a
    foreign, truncated or mismatched buffer is refused."""
    inst = I.cvrptw(14, 69, vehicles=4, capacity=80)
    p = params_for(inst, P=6, C=48, G=17, U=4, ops=[SW, INS, OR] + ROWS)
    prob = cgo.Problem(inst)
    prob.solve(p, 4)
    blob = prob.export_state()
    assert blob[:4] == b"CGO1"
    fresh = cgo.Problem(inst)
    fresh.import_state(p, 4, blob)
    assert_same_state(fresh.state(), prob.state(), "imported")
    fresh.solve_continue(9)
    assert_same_state(fresh.state(), oracle_run(inst, p, 4, 26), "resumed from the buffer")
    for bad in (b"XXXX" + blob[4:], blob[:len(blob) // 2], blob[:10]):
        with pytest.raises(cgo.CgoError) as e:
            fresh.import_state(p, 4, bad)
        assert e.value.status == cgo.ERR_INVALID
    other = cgo.Problem(I.cvrptw(15, 69, vehicles=4, capacity=80))
    with pytest.raises(cgo.CgoError):
        other.import_state(p, 4, blob)


@pytest.mark.parametrize("maker", [lambda: I.tsp_uniform(28, 65), lambda: I.gap(30, 66, m=5),
                                   lambda: I.cvrptw(15, 67, vehicles=4, capacity=80)])
def test_split_and_resume_with_population_steps(cgo, maker):
    """Islands, crossover, injection and the extra operators across launches
    that end mid-window and a checkpoint restored on a fresh handle."""
    inst = maker()
    extra = [O.SEGMENT] if inst["model"] == 3 else [O.THREE_OPT]
    base = [O.PERTURB] if inst["model"] == 3 else [SW, TO, INS, OR]
    p = params_for(inst, P=12, C=48, G=11, U=4, elite_period=12, islands=3, migrate_period=8,
                   migrate_strategy=2, migrate_n=2, cross_q16=40000, ops=base + extra)
    prob = cgo.Problem(inst)
    prob.solve(p, 23)
    prob.solve_continue(7)
    prob.solve_continue(13)
    g = prob.state()
    assert_same_state(g, oracle_run(inst, p, 23, 31), "split")
    prob2 = cgo.Problem(inst)
    prob2.set_state(p, 23, g)
    prob2.solve_continue(10)
    assert_same_state(prob2.state(), oracle_run(inst, p, 23, 41), "resume vs oracle")


def test_best_is_the_elite(cgo):
    inst = I.tsp_uniform(35, 64)
    p = params_for(inst, P=10, C=64, G=50)
    prob = cgo.Problem(inst)
    prob.solve(p, 5)
    sol, cost = prob.best()
    st = prob.state()
    e = int(np.argmin(st["best_cost"]))
    assert cost == st["best_cost"][e]
    assert (sol == st["best_sol"][e]).all()
    assert O.cost(inst, sol) == cost and O.valid(inst, sol)


def test_params_default_matches_oracle(cgo):
    for inst in (I.tsp_uniform(50, 1), I.tsp_uniform(200, 2), I.tsp_clustered(442, 0),
                 I.knapsack(30, 3), I.gap(20, 4, m=4), I.qap_random(6, 5)):
        prob = cgo.Problem(inst)
        d = prob.default_params()
        o = O.default_params(inst)
        for k in o:
            if k == "op_mask":
                assert d[k] == o[k] & {0: 0xF, 1: 0xF, 2: 0x10, 3: 0x20}[inst["model"]]
            else:
                assert d[k] == o[k], k


def test_device_pointer_instance(cgo):
    torch = pytest.importorskip("torch")
    inst = I.tsp_uniform(26, 65)
    dev = dict(inst, mat0=torch.from_numpy(inst["mat0"]).cuda())
    prob = cgo.Problem(dev, on_device=True)
    p = params_for(inst, P=4, C=32, G=20)
    prob.solve(p, 3)
    assert_same_state(prob.state(), oracle_run(inst, p, 3, 20), "device pointers")


def test_barrier_timeout_is_reported(cgo):
    """A member barrier that cannot complete (phantom members) ends with
    CGO_ERR_TIMEOUT after the bounded wait; the handle recovers."""
    inst = I.tsp_uniform(20, 66)
    p = params_for(inst, P=4, C=32, G=20, U=5)
    prob = cgo.Problem(inst)
    prob.inject(2, 200)            # 200 ms wait limit
    prob.inject(1, 3)              # 3 members that never arrive
    with pytest.raises(cgo.CgoError) as e:
        prob.solve(p, 1)
    assert e.value.status == cgo.ERR_TIMEOUT
    with pytest.raises(cgo.CgoError) as e:
        prob.state()
    assert e.value.status == cgo.ERR_STATE
    prob.inject(1, 0)
    prob.solve(p, 1)
    assert_same_state(prob.state(), oracle_run(inst, p, 1, 20), "after timeout")


def test_invalid_inputs(cgo):
    inst = I.tsp_uniform(10, 67)
    prob = cgo.Problem(inst)
    bad = [dict(P=0), dict(C=0), dict(C=5000), dict(U=0), dict(w_floor=3), dict(op_mask=0x10),
           dict(alpha=(1 << 32) + 1), dict(w_cap=2000)]
    for b in bad:
        with pytest.raises(cgo.CgoError) as e:
            prob.solve(params_for(inst, **dict(dict(P=4, C=8, G=1), **b)), 1)
        assert e.value.status == cgo.ERR_INVALID, b
    with pytest.raises(cgo.CgoError) as e:
        prob.solve(params_for(inst, P=4, C=8, G=1, U=4, elite_period=6), 1)
    assert e.value.status == cgo.ERR_UNSUPPORTED
    with pytest.raises(cgo.CgoError) as e:
        prob.best()
    assert e.value.status == cgo.ERR_STATE


def test_atsp_refuses_three_generations_in_flight(cgo):
    inst = I.tsp_asym(20, 44)
    prob = cgo.Problem(inst)
    prob.set_launch(12, 0, 4, 3)
    with pytest.raises(cgo.CgoError) as e:
        prob.solve(params_for(inst, P=2, C=64, G=3), 1)
    assert e.value.status == cgo.ERR_UNSUPPORTED
