"""Oracle pins for the row operators of CVRPTW's separator encoding
(Table "operators", row level: row_swap, row_merge, row_split; rows are
routes).  Hand-worked examples plus their route-list semantics on random
solutions, checked through an independent decode of the routes."""
import numpy as np
import pytest

import instances as I
import oracle as O

INST = I.cvrptw(5, 1, vehicles=3)      # symbols 0..4 customers, 5 and 6 separators

# (kind, a, b, sol, out, what) worked by hand
GOLDEN = [
    (O.ROW_SWAP, 0, 65535, [0, 1, 5, 2, 6, 3, 4], [3, 4, 5, 2, 6, 0, 1],
     "routes 0 and 2 (r2 = pos(65535, 2) = 1, stepped over 0 to 2) exchange"),
    (O.ROW_SWAP, 32768, 0, [0, 1, 5, 2, 6, 3, 4], [2, 5, 0, 1, 6, 3, 4],
     "r1 = pos(32768, 3) = 1, r2 = 0: routes 0 and 1 exchange"),
    (O.ROW_MERGE, 0, 0, [0, 1, 5, 2, 6, 3, 4], [0, 1, 2, 5, 6, 3, 4],
     "route 0 takes route 1's customer, an empty route follows"),
    (O.ROW_MERGE, 65535, 0, [0, 1, 5, 2, 6, 3, 4], [0, 1, 5, 2, 3, 4, 6],
     "r = pos(65535, 2) = 1: route 1 takes the last route, the separator goes to the end"),
    (O.ROW_SPLIT, 0, 0, [0, 1, 2, 5, 6, 3, 4], [0, 6, 1, 2, 5, 3, 4],
     "route 0 (3 customers) splits after k = 1; the empty route 1 disappears"),
    (O.ROW_SPLIT, 0, 65535, [0, 1, 2, 5, 6, 3, 4], [0, 1, 6, 2, 5, 3, 4],
     "k = 1 + pos(65535, 2) = 2"),
    (O.ROW_SPLIT, 0, 0, [0, 1, 5, 2, 3, 4, 6], [0, 6, 1, 5, 2, 3, 4],
     "the empty route is the last one: the separator that opens it moves"),
    (O.ROW_SPLIT, 0, 0, [0, 1, 5, 2, 6, 3, 4], [0, 1, 5, 2, 6, 3, 4],
     "no empty route: nothing changes"),
    (O.ROW_SPLIT, 32768, 0, [0, 1, 2, 5, 6, 3, 4], [0, 1, 2, 5, 6, 3, 4],
     "route 1 is empty (fewer than two customers): nothing changes"),
]


@pytest.mark.parametrize("kind,a,b,sol,out,what", GOLDEN)
def test_row_moves_golden(kind, a, b, sol, out, what):
    assert O.row_move(INST, kind, a, b, sol).tolist() == out, what


def routes(sol, n):
    out, cur = [], []
    for s in sol:
        if s >= n:
            out.append(cur)
            cur = []
        else:
            cur.append(int(s))
    out.append(cur)
    return out


def pos(h, m):
    return (h * m) >> 16


def test_row_move_semantics_random():
    rng = np.random.default_rng(41)
    for n, V in ((6, 3), (12, 5), (30, 8)):
        inst = I.cvrptw(n, 50 + n, vehicles=V)
        for _ in range(400):
            s = rng.permutation(n + V - 1).astype(np.int32)
            a, b = (int(v) for v in rng.integers(0, 65536, 2))
            R = routes(s, n)
            # row_swap: two routes exchange their customer sequences
            r1, r2 = pos(a, V), pos(b, V - 1)
            r2 += r2 >= r1
            want = list(R)
            want[r1], want[r2] = R[r2], R[r1]
            got = O.row_move(inst, O.ROW_SWAP, a, b, s)
            assert routes(got, n) == want
            assert sorted(got.tolist()) == list(range(n + V - 1))
            # row_merge: r and r + 1 join, an empty route follows
            r = pos(a, V - 1)
            want = R[:r] + [R[r] + R[r + 1], []] + R[r + 2:]
            assert routes(O.row_move(inst, O.ROW_MERGE, a, b, s), n) == want
            # row_split: the lowest empty route goes, route r splits after k
            r = pos(a, V)
            empty = [q for q in range(V) if not R[q]]
            got = routes(O.row_move(inst, O.ROW_SPLIT, a, b, s), n)
            if len(R[r]) < 2 or not empty:
                assert got == R
            else:
                k = 1 + pos(b, len(R[r]) - 1)
                rest = [R[q] for q in range(V) if q != empty[0]]
                i = [q for q in range(V) if q != empty[0]].index(r)
                want = rest[:i] + [R[r][:k], R[r][k:]] + rest[i + 1:]
                assert got == want


def test_row_moves_only_for_cvrptw():
    with pytest.raises(ValueError):
        O.row_move(I.tsp_uniform(6, 1), O.ROW_SWAP, 0, 0, list(range(6)))


@pytest.mark.parametrize("sol", [
    [0, 1, 5, 2, 6, 3],            # one symbol short
    [0, 1, 5, 2, 6, 3, 4, 4],      # one symbol too many
    [0, 1, 5, 2, 6, 5, 4],         # three separators in a length-7 sequence
    [0, 1, 2, 2, 6, 3, 4],         # one separator
])
def test_row_moves_reject_malformed(sol):
    with pytest.raises(ValueError):
        O.row_move(INST, O.ROW_SWAP, 0, 0, sol)


# ----------------------------------------------- the row level in the search
ROW_OPS = (O.ROW_SWAP_OP, O.ROW_MERGE_OP, O.ROW_SPLIT_OP)


def test_search_applies_the_row_moves():
    """Operator slots 8..10 of the search apply row_swap, row_merge and
    row_split exactly as the pinned primitives do (the search's move hook is
    orc_apply_move)."""
    rng = np.random.default_rng(43)
    inst = I.cvrptw(9, 61, vehicles=4)
    for _ in range(300):
        s = rng.permutation(9 + 3).astype(np.int32)
        a, b, x = (int(v) for v in rng.integers(0, 65536, 3))
        for kind, op in zip((O.ROW_SWAP, O.ROW_MERGE, O.ROW_SPLIT), ROW_OPS):
            assert O.apply_move(inst, op, a, b, x, s).tolist() == O.row_move(inst, kind, a, b, s).tolist()


def test_row_level_applies_to_cvrptw_with_two_routes_or_more():
    full = (1 << O.NOPS) - 1
    assert [O.enabled_ops(I.cvrptw(8, 62, vehicles=3), full)[i] for i in ROW_OPS] == [1, 1, 1]
    assert [O.enabled_ops(I.cvrptw(8, 62, vehicles=1), full)[i] for i in ROW_OPS] == [0, 0, 0]
    for other in (I.tsp_uniform(8, 63), I.qap_random(6, 64), I.knapsack(10, 65), I.gap(8, 66, m=3)):
        assert [O.enabled_ops(other, full)[i] for i in ROW_OPS] == [0, 0, 0]
    # off in the default mask, with the O(1) prior 1.0 for callers that enable them
    inst = I.cvrptw(20, 67, vehicles=5)
    p = O.default_params(inst)
    assert all(not (p["op_mask"] >> i) & 1 for i in ROW_OPS)
    assert p["w_op"][O.ROW_SWAP_OP] == p["w_op"][O.SWAP] > 0
    assert p["w_op"][O.ROW_SWAP_OP] == p["w_op"][O.ROW_MERGE_OP] == p["w_op"][O.ROW_SPLIT_OP]


def _routes_cost(inst, R):
    n = inst["n"]
    seq = []
    for i, r in enumerate(R):
        seq += r
        if i < len(R) - 1:
            seq.append(n + i)
    return O.cost(inst, seq)


def test_row_search_states_and_counts():
    """A search with the row level on keeps valid sequences whose costs
    equal full re-evaluation, and its counts cover the row operators."""
    inst = I.cvrptw(14, 68, vehicles=5, capacity=90)
    p = O.default_params(inst)
    w = [0] * O.NOPS
    for o in (O.SWAP, O.INSERT, O.TWO_OPT) + ROW_OPS:
        w[o] = 65536 // 6
    p.update(P=6, C=24, U=4, op_mask=sum(1 << o for o in (O.SWAP, O.INSERT, O.TWO_OPT) + ROW_OPS),
             w_op=w)
    st = O.solve(inst, p, 3, 22)
    for m in range(6):
        assert O.valid(inst, st["cur"][m]) and O.cost(inst, st["cur"][m]) == st["cost"][m]
        assert O.cost(inst, st["best_sol"][m]) == st["best_cost"][m] <= st["cost"][m]
    oc = st["op_counts"]
    assert all(oc["u_op"][i] > 0 for i in ROW_OPS)
    assert sum(oc["u_k"]) == 6 * 24 * 22
    assert sum(oc["u_op"]) == oc["u_k"][0] + 2 * oc["u_k"][1] + 3 * oc["u_k"][2]


@pytest.mark.parametrize("seed", [1, 42, 123, 456, 789])
def test_row_level_with_insertion_reaches_bruteforce_optimum(seed):
    """Insertion plus the row level alone (no swap, 2-opt or or-opt) still
    reaches the brute-force optimum of a tiny CVRPTW."""
    import itertools
    inst = I.cvrptw(5, 104, vehicles=3, capacity=60, box=60, horizon=300, width=80)
    n, V = 5, 3
    best = min(O.cost(inst, list(pm)) for pm in itertools.permutations(range(n + V - 1)))
    p = O.default_params(inst)
    ops = (O.INSERT,) + ROW_OPS
    w = [0] * O.NOPS
    for o in ops:
        w[o] = 65536 // 4
    p.update(P=8, C=32, op_mask=sum(1 << o for o in ops), w_op=w)
    st = O.solve(inst, p, seed, 400, threads=2)
    assert st["best_cost"].min() == best
