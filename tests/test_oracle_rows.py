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
