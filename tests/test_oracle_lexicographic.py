"""Pins of CVRPTW's lexicographic mode in the oracle (reading R37; Sec. 6.8,
Table "lexicographic_mode").

The mode compares solutions by their penalty first, then by the
prioritised objectives in order (distance, vehicles used, the longest
route's distance), each in buckets of width tolerance + 1: values in one
bucket tie and the next objective decides.  The oracle writes this order as
one integer key.  The tests enumerate every solution of tiny instances and
check, independently of how the key is written:

- the key orders any two solutions exactly as the tuples (penalty,
  bucket_1, bucket_2, ...) do (equal keys for equal tuples);
- a larger tolerance lets the next objective decide between distances that
  it puts in one bucket (the Table's effect: a distance within tolerance of
  the best loses to one with fewer vehicles);
- the search reaches the brute-force lexicographic optimum.

A hand-worked key pins the integer itself.
"""
import itertools

import numpy as np
import pytest

import instances as I
import oracle as O
from conftest import SEEDS

D_, V_, L_ = O.LEX_DISTANCE, O.LEX_VEHICLES, O.LEX_LONGEST


def objectives(inst, perm):
    """(distance, capacity excess, lateness, vehicles used, longest route) of
    a separator-encoded sequence, walked route by route."""
    n = inst["n"]
    d, dem, rdy, due, svc = (inst[k] for k in ("mat0", "vec0", "vec1", "vec2", "vec3"))
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
        t = load = prev = rd = 0
        for c in rt:
            dd = int(d[prev][c])
            dist += dd
            rd += dd
            t = max(t + dd, int(rdy[c]))
            late += max(0, t - int(due[c]))
            t += int(svc[c])
            load += int(dem[c])
            prev = c
        back = int(d[prev][0])
        dist += back
        rd += back
        longest = max(longest, rd)
        t += back
        late += max(0, t - int(due[0]))
        excess += max(0, load - int(inst["capacity"]))
    return dist, excess, late, used, longest


def lex_tuple(inst, perm):
    dist, excess, late, used, longest = objectives(inst, perm)
    o = {D_: dist, V_: used, L_: longest}
    return (100 * excess + 100 * late,) + tuple(o[obj] // (tol + 1)
                                                 for obj, tol in inst["lexicographic"])


def small(index, lex, V=3):
    return dict(I.cvrptw(5, index, vehicles=V, capacity=60, box=60, horizon=300, width=80),
                lexicographic=lex)


MODES = [[(D_, 0), (V_, 0)], [(D_, 50), (V_, 0)], [(V_, 0), (D_, 100)],
         [(D_, 0), (V_, 0), (L_, 0)], [(V_, 0), (D_, 30), (L_, 20)], [(L_, 15)]]


@pytest.mark.parametrize("lex", MODES)
@pytest.mark.parametrize("index", [104, 105])
def test_key_orders_solutions_as_the_bucketed_tuples(index, lex):
    inst = small(index, lex)
    perms = list(itertools.permutations(range(inst["n"] + inst["vehicles"] - 1)))
    rows = [(lex_tuple(inst, p), O.cost(inst, list(p))) for p in perms]
    tuples = sorted({t for t, _ in rows})
    keys = {}
    for t, k in rows:
        assert keys.setdefault(t, k) == k      # equal tuples, equal keys
    ks = [keys[t] for t in tuples]
    assert all(a < b for a, b in zip(ks, ks[1:]))   # strictly increasing with the tuple order


def test_tolerance_lets_the_next_objective_decide():
    """Among the solutions, the lexicographic best under (distance, tol 0)
    and (distance, tol 100) then vehicles: the wider bucket holds distances
    up to 100 apart, within which fewer vehicles win."""
    for index in range(104, 124):
        inst0 = small(index, [(D_, 0), (V_, 0)])
        inst1 = small(index, [(D_, 100), (V_, 0)])
        perms = list(itertools.permutations(range(inst0["n"] + inst0["vehicles"] - 1)))
        b0 = min(perms, key=lambda p: O.cost(inst0, list(p)))
        b1 = min(perms, key=lambda p: O.cost(inst1, list(p)))
        o0, o1 = objectives(inst0, b0), objectives(inst1, b1)
        if o1[3] < o0[3]:                        # fewer vehicles for a longer distance
            assert o1[0] > o0[0]
            assert o1[0] // 101 == o0[0] // 101 or o1[1:3] != o0[1:3]
            return
    pytest.fail("no instance where the tolerance changes the lexicographic best")


def test_hand_worked_key():
    """Three customers at distance 3 (and 4 between them) from the depot, no
    time pressure, capacity for two; solution [c1, c2 | c3].
    Route 1: 3 + 4 + 3 = 10; route 2: 3 + 3 = 6.  distance 16, vehicles 2,
    longest 10, penalty 0.  lex_dmax = (n + V) * max travel = (3 + 2) * 4 = 20.
    Mode (distance tol 4, vehicles tol 0): q = (16 // 5, 2 // 1) = (3, 2),
    radices (20 // 5 + 1, 2 // 1 + 1) = (5, 3): key = (0 * 5 + 3) * 3 + 2 = 11.
    Mode (longest tol 0, distance tol 9): q = (10, 16 // 10 = 1), radices
    (21, 20 // 10 + 1 = 3): key = (0 * 21 + 10) * 3 + 1 = 31."""
    d = np.array([[0, 3, 3, 3], [3, 0, 4, 4], [3, 4, 0, 4], [3, 4, 4, 0]], np.int32)
    inst = dict(model=I.CVRPTW, n=3, vehicles=2, capacity=2, mat0=d,
                vec0=np.array([0, 1, 1, 1], np.int32), vec1=np.zeros(4, np.int32),
                vec2=np.array([1000, 1000, 1000, 1000], np.int32), vec3=np.zeros(4, np.int32))
    sol = [0, 1, 3, 2]                           # c1 c2 | c3 (symbol 3 is the separator)
    assert O.cost(dict(inst, lexicographic=[(D_, 4), (V_, 0)]), sol) == 11
    assert O.cost(dict(inst, lexicographic=[(L_, 0), (D_, 9)]), sol) == 31
    assert O.cost(inst, sol) == 16               # the weighted cost without the mode


@pytest.mark.parametrize("seed", SEEDS)
@pytest.mark.parametrize("lex", [MODES[1], MODES[2], MODES[4]])
def test_search_reaches_the_lexicographic_optimum(seed, lex):
    inst = small(104, lex)
    perms = itertools.permutations(range(inst["n"] + inst["vehicles"] - 1))
    opt = min(O.cost(inst, list(p)) for p in perms)
    p = O.default_params(inst)
    p.update(P=8, C=32)
    st = O.solve(inst, p, seed, 400, threads=2)
    assert st["best_cost"].min() == opt
