"""Oracle pins for crossover (Table "operators", crossover level: order
crossover for permutations, uniform crossover for binary and integer
vectors).

The order crossover is pinned by hand-worked examples and by its defining
properties on random parents; the population step by brute force over every
partner and cut pair (the child must be one of them), by the acceptance
limits, and by the run loop taking it after each AOS window."""
import numpy as np
import pytest

import instances as I
import oracle as O
from helpers import params_for

# hand-worked: (A, B, lo, hi, child)
OX_GOLDEN = [
    # segment 3..6 kept; positions 7, 8, 0, 1, 2 take 8, 2, 1, 0, 7 (B from
    # index 7 on, wrapping, without 3, 4, 5, 6)
    ([0, 1, 2, 3, 4, 5, 6, 7, 8], [3, 4, 1, 0, 7, 6, 5, 8, 2], 3, 6, [1, 0, 7, 3, 4, 5, 6, 8, 2]),
    # segment at the end: filling starts at position 0 with B[0]
    ([0, 1, 2, 3, 4], [4, 3, 2, 1, 0], 3, 4, [2, 1, 0, 3, 4]),
    # segment at the start: positions 2, 3, 4 take 4, 2, 3 (B from index 2 on)
    ([0, 1, 2, 3, 4], [3, 0, 4, 1, 2], 0, 1, [0, 1, 4, 2, 3]),
    # the whole array is the segment: the child is A
    ([2, 0, 1], [0, 1, 2], 0, 2, [2, 0, 1]),
    # one element kept: positions 3, 0, 1 take 0, 3, 1 (B from index 3 on)
    ([0, 1, 2, 3], [3, 2, 1, 0], 2, 2, [3, 1, 2, 0]),
]


@pytest.mark.parametrize("A,B,lo,hi,child", OX_GOLDEN)
def test_ox_golden(A, B, lo, hi, child):
    assert O.ox(A, B, lo, hi).tolist() == child


def test_ox_properties_random():
    """The child is a permutation, keeps A[lo..hi] in place, and lists the
    other elements in B's cyclic order starting after position hi."""
    rng = np.random.default_rng(31)
    for n in (2, 3, 5, 8, 17, 60):
        for _ in range(60):
            A, B = rng.permutation(n), rng.permutation(n)
            lo, hi = sorted(rng.integers(0, n, 2).tolist())
            c = O.ox(A, B, lo, hi)
            assert sorted(c.tolist()) == list(range(n))
            assert (c[lo:hi + 1] == A[lo:hi + 1]).all()
            seg = set(A[lo:hi + 1].tolist())
            rest_b = [int(B[(hi + 1 + t) % n]) for t in range(n) if int(B[(hi + 1 + t) % n]) not in seg]
            rest_c = [int(c[(hi + 1 + t) % n]) for t in range(n - (hi - lo + 1))]
            assert rest_b == rest_c


def ox_children(A, B):
    n = len(A)
    out = set()
    for lo in range(n):
        for hi in range(lo, n):
            out.add(tuple(O.ox(A, B, lo, hi).tolist()))
    return out


def start_state(inst, P, seed, gens):
    p = params_for(inst, P=P, C=24, U=5)
    return p, O.solve(inst, p, seed, gens)


@pytest.mark.parametrize("maker", [lambda: I.tsp_uniform(7, 40), lambda: I.qap_random(6, 41),
                                   lambda: I.cvrptw(5, 42, vehicles=2, capacity=60)])
def test_permutation_children_are_ox_of_a_partner_best(maker):
    """With crossover certain and every child accepted (huge temperature),
    each member's new solution is the order crossover of its old one and the
    pre-step best of some other member, at some cut pair."""
    inst = maker()
    p, st = start_state(inst, 5, 3, 10)
    st = dict(st, T=1 << 62)
    got = O.crossover(inst, dict(p, cross_q16=65536), 7, st)
    n_changed = 0
    for m in range(5):
        cands = set()
        for q in range(5):
            if q != m:
                cands |= ox_children(st["cur"][m], st["best_sol"][q])
        assert tuple(got["cur"][m].tolist()) in cands, m
        assert got["cost"][m] == O.cost(inst, got["cur"][m])
        assert got["best_cost"][m] == min(st["best_cost"][m], got["cost"][m])
        n_changed += int((got["cur"][m] != st["cur"][m]).any())
    assert n_changed >= 3


@pytest.mark.parametrize("maker", [lambda: I.knapsack(40, 43), lambda: I.gap(30, 44, m=4)])
def test_uniform_children_mix_a_and_one_partner_best(maker):
    inst = maker()
    P = 6
    p, st = start_state(inst, P, 4, 10)
    st = dict(st, T=1 << 62)
    got = O.crossover(inst, dict(p, cross_q16=65536), 8, st)
    took, differ = 0, 0
    for m in range(P):
        A, c = st["cur"][m], got["cur"][m]
        fits = [q for q in range(P) if q != m and
                all(c[k] == A[k] or c[k] == st["best_sol"][q][k] for k in range(len(A)))]
        assert fits, m
        assert got["cost"][m] == O.cost(inst, c)
        if len(fits) == 1:
            B = st["best_sol"][fits[0]]
            d = A != B
            differ += int(d.sum())
            took += int((c[d] == B[d]).sum())
    # each element comes from the partner with probability 1/2
    assert differ > 50 and 0.35 < took / differ < 0.65, (took, differ)


def test_probability_zero_and_greedy_temperature():
    inst = I.tsp_uniform(15, 45)
    p, st = start_state(inst, 8, 5, 10)
    same = O.crossover(inst, dict(p, cross_q16=0), 9, st)
    for k in ("cur", "cost", "best_sol", "best_cost"):
        assert (same[k] == st[k]).all()
    greedy = O.crossover(inst, dict(p, cross_q16=65536), 9, dict(st, T=0))
    assert (greedy["cost"] <= st["cost"]).all()
    for m in range(8):
        assert greedy["cost"][m] == O.cost(inst, greedy["cur"][m])


def test_crossing_frequency_follows_the_probability():
    """A member crosses when the top 16 bits of its first draw fall below
    cross_q16: over many members and windows the share of crossing members
    (seen as children differing from A, at a huge temperature, n large enough
    that a child rarely equals A) is close to the probability."""
    inst = I.tsp_uniform(60, 46)
    P = 64
    p, st = start_state(inst, P, 6, 10)
    st = dict(st, T=1 << 62)
    for q16, share in ((16384, 0.25), (49152, 0.75)):
        changed = 0
        total = 0
        for g in range(10, 210, 10):
            got = O.crossover(inst, dict(p, cross_q16=q16), 10, dict(st, g=g))
            changed += sum(int((got["cur"][m] != st["cur"][m]).any()) for m in range(P))
            total += P
        assert abs(changed / total - share) < 0.06, (q16, changed / total)


def test_invalid_probability_rejected():
    inst = I.tsp_uniform(10, 47)
    p, st = start_state(inst, 4, 7, 5)
    with pytest.raises(ValueError):
        O.crossover(inst, dict(p, cross_q16=65537), 1, st)


@pytest.mark.parametrize("maker", [lambda: I.tsp_uniform(20, 48), lambda: I.knapsack(50, 49),
                                   lambda: I.gap(25, 50, m=5), lambda: I.qap_random(9, 51),
                                   lambda: I.cvrptw(10, 52, vehicles=3, capacity=70)])
def test_run_with_crossover_is_run_then_crossover(maker):
    """The run loop takes the crossover step after every U-th generation
    (after the AOS update, before injection)."""
    inst = maker()
    base = params_for(inst, P=6, C=32, U=5)
    cross = dict(base, cross_q16=40000)
    a = O.solve(inst, cross, 11, 5)
    plain = O.solve(inst, base, 11, 5)
    want = O.crossover(inst, cross, 11, plain)
    for k in ("cur", "cost", "best_sol", "best_cost"):
        assert (a[k] == want[k]).all(), k
    assert a["T"] == plain["T"] and a["w_op"] == plain["w_op"]
