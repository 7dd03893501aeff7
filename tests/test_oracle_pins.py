"""Pins of the CPU oracle against things other than itself (no GPU).

- Philox4x32-10 against PyTorch's independent header implementation;
- the fixed-point acceptance test against double-precision logarithms, its
  exact points and its limits (T -> 0 is greedy, T huge accepts all);
- the index/roulette mappings against exact counting;
- operators and cost models against hand-worked examples (tests/golden);
- the Q16 EMA update against a hand-worked example (Eq. "ema").
"""
import json
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
BUILD = os.path.join(os.path.dirname(__file__), "_build")


# --------------------------------------------------------------------- Philox
PX_SRC = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
int main() {
  unsigned long long seed; unsigned c0, c1, c2, c3;
  while (std::scanf("%llu %u %u %u %u", &seed, &c0, &c1, &c2, &c3) == 5) {
    at::philox_engine e(seed, ((uint64_t)c3 << 32) | c2, ((uint64_t)c1 << 32) | c0);
    unsigned r0 = e(), r1 = e(), r2 = e(), r3 = e();
    std::printf("%u %u %u %u\n", r0, r1, r2, r3);
  }
  return 0;
}
"""


def _torch_philox_tool():
    torch = pytest.importorskip("torch")
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    if not os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")):
        pytest.skip("PyTorch Philox header not installed")
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    os.makedirs(BUILD, exist_ok=True)
    src = os.path.join(BUILD, "px.cpp")
    exe = os.path.join(BUILD, "px")
    with open(src, "w") as f:
        f.write(PX_SRC)
    subprocess.run(["g++", "-std=c++17", "-O1", "-I" + inc, src, "-o", exe], check=True,
                   capture_output=True)
    return exe


def test_philox_matches_pytorch_header():
    exe = _torch_philox_tool()
    rng = np.random.default_rng(7)
    rows = [(0, 0, 0, 0, 0), (2**64 - 1, 2**32 - 1, 2**32 - 1, 2**32 - 1, 2**32 - 1),
            (1, 1 << 24, 5, 17, 0xFFFFFFFF)]
    for _ in range(2000):
        rows.append((int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2)),
                     *[int(x) for x in rng.integers(0, 2**32, 4, dtype=np.uint64)]))
    inp = "\n".join(" ".join(str(v) for v in r) for r in rows) + "\n"
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
    ref = [list(map(int, line.split())) for line in out.strip().splitlines()]
    assert len(ref) == len(rows)
    for r, want in zip(rows, ref):
        seed, c0, c1, c2, c3 = r
        got = O.philox([c0, c1, c2, c3], [seed & 0xFFFFFFFF, seed >> 32])
        assert got == want, r


# ------------------------------------------------------- fixed-point log/exp
def test_log2_exact_points():
    L = O.lib()
    assert L.orc_log2_q32(0xFFFFFFFF) == 0                # u = 1
    assert L.orc_log2_q32(0x7FFFFFFF) == 1 << 32          # u = 1/2
    assert L.orc_log2_q32(0x3FFFFFFF) == 2 << 32          # u = 1/4
    assert L.orc_log2_q32(0) == 32 << 32                  # u = 2^-32
    for k in range(33):
        A = (1 << k) - 1                                  # u = 2^(k-32)
        if A <= 0xFFFFFFFF:
            assert L.orc_log2_q32(A) == (32 - k) << 32
    # ln 2 exactly where -log2(u) = 1
    assert L.orc_exp_q32(0x7FFFFFFF) == 2977044472


def _sweep():
    rng = np.random.default_rng(11)
    a = np.concatenate([np.arange(0, 4096), 0xFFFFFFFF - np.arange(0, 4096),
                        rng.integers(0, 2**32, 60000, dtype=np.uint64),
                        (np.uint64(1) << np.arange(32, dtype=np.uint64)) - np.uint64(1)])
    return np.unique(a.astype(np.uint64))


def test_exp_error_bound_vs_double():
    L = O.lib()
    worst = 0.0
    for A in _sweep():
        A = int(A)
        E = L.orc_exp_q32(A) / 2.0**32
        u = (A + 1) / 2.0**32
        err = abs(E - (-math.log(u)))
        worst = max(worst, err)
    assert worst <= 2.0**-28, worst


def test_exp_monotone():
    L = O.lib()
    prev = None
    for A in _sweep():
        E = L.orc_exp_q32(int(A))
        if prev is not None:
            assert E <= prev
        prev = E


def test_accept_limits():
    L = O.lib()
    rng = np.random.default_rng(3)
    for _ in range(2000):
        A = int(rng.integers(0, 2**32))
        d = int(rng.integers(-10**6, 10**6))
        assert L.orc_accept(d, 0, A) == (1 if d <= 0 else 0)          # T = 0: greedy
        if A != 0xFFFFFFFF and 0 < d < 2**20:
            assert L.orc_accept(d, 2**63, A) == 1                      # huge T: all
    assert L.orc_accept(1, 2**63, 0xFFFFFFFF) == 0                      # u = 1: exp(-d/T) < 1


def test_accept_matches_double_away_from_ties():
    L = O.lib()
    rng = np.random.default_rng(5)
    checked = 0
    for _ in range(20000):
        A = int(rng.integers(0, 2**32))
        d = int(rng.integers(1, 5000))
        T = int(rng.integers(1, 500 << 32))
        u = (A + 1) / 2.0**32
        x = (T / 2.0**32) * (-math.log(u))
        if abs(d - x) < 1e-3 * max(1.0, x):
            continue
        checked += 1
        assert L.orc_accept(d, T, A) == (1 if d < x else 0)
    assert checked > 19000


def test_cooling_tracks_geometric_series():
    L = O.lib()
    T = 100 << 32
    alpha = 4290672329                    # round(0.999 * 2^32)
    for g in range(1, 3001):
        T = L.orc_cool(T, alpha)
        want = 100 * (alpha / 2.0**32) ** g
        assert abs(T / 2.0**32 - want) <= 1e-6 * 100 + g * 2.0**-32
    assert abs(alpha / 2.0**32 - 0.999) < 2.0**-32


# ------------------------------------------------------------ index mappings
@pytest.mark.parametrize("m", [1, 2, 3, 7, 10, 441, 442, 1000, 65535, 65536])
def test_pos_is_equidistributed(m):
    L = O.lib()
    counts = np.zeros(m, np.int64)
    for h in range(0, 65536, 1 if m < 2000 else 7):
        v = L.orc_pos(h, m)
        assert 0 <= v < m
        counts[v] += 1
    if m < 2000:
        assert counts.sum() == 65536
        assert counts.max() - counts.min() <= 1          # floor/ceil(65536/m) each
    assert L.orc_pos(65535, m) == m - 1 if m <= 65536 else True


def test_wsample_boundaries():
    L = O.lib()
    import ctypes
    w = (ctypes.c_uint32 * 3)(1, 2, 1)                  # W = 4: quarters of the word range
    for word, want in [(0, 0), (2**30 - 1, 0), (2**30, 1), (3 * 2**30 - 1, 1),
                       (3 * 2**30, 2), (2**32 - 1, 2)]:
        assert L.orc_wsample(w, 3, word) == want
    z = (ctypes.c_uint32 * 4)(0, 5, 0, 5)               # zero weights never chosen
    rng = np.random.default_rng(1)
    picks = [L.orc_wsample(z, 4, int(x)) for x in rng.integers(0, 2**32, 5000)]
    assert set(picks) == {1, 3}
    frac = picks.count(1) / len(picks)
    assert 0.45 < frac < 0.55


# ------------------------------------------------------------- golden moves
def _inst_for(case):
    inst = dict(model=case["model"], n=len(case["sol"]))
    if case["model"] == 3:
        inst.update(m=case["m"], mat0=np.zeros((case["m"], inst["n"]), np.int32),
                    mat1=np.zeros((case["m"], inst["n"]), np.int32),
                    vec0=np.zeros(case["m"], np.int32))
    return inst


def test_moves_golden():
    cases = json.load(open(os.path.join(GOLDEN, "moves.json")))["cases"]
    L = O.lib()
    for c in cases:
        m = len(c["sol"])
        # the fields encode the stated positions under pos(h16, m)
        if c["op"] in (0, 1, 2):
            i = L.orc_pos(c["a"], m)
            j = L.orc_pos(c["b"], m - 1)
            j += j >= i
            assert (i, j) == (c["i"], c["j"]), c["name"]
        got = O.apply_move(_inst_for(c), c["op"], c["a"], c["b"], c["x"], c["sol"])
        assert got.tolist() == c["out"], c["name"]


def test_move_invariants_random():
    rng = np.random.default_rng(9)
    for m in (2, 3, 4, 5, 9, 31):
        inst = dict(model=0, n=m)
        for _ in range(400):
            op = int(rng.integers(0, 4 if m >= 4 else 3))
            a, b, x = (int(v) for v in rng.integers(0, 65536, 3))
            s = rng.permutation(m).astype(np.int32)
            t = O.apply_move(inst, op, a, b, x, s)
            assert sorted(t.tolist()) == list(range(m))
            if op == O.INSERT:           # the moved element lands at j
                i = O.lib().orc_pos(a, m)
                j = O.lib().orc_pos(b, m - 1)
                j += j >= i
                assert t[j] == s[i]
            if op == O.SWAP:
                assert (t != s).sum() == 2
            if op == O.OR_OPT:           # the block stays contiguous and in order
                L_ = 2 + (x & 1)
                i = O.lib().orc_pos(a, m - L_ + 1)
                blk = s[i:i + L_].tolist()
                k = t.tolist().index(blk[0])
                assert t[k:k + L_].tolist() == blk
                assert t.tolist() != s.tolist()
    gi = dict(model=3, n=6, m=5, mat0=np.zeros((5, 6), np.int32),
              mat1=np.zeros((5, 6), np.int32), vec0=np.zeros(5, np.int32))
    for _ in range(500):
        s = rng.integers(0, 5, 6).astype(np.int32)
        a, b = (int(v) for v in rng.integers(0, 65536, 2))
        t = O.apply_move(gi, O.PERTURB, a, b, 0, s)
        assert (t != s).sum() == 1 and t.min() >= 0 and t.max() <= 4


def _preimage(q, m):
    """a 16-bit field a with pos(a, m) = q"""
    return -(-(q << 16) // m)


def test_segment_operators_are_runs_of_the_element_operators():
    """seg_flip is L flips and seg_reset L random resets with one offset, at
    the L consecutive positions from i = pos(a, n-L+1), L = min(2 + (x & 1), n);
    segment starts are (nearly) uniform over the n-L+1 choices."""
    rng = np.random.default_rng(22)
    L_ = O.lib()
    for n in (2, 3, 5, 9, 40):
        ki = dict(model=2, n=n)
        gi = dict(model=3, n=n, m=5, mat0=np.zeros((5, n), np.int32),
                  mat1=np.zeros((5, n), np.int32), vec0=np.zeros(5, np.int32))
        starts = {}
        for _ in range(1500 if n == 9 else 200):
            a, b = (int(v) for v in rng.integers(0, 65536, 2))
            x = int(rng.integers(0, 2**32))
            L = min(2 + (x & 1), n)
            i = L_.orc_pos(a, n - L + 1)
            s = rng.integers(0, 2, n).astype(np.int32)
            t = O.apply_move(ki, O.SEGMENT, a, b, x, s)
            want = s.copy()
            for q in range(i, i + L):
                want = O.apply_move(ki, O.FLIP, _preimage(q, n), 0, 0, want)
            assert (t == want).all() and (t != s).sum() == L
            s = rng.integers(0, 5, n).astype(np.int32)
            t = O.apply_move(gi, O.SEGMENT, a, b, x, s)
            want = s.copy()
            for q in range(i, i + L):
                want = O.apply_move(gi, O.PERTURB, _preimage(q, n), b, 0, want)
            assert (t == want).all()
            d = (t - s) % 5
            assert (d[i:i + L] == d[i]).all() and d[i] != 0 and (d[:i] == 0).all() and (d[i + L:] == 0).all()
            if n == 9:
                starts[(L, i)] = starts.get((L, i), 0) + 1
        if n == 9:
            for L in (2, 3):
                cnt = [starts.get((L, i), 0) for i in range(n - L + 1)]
                mean = sum(cnt) / len(cnt)
                assert min(cnt) > 0.6 * mean and max(cnt) < 1.4 * mean, (L, cnt)
    # a single element has no segment: the operator is not applicable
    assert O.enabled_ops(dict(model=2, n=1), 0xFF)[O.SEGMENT] == 0


def _exchange_cuts(s, t):
    """All (i, j, k) with t = s[:i] + s[j:k] + s[i:j] + s[k:], i < j < k."""
    m = len(s)
    s, t = list(s), list(t)
    return [(i, j, k) for i in range(m) for j in range(i + 1, m) for k in range(j + 1, m + 1)
            if s[:i] + s[j:k] + s[i:j] + s[k:] == t]


def test_three_opt_is_an_adjacent_segment_exchange_with_uniform_cuts():
    """3-opt (Table "operators", segment level): the result is the original
    with two adjacent segments exchanged, and the cut triples are (nearly)
    uniform over all C(m+1, 3) choices."""
    rng = np.random.default_rng(21)
    for m in (2, 3, 5, 8, 13):
        inst = dict(model=0, n=m)
        seen = {}
        s = np.arange(m, dtype=np.int32)
        draws = 6000 if m == 5 else 300
        for _ in range(draws):
            a, b = (int(v) for v in rng.integers(0, 65536, 2))
            x = int(rng.integers(0, 2**32))
            t = O.apply_move(inst, O.THREE_OPT, a, b, x, s)
            cuts = _exchange_cuts(s, t)
            assert cuts, (m, a, b, x, t)
            seen[tuple(t.tolist())] = seen.get(tuple(t.tolist()), 0) + 1
        if m == 5:
            # every exchange is reachable; frequencies within 30% of uniform
            # (distinct triples can give the same array only for equal lengths)
            total = sum(seen.values())
            assert len(seen) >= 15
            per_triple = draws / 20
            for arr, cnt in seen.items():
                n_tr = len(_exchange_cuts(s, np.array(arr)))
                assert abs(cnt - n_tr * per_triple) < 0.3 * n_tr * per_triple, (arr, cnt, n_tr)


# ------------------------------------------------------------- golden costs
def _inst_from_case(c):
    inst = {k: v for k, v in c.items() if k not in ("name", "sol", "cost", "work")}
    for k in ("mat0", "mat1", "vec0", "vec1", "vec2", "vec3"):
        if k in inst:
            inst[k] = np.asarray(inst[k], np.int32)
    return inst


def test_costs_golden():
    cases = json.load(open(os.path.join(GOLDEN, "costs.json")))["cases"]
    for c in cases:
        assert O.cost(_inst_from_case(c), c["sol"]) == c["cost"], c["name"]


# --------------------------------------------------------------------- AOS
def test_ema_golden():
    """Eq. "ema" in Q16, worked by hand:
    ratio0 = floor(5*65536/11) = 29789, ratio1 = 0;
    w0 = floor((52429*32768 + 13107*(29789+3277)) / 65536) = floor(2151389534/65536) = 32827;
    w1 = floor((52429*32768 + 13107*3277) / 65536) = floor(1760945111/65536) = 26869;
    normalise: S = 59696; floor(32827*65536/59696) = 36038; floor(26869*65536/59696) = 29497."""
    w = O.aos_level([32768, 32768, 7, 0], [10, 10, 99, 0], [5, 0, 99, 0], [1, 1, 0, 0],
                    [65536] * 4, 52429, 3277, 39322)
    assert w == [36038, 29497, 7, 0]


def test_ema_cap_and_floor():
    # an op that always improves is capped at w_cap before normalising; one
    # that never does decays to the floor: w = (a*w + (1-a)*floor) >> 16
    w = O.aos_level([65536, 0], [100, 100], [100, 0], [1, 1], [65536, 65536],
                    52429, 3277, 39322)
    # w0 clamps to 39322; w1 = floor(13107*3277/65536) = 655 -> floor 3277
    S = 39322 + 3277
    assert w == [(39322 << 16) // S, (3277 << 16) // S]
    # a per-operator cap below w_cap wins
    w = O.aos_level([65536, 0], [100, 100], [100, 0], [1, 1], [20000, 65536],
                    52429, 3277, 39322)
    S = 20000 + 3277
    assert w == [(20000 << 16) // S, (3277 << 16) // S]


def test_ema_fixed_point():
    # if v/(u+1) + floor equals w for every op and sums to 1, weights stay put
    w = O.aos_level([32768, 32768], [65535, 65535], [(32768 - 3277) * 65536 // 65536, 29491],
                    [1, 1], [65536, 65536], 52429, 3277, 65536)
    assert abs(w[0] - 32768) <= 2 and abs(w[1] - 32768) <= 2
    assert 65536 - 2 <= sum(w) <= 65536
