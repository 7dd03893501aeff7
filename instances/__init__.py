"""Seeded synthetic instance generators.

These produce the input data (integer matrices and vectors) that both the CPU
oracle and the CUDA path consume.  Nothing here implements any step of the
search method: no moves, no costs, no acceptance, no operator selection.  It
only draws random instance data of the shapes the paper's workloads have
(TSPLIB-like Euclidean TSP, QAPLIB-like QAP, Pisinger-like 0-1 knapsack,
generalized assignment, Solomon-like CVRPTW) and the Poisson arrival trace of
the serving workload.

Randomness comes from NumPy's Philox4x64 bit generator, keyed by
(GEN_SEED, instance index, stream).  Only ``random_raw`` words are used and
every mapping to integers is written out here, so the data do not depend on
NumPy's distribution code.  Every generator returns plain ``int32`` / ``int64``
numpy arrays in a dict whose keys follow the library's problem description
(``mat0``, ``mat1``, ``vec0`` ... ``vec3``, ``capacity`` ...).
"""
from __future__ import annotations

import math

import numpy as np

GEN_SEED = 20260319

# model ids, mirrored by the C ABI and the oracle (each declares its own copy)
TSP, QAP, KNAPSACK, GAP, CVRPTW = 0, 1, 2, 3, 4
ENC_PERM, ENC_BINARY, ENC_INTEGER = 0, 1, 2
MODEL_ENCODING = {TSP: ENC_PERM, QAP: ENC_PERM, KNAPSACK: ENC_BINARY,
                  GAP: ENC_INTEGER, CVRPTW: ENC_PERM}


class Stream:
    """Philox4x64-keyed stream of raw 64-bit words with integer mappings."""

    def __init__(self, index: int, stream: int = 0):
        key = np.array([GEN_SEED + (stream << 32), index], dtype=np.uint64)
        self._bg = np.random.Philox(key=key)

    def raw(self, size: int) -> np.ndarray:
        return np.asarray(self._bg.random_raw(size), dtype=np.uint64).reshape(-1)

    def ints(self, lo: int, hi: int, size: int) -> np.ndarray:
        """Uniform integers in [lo, hi] (inclusive): hi32(word) * R >> 32."""
        r = np.uint64(hi - lo + 1)
        w = self.raw(size) >> np.uint64(32)
        return (lo + ((w * r) >> np.uint64(32)).astype(np.int64)).astype(np.int64)

    def unit(self, size: int) -> np.ndarray:
        """Uniform doubles in (0, 1]: (top 53 bits + 1) / 2^53."""
        w = self.raw(size) >> np.uint64(11)
        return (w.astype(np.float64) + 1.0) / float(1 << 53)

    def normal(self, size: int) -> np.ndarray:
        """Standard normal draws by Box-Muller (double precision)."""
        u1 = self.unit(size)
        u2 = self.unit(size)
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def nint_sqrt(s: np.ndarray) -> np.ndarray:
    """round(sqrt(s)) for non-negative integers s, computed exactly.

    r = isqrt(s); r += (s - r*r > r).  (sqrt(s) >= r + 1/2  <=>  s > r^2 + r.)
    """
    s = np.asarray(s, dtype=np.int64)
    r = np.floor(np.sqrt(s.astype(np.float64))).astype(np.int64)
    # fix the float estimate to the exact integer square root
    while True:
        hi = r * r > s
        if not hi.any():
            break
        r = r - hi
    while True:
        lo = (r + 1) * (r + 1) <= s
        if not lo.any():
            break
        r = r + lo
    return r + ((s - r * r) > r)


def euclid_matrix(xy: np.ndarray) -> np.ndarray:
    """Rounded Euclidean distance matrix (int32) of integer coordinates."""
    xy = np.asarray(xy, dtype=np.int64)
    dx = xy[:, None, 0] - xy[None, :, 0]
    dy = xy[:, None, 1] - xy[None, :, 1]
    return nint_sqrt(dx * dx + dy * dy).astype(np.int32)


# --------------------------------------------------------------------------- TSP
def tsp_uniform(n: int, index: int, box: int = 1000) -> dict:
    """TSP: n cities with integer coordinates uniform in [0, box]^2."""
    st = Stream(index, 1)
    xy = st.ints(0, box, 2 * n).reshape(n, 2)
    return dict(model=TSP, n=n, mat0=euclid_matrix(xy), coords=xy)


def tsp_asym(n: int, index: int, box: int = 1000, skew: int = 300) -> dict:
    """TSP of an asymmetric matrix: the Euclidean distances of n integer
    points uniform in [0, box]^2 plus an independent offset uniform in
    [0, skew] for every ordered pair i != j (diagonal 0)."""
    st = Stream(index, 11)
    xy = st.ints(0, box, 2 * n).reshape(n, 2)
    D = euclid_matrix(xy).astype(np.int64) + st.ints(0, skew, n * n).reshape(n, n)
    np.fill_diagonal(D, 0)
    return dict(model=TSP, n=n, mat0=D.astype(np.int32), coords=xy)


def tsp_clustered(n: int, index: int, box: int = 4000, clusters: int = 6,
                  sigma: float = 40.0, noise: float = 0.10) -> dict:
    """TSP: Gaussian clusters plus uniform noise (pcb442-shaped stand-in).

    ``clusters`` centres uniform in [120, box-120]^2; round(noise*n) points
    uniform in [0, box]^2; the rest N(centre, sigma) around a uniformly chosen
    centre; clamped to the box and rounded to integers.
    """
    st = Stream(index, 2)
    centres = st.ints(120, box - 120, 2 * clusters).reshape(clusters, 2)
    n_noise = int(round(noise * n))
    n_clu = n - n_noise
    pick = st.ints(0, clusters - 1, n_clu)
    g = st.normal(2 * n_clu).reshape(n_clu, 2)
    pts = centres[pick].astype(np.float64) + sigma * g
    pts = np.clip(np.rint(pts), 0, box).astype(np.int64)
    noise_pts = st.ints(0, box, 2 * n_noise).reshape(n_noise, 2)
    xy = np.concatenate([pts, noise_pts], axis=0)
    return dict(model=TSP, n=n, mat0=euclid_matrix(xy), coords=xy)


# --------------------------------------------------------------------------- QAP
def qap_grid(n: int, index: int, zero_frac: float = 0.70,
             symmetric: bool = True) -> dict:
    """QAP: sparse flow matrix F and Manhattan distances D on a grid.

    F: zero diagonal, each off-diagonal pair zero with probability zero_frac,
    otherwise uniform in [1, 100]; symmetric unless ``symmetric`` is False.
    D: Manhattan distance between grid cells k = (k // w, k % w), w = ceil(sqrt n).
    """
    st = Stream(index, 3)
    keep = st.ints(0, 999, n * n).reshape(n, n) >= int(round(zero_frac * 1000))
    val = st.ints(1, 100, n * n).reshape(n, n)
    F = np.where(keep, val, 0)
    if symmetric:
        F = np.triu(F, 1)
        F = F + F.T
    np.fill_diagonal(F, 0)
    w = int(math.ceil(math.sqrt(n)))
    k = np.arange(n)
    r, c = k // w, k % w
    D = np.abs(r[:, None] - r[None, :]) + np.abs(c[:, None] - c[None, :])
    return dict(model=QAP, n=n, mat0=F.astype(np.int32), mat1=D.astype(np.int32))


def qap_random(n: int, index: int, lo: int = -20, hi: int = 50) -> dict:
    """QAP with asymmetric F, D and non-zero diagonals (edge-case instances)."""
    st = Stream(index, 4)
    F = st.ints(lo, hi, n * n).reshape(n, n)
    D = st.ints(lo, hi, n * n).reshape(n, n)
    return dict(model=QAP, n=n, mat0=F.astype(np.int32), mat1=D.astype(np.int32))


# ---------------------------------------------------------------------- knapsack
def knapsack(n: int, index: int, lo: int = 1, hi: int = 1000) -> dict:
    """0-1 knapsack: weights/values uniform in [lo, hi], capacity floor(sum w / 2)."""
    st = Stream(index, 5)
    w = st.ints(lo, hi, n)
    v = st.ints(lo, hi, n)
    return dict(model=KNAPSACK, n=n, vec0=w.astype(np.int32), vec1=v.astype(np.int32),
                capacity=int(w.sum() // 2))


# --------------------------------------------------------------------------- GAP
def gap(n: int, index: int, m: int = 10) -> dict:
    """Generalized assignment: n jobs, m agents, cost/requirement in [1, 100].

    mat0 = cost[m][n], mat1 = req[m][n]; every agent's capacity is
    floor(1.2 * sum(req) / m^2), i.e. 1.2 x the mean load of an agent.
    """
    st = Stream(index, 6)
    c = st.ints(1, 100, m * n).reshape(m, n)
    r = st.ints(1, 100, m * n).reshape(m, n)
    cap = np.full(m, int(12 * int(r.sum()) // (10 * m * m)), dtype=np.int64)
    return dict(model=GAP, n=n, m=m, mat0=c.astype(np.int32), mat1=r.astype(np.int32),
                vec0=cap.astype(np.int32))


# ------------------------------------------------------------------------ CVRPTW
def cvrptw(n: int, index: int, vehicles: int = 25, capacity: int = 200,
           box: int = 100, horizon: int = 1000, width: int = 60,
           service: int = 10) -> dict:
    """CVRPTW (Solomon-R-like): n customers, depot at the box centre.

    Node 0 is the depot.  Coordinates uniform in [0, box]^2, demand in [1, 50],
    ready uniform in [0, horizon - width], due = ready + width, service time
    ``service``; the depot window is [0, horizon].  mat0 is the (n+1)^2
    rounded-Euclidean travel matrix; vec0..vec3 = demand, ready, due, service
    (n+1 entries each, entry 0 the depot).
    """
    st = Stream(index, 7)
    xy = st.ints(0, box, 2 * n).reshape(n, 2)
    depot = np.array([[box // 2, box // 2]], dtype=np.int64)
    allxy = np.concatenate([depot, xy], axis=0)
    demand = np.concatenate([[0], st.ints(1, 50, n)])
    ready = np.concatenate([[0], st.ints(0, horizon - width, n)])
    due = np.concatenate([[horizon], ready[1:] + width])
    serv = np.concatenate([[0], np.full(n, service)])
    return dict(model=CVRPTW, n=n, vehicles=vehicles, capacity=capacity,
                mat0=euclid_matrix(allxy), vec0=demand.astype(np.int32),
                vec1=ready.astype(np.int32), vec2=due.astype(np.int32),
                vec3=serv.astype(np.int32))


# ----------------------------------------------------------------- workload sets
def batch_mix(count: int = 512, index: int = 0) -> list[dict]:
    """The uneven batch: 40% TSP n~U[50,500], 40% knapsack n~U[100,2000],
    20% GAP n~U[50,300] (m=10); order shuffled by the stream; every instance
    gets its own index (and so its own data) and instance tag = position."""
    st = Stream(index, 8)
    n_tsp = int(round(0.4 * count))
    n_kp = int(round(0.4 * count))
    n_gap = count - n_tsp - n_kp
    kinds = np.array([TSP] * n_tsp + [KNAPSACK] * n_kp + [GAP] * n_gap)
    order = np.argsort(st.raw(count), kind="stable")
    kinds = kinds[order]
    sizes_t = st.ints(50, 500, count)
    sizes_k = st.ints(100, 2000, count)
    sizes_g = st.ints(50, 300, count)
    out = []
    for i, kd in enumerate(kinds):
        sub = 1000 + 1000 * index + i
        if kd == TSP:
            inst = tsp_uniform(int(sizes_t[i]), sub)
        elif kd == KNAPSACK:
            inst = knapsack(int(sizes_k[i]), sub)
        else:
            inst = gap(int(sizes_g[i]), sub)
        inst["tag"] = i
        out.append(inst)
    return out


def serving_pool(index: int = 0, cvrptw_count: int = 96) -> list[dict]:
    """Instance pool of the serving workload: the 512-instance batch mix
    (TSP / knapsack / GAP) followed by `cvrptw_count` CVRPTW instances with
    100 customers."""
    pool = batch_mix(512, index)
    for i in range(cvrptw_count):
        pool.append(cvrptw(100, 700000 + 1000 * index + i))
    return pool


def poisson_arrivals(rate: float = 200.0, duration: float = 60.0, index: int = 7,
                     cvrptw_frac: float = 0.15, pool_mix: int = 512,
                     pool_cvrptw: int = 96) -> list[tuple[float, int]]:
    """Arrival times (exponential inter-arrivals at `rate` per second over
    `duration` seconds) and, for each, an index into serving_pool(): a
    CVRPTW instance with probability `cvrptw_frac`, else a uniformly drawn
    member of the batch mix."""
    st = Stream(index, 10)
    out = []
    t = 0.0
    while True:
        t += -math.log(float(st.unit(1)[0])) / rate
        if t >= duration:
            break
        u = int(st.ints(0, 999, 1)[0])
        if u < int(round(cvrptw_frac * 1000)):
            k = pool_mix + int(st.ints(0, pool_cvrptw - 1, 1)[0])
        else:
            k = int(st.ints(0, pool_mix - 1, 1)[0])
        out.append((t, k))
    return out


def poisson_trace(rate: float = 200.0, duration: float = 60.0, index: int = 7,
                  cvrptw_frac: float = 0.15) -> list[dict]:
    """Serving trace: exponential inter-arrivals (rate per second) over
    ``duration`` seconds; each request is a CVRPTW instance with probability
    ``cvrptw_frac`` and otherwise a draw from the batch mixture's classes.
    Returns [{'t': arrival_seconds, 'inst': instance dict}, ...]."""
    st = Stream(index, 9)
    out = []
    t = 0.0
    i = 0
    while True:
        t += -math.log(float(st.unit(1)[0])) / rate
        if t >= duration:
            break
        u = int(st.ints(0, 999, 1)[0])
        sub = 500000 + 1000 * index + i
        if u < int(round(cvrptw_frac * 1000)):
            inst = cvrptw(100, sub)
        else:
            cls = int(st.ints(0, 4, 1)[0])  # 2/5 TSP, 2/5 knapsack, 1/5 GAP
            if cls < 2:
                inst = tsp_uniform(int(st.ints(50, 500, 1)[0]), sub)
            elif cls < 4:
                inst = knapsack(int(st.ints(100, 2000, 1)[0]), sub)
            else:
                inst = gap(int(st.ints(50, 300, 1)[0]), sub)
        inst["tag"] = i
        out.append(dict(t=t, inst=inst))
        i += 1
    return out

