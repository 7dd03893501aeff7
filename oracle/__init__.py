"""ctypes access to the CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg import this package.  It mirrors the C structs of ``oracle/oracle.h``
and converts instance dicts (from ``instances``) and parameter dicts into
them; the arithmetic itself lives in ``oracle.c``.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import build as _build

NOPS = 11
SWAP, TWO_OPT, INSERT, OR_OPT, FLIP, PERTURB, THREE_OPT, SEGMENT = range(8)
ROW_SWAP_OP, ROW_MERGE_OP, ROW_SPLIT_OP = 8, 9, 10     # operator slots of the row level
SEG_FLIP = SEG_RESET = SEGMENT     # slot 7: the binary and the integer segment operator

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)


class OrcInstance(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("n", ctypes.c_int32), ("m", ctypes.c_int32),
                ("vehicles", ctypes.c_int32),
                ("mat0", _i32p), ("mat1", _i32p),
                ("vec0", _i32p), ("vec1", _i32p), ("vec2", _i32p), ("vec3", _i32p),
                ("capacity", ctypes.c_int64), ("lb", ctypes.c_int32), ("ub", ctypes.c_int32),
                ("penalty0", ctypes.c_int64), ("penalty1", ctypes.c_int64),
                ("tag", ctypes.c_uint32), ("weight0", ctypes.c_int64), ("weight1", ctypes.c_int64),
                ("weight2", ctypes.c_int64), ("lex_n", ctypes.c_int32),
                ("lex_obj", ctypes.c_int32 * 3), ("lex_tol", ctypes.c_int64 * 3),
                ("lex_dmax", ctypes.c_int64)]

# CVRPTW objectives of the lexicographic mode [R37]
LEX_DISTANCE, LEX_VEHICLES, LEX_LONGEST = 0, 1, 2


class OrcParams(ctypes.Structure):
    _fields_ = [("P", ctypes.c_int32), ("C", ctypes.c_int32), ("op_mask", ctypes.c_uint32),
                ("w_op", ctypes.c_uint32 * NOPS), ("w_k", ctypes.c_uint32 * 3),
                ("T0", ctypes.c_uint64), ("alpha", ctypes.c_uint64),
                ("U", ctypes.c_uint32), ("ema_a", ctypes.c_uint32), ("w_floor", ctypes.c_uint32),
                ("w_cap", ctypes.c_uint32), ("op_cap", ctypes.c_uint32 * NOPS),
                ("stag_limit", ctypes.c_uint32), ("elite_period", ctypes.c_uint32),
                ("init_oversample", ctypes.c_uint32), ("init_heuristic", ctypes.c_uint32),
                ("islands", ctypes.c_uint32), ("migrate_period", ctypes.c_uint32),
                ("migrate_strategy", ctypes.c_uint32), ("migrate_n", ctypes.c_uint32),
                ("cross_q16", ctypes.c_uint32)]


class OrcState(ctypes.Structure):
    _fields_ = [("P", ctypes.c_int32), ("len", ctypes.c_int32), ("g", ctypes.c_int64),
                ("T", ctypes.c_uint64), ("w_op", ctypes.c_uint32 * NOPS),
                ("w_k", ctypes.c_uint32 * 3), ("stag", ctypes.c_uint32),
                ("elite_prev", ctypes.c_int64),
                ("u_op", ctypes.c_uint32 * NOPS), ("v_op", ctypes.c_uint32 * NOPS),
                ("u_k", ctypes.c_uint32 * 3), ("v_k", ctypes.c_uint32 * 3),
                ("cur", _i32p), ("best_sol", _i32p), ("cost", _i64p), ("best_cost", _i64p),
                ("all_u_op", ctypes.c_uint64 * NOPS), ("all_v_op", ctypes.c_uint64 * NOPS),
                ("all_u_k", ctypes.c_uint64 * 3), ("all_v_k", ctypes.c_uint64 * 3)]


_LIB = None
_LOCK = threading.Lock()


def lib() -> ctypes.CDLL:
    global _LIB
    with _LOCK:
        if _LIB is None:
            L = ctypes.CDLL(_build.build())
            u32, i32, i64, u64 = ctypes.c_uint32, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
            L.orc_philox.argtypes = [ctypes.POINTER(u32), ctypes.POINTER(u32), ctypes.POINTER(u32)]
            L.orc_pos.argtypes = [u32, u32]
            L.orc_pos.restype = u32
            L.orc_wsample.argtypes = [ctypes.POINTER(u32), i32, u32]
            L.orc_wsample.restype = i32
            L.orc_log2_q32.argtypes = [u32]
            L.orc_log2_q32.restype = u64
            L.orc_exp_q32.argtypes = [u32]
            L.orc_exp_q32.restype = u64
            L.orc_accept.argtypes = [i64, u64, u32]
            L.orc_accept.restype = i32
            L.orc_cool.argtypes = [u64, u64]
            L.orc_cool.restype = u64
            L.orc_apply_move.argtypes = [ctypes.POINTER(OrcInstance), i32, u32, u32, u32, _i32p, i32]
            L.orc_apply_move.restype = i32
            L.orc_aos_level.argtypes = [ctypes.POINTER(u32), ctypes.POINTER(u32),
                                        ctypes.POINTER(u32), _i32p, ctypes.POINTER(u32), i32,
                                        u32, u32, u32]
            L.orc_params_default.argtypes = [ctypes.POINTER(OrcInstance), ctypes.POINTER(OrcParams)]
            L.orc_solution_length.argtypes = [ctypes.POINTER(OrcInstance)]
            L.orc_solution_length.restype = i32
            L.orc_cost.argtypes = [ctypes.POINTER(OrcInstance), _i32p]
            L.orc_cost.restype = i64
            L.orc_valid.argtypes = [ctypes.POINTER(OrcInstance), _i32p]
            L.orc_valid.restype = i32
            L.orc_enabled_ops.argtypes = [ctypes.POINTER(OrcInstance), u32, _i32p]
            L.orc_enabled_ops.restype = i32
            L.orc_init.argtypes = [ctypes.POINTER(OrcInstance), ctypes.POINTER(OrcParams), u64,
                                   ctypes.POINTER(OrcState)]
            L.orc_init.restype = i32
            L.orc_migrate.argtypes = [ctypes.POINTER(OrcParams), ctypes.POINTER(OrcState)]
            L.orc_migrate.restype = i32
            L.orc_crossover.argtypes = [ctypes.POINTER(OrcInstance), ctypes.POINTER(OrcParams), u64,
                                        ctypes.POINTER(OrcState)]
            L.orc_crossover.restype = i32
            L.orc_ox.argtypes = [_i32p, _i32p, i32, i32, i32, _i32p]
            L.orc_row_move.argtypes = [ctypes.POINTER(OrcInstance), i32, u32, u32, _i32p, i32]
            L.orc_row_move.restype = i32
            L.orc_heuristic_perms.argtypes = [ctypes.POINTER(OrcInstance), _i32p]
            L.orc_heuristic_perms.restype = i32
            L.orc_run.argtypes = [ctypes.POINTER(OrcInstance), ctypes.POINTER(OrcParams), u64,
                                  ctypes.POINTER(OrcState), i64, i32]
            L.orc_run.restype = i32
            L.orc_elite.argtypes = [ctypes.POINTER(OrcState)]
            L.orc_elite.restype = i32
            L.orc_threads.argtypes = [i32]
            L.orc_threads.restype = i32
            _LIB = L
    return _LIB


def _arr(a):
    if a is None:
        return None, None
    x = np.ascontiguousarray(np.asarray(a, dtype=np.int32).reshape(-1))
    return x, x.ctypes.data_as(_i32p)


class Instance:
    """Owns the int32 copies behind an OrcInstance."""

    def __init__(self, inst: dict):
        self.inst = inst
        self.keep = []
        s = OrcInstance()
        s.model = int(inst["model"])
        s.n = int(inst["n"])
        s.m = int(inst.get("m", 0))
        s.vehicles = int(inst.get("vehicles", 0))
        for f in ("mat0", "mat1", "vec0", "vec1", "vec2", "vec3"):
            arr, ptr = _arr(inst.get(f))
            if arr is not None:
                self.keep.append(arr)
                setattr(s, f, ptr)
        s.capacity = int(inst.get("capacity", 0))
        s.lb = int(inst.get("lb", 0))
        s.ub = int(inst.get("ub", 0))
        s.penalty0 = int(inst.get("penalty0", 0))
        s.penalty1 = int(inst.get("penalty1", 0))
        s.weight0 = int(inst.get("weight_distance", 0))
        s.weight1 = int(inst.get("weight_vehicles", 0))
        s.weight2 = int(inst.get("weight_longest", 0))
        # [R37] lexicographic mode: [(objective, tolerance), ...] in priority order
        lex = list(inst.get("lexicographic", ()))
        s.lex_n = len(lex)
        for i, (obj, tol) in enumerate(lex):
            s.lex_obj[i] = int(obj)
            s.lex_tol[i] = int(tol)
        if lex:
            maxd = int(np.max(np.asarray(inst["mat0"], np.int64)))
            s.lex_dmax = (int(inst["n"]) + int(inst["vehicles"])) * max(maxd, 0)
        s.tag = int(inst.get("tag", 0)) & 0xFFFFFFFF
        self.s = s

    @property
    def ref(self):
        return ctypes.byref(self.s)

    def length(self) -> int:
        return int(lib().orc_solution_length(self.ref))


PARAM_KEYS = ("P", "C", "op_mask", "w_op", "w_k", "T0", "alpha", "U", "ema_a", "w_floor",
              "w_cap", "op_cap", "stag_limit", "elite_period", "init_oversample", "init_heuristic",
              "islands", "migrate_period", "migrate_strategy", "migrate_n", "cross_q16")


def default_params(inst: dict) -> dict:
    """The oracle's own defaults for this instance, as a plain dict."""
    I = Instance(inst)
    p = OrcParams()
    lib().orc_params_default(I.ref, ctypes.byref(p))
    return params_to_dict(p)


def params_to_dict(p: OrcParams) -> dict:
    d = {}
    for k in PARAM_KEYS:
        v = getattr(p, k)
        d[k] = list(v) if hasattr(v, "__len__") else int(v)
    return d


def make_params(d: dict) -> OrcParams:
    p = OrcParams()
    for k in PARAM_KEYS:
        v = d[k]
        if isinstance(v, (list, tuple, np.ndarray)):
            arr = getattr(p, k)
            for i, x in enumerate(v):
                arr[i] = int(x)
        else:
            setattr(p, k, int(v))
    return p


def new_state(P: int, length: int) -> tuple[OrcState, dict]:
    arrays = dict(cur=np.zeros((P, length), np.int32), best_sol=np.zeros((P, length), np.int32),
                  cost=np.zeros(P, np.int64), best_cost=np.zeros(P, np.int64))
    st = OrcState()
    st.P, st.len = P, length
    st.cur = arrays["cur"].ctypes.data_as(_i32p)
    st.best_sol = arrays["best_sol"].ctypes.data_as(_i32p)
    st.cost = arrays["cost"].ctypes.data_as(_i64p)
    st.best_cost = arrays["best_cost"].ctypes.data_as(_i64p)
    return st, arrays


def migrate(params: dict, state: dict) -> dict:
    """One migration step (islands) applied to a copy of a state dict with
    fields cur, best_sol, cost, best_cost, g (the rest is carried over)."""
    P, length = int(state["cur"].shape[0]), int(state["cur"].shape[1])
    st, arrays = new_state(P, length)
    for k in ("cur", "best_sol", "cost", "best_cost"):
        arrays[k][...] = state[k]
    st.g = int(state["g"])
    p = make_params(params)
    if lib().orc_migrate(ctypes.byref(p), ctypes.byref(st)) != 0:
        raise ValueError("orc_migrate failed")
    out = dict(state)
    out.update({k: v.copy() for k, v in arrays.items()})
    return out


ROW_SWAP, ROW_MERGE, ROW_SPLIT = range(3)


def row_move(inst: dict, kind: int, a: int, b: int, sol) -> np.ndarray:
    """A row operator (row_swap / row_merge / row_split) on a CVRPTW solution."""
    I = Instance(inst)
    s = np.ascontiguousarray(np.asarray(sol, dtype=np.int32).copy())
    if int(inst["model"]) == 4 and len(s) != int(inst["n"]) + int(inst.get("vehicles", 0)) - 1:
        raise ValueError("a CVRPTW solution has n + vehicles - 1 symbols")
    rc = lib().orc_row_move(I.ref, kind, a, b, s.ctypes.data_as(_i32p), len(s))
    if rc == -1:
        raise ValueError("row operators need a CVRPTW instance")
    if rc != 0:
        raise ValueError("malformed CVRPTW solution (need exactly vehicles - 1 separators)")
    return s


def ox(A, B, lo: int, hi: int) -> np.ndarray:
    """Order crossover of two permutations keeping A[lo..hi]."""
    A = np.ascontiguousarray(A, dtype=np.int32)
    B = np.ascontiguousarray(B, dtype=np.int32)
    out = np.zeros(len(A), np.int32)
    lib().orc_ox(A.ctypes.data_as(_i32p), B.ctypes.data_as(_i32p), len(A), lo, hi,
                 out.ctypes.data_as(_i32p))
    return out


def crossover(inst: dict, params: dict, seed: int, state: dict) -> dict:
    """One crossover step of the population applied to a copy of a state dict
    with fields cur, best_sol, cost, best_cost, g, T (the rest is carried over)."""
    P, length = int(state["cur"].shape[0]), int(state["cur"].shape[1])
    st, arrays = new_state(P, length)
    for k in ("cur", "best_sol", "cost", "best_cost"):
        arrays[k][...] = state[k]
    st.g, st.T = int(state["g"]), int(state["T"])
    I = Instance(inst)
    p = make_params(params)
    if lib().orc_crossover(I.ref, ctypes.byref(p), seed, ctypes.byref(st)) != 0:
        raise ValueError("orc_crossover failed")
    out = dict(state)
    out.update({k: v.copy() for k, v in arrays.items()})
    return out


def state_dict(st: OrcState, arrays: dict) -> dict:
    d = {k: v.copy() for k, v in arrays.items()}
    d.update(P=st.P, len=st.len, g=st.g, T=st.T, w_op=list(st.w_op), w_k=list(st.w_k),
             stag=st.stag, elite_prev=st.elite_prev, u_op=list(st.u_op), v_op=list(st.v_op),
             u_k=list(st.u_k), v_k=list(st.v_k),
             op_counts=dict(u_op=list(st.all_u_op), v_op=list(st.all_v_op), u_k=list(st.all_u_k),
                            v_k=list(st.all_v_k)))
    return d


class Solver:
    """One oracle search: init with a seed, then run generations."""

    def __init__(self, inst: dict, params: dict, seed: int):
        self.I = Instance(inst)
        self.params = params
        self.p = make_params(params)
        self.seed = int(seed)
        self.st, self.arrays = new_state(int(params["P"]), self.I.length())
        rc = lib().orc_init(self.I.ref, ctypes.byref(self.p), self.seed, ctypes.byref(self.st))
        if rc != 0:
            raise ValueError("orc_init failed")

    def run(self, generations: int, threads: int = 0) -> "Solver":
        rc = lib().orc_run(self.I.ref, ctypes.byref(self.p), self.seed, ctypes.byref(self.st),
                           int(generations), int(threads))
        if rc != 0:
            raise ValueError("orc_run failed")
        return self

    def state(self) -> dict:
        return state_dict(self.st, self.arrays)

    def elite(self) -> int:
        return int(lib().orc_elite(ctypes.byref(self.st)))


def solve(inst: dict, params: dict, seed: int, generations: int, threads: int = 0) -> dict:
    return Solver(inst, params, seed).run(generations, threads).state()


def heuristic_perms(inst: dict) -> np.ndarray:
    """The attribute-agnostic start permutations (H x n; H = 0 for models
    without square data matrices)."""
    I = Instance(inst)
    out = np.zeros(8 * int(inst["n"]), np.int32)
    H = int(lib().orc_heuristic_perms(I.ref, out.ctypes.data_as(_i32p)))
    return out[:H * int(inst["n"])].reshape(H, int(inst["n"]))


def cost(inst: dict, sol) -> int:
    I = Instance(inst)
    arr, ptr = _arr(sol)
    return int(lib().orc_cost(I.ref, ptr))


def valid(inst: dict, sol) -> bool:
    I = Instance(inst)
    arr, ptr = _arr(sol)
    return bool(lib().orc_valid(I.ref, ptr))


def philox(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox(c, k, o)
    return list(o)


def apply_move(inst: dict, op: int, a: int, b: int, x: int, sol) -> np.ndarray:
    I = Instance(inst)
    s = np.ascontiguousarray(np.asarray(sol, dtype=np.int32).copy())
    rc = lib().orc_apply_move(I.ref, op, a, b, x, s.ctypes.data_as(_i32p), len(s))
    if rc != 0:
        raise ValueError("move not applicable")
    return s


def enabled_ops(inst: dict, op_mask: int) -> list:
    """Which operators of the mask apply to the instance's encoding (0/1 per slot)."""
    I = Instance(inst)
    e = np.zeros(NOPS, np.int32)
    lib().orc_enabled_ops(I.ref, op_mask, e.ctypes.data_as(_i32p))
    return e.tolist()


def aos_level(w, u, v, enabled, cap_i, a, w_floor, w_cap):
    n = len(w)
    W = (ctypes.c_uint32 * n)(*w)
    Uu = (ctypes.c_uint32 * n)(*u)
    Vv = (ctypes.c_uint32 * n)(*v)
    E = (ctypes.c_int32 * n)(*enabled)
    Cc = (ctypes.c_uint32 * n)(*cap_i)
    lib().orc_aos_level(W, Uu, Vv, E, Cc, n, a, w_floor, w_cap)
    return list(W)
