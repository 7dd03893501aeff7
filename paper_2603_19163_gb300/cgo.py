"""Python binding of the cgo C ABI (include/cgo.h) — argument marshalling only.

Every function of the header is exposed under the same name with ctypes
types; ``Problem`` is a small convenience wrapper that builds a
``cgo_problem_desc`` from an instance dict (numpy arrays, or torch tensors on
the GPU) and converts parameter/state structs to and from plain dicts.
All search work runs in the CUDA library; there is no Python or CPU path.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

NOPS = 8        # slots of the first operator arrays of cgo_params / cgo_state
NROW = 3        # the row level's slots (8 .. 10), in arrays of their own
NOPS_ALL = NOPS + NROW
OK, ERR_INVALID, ERR_NOMEM, ERR_CUDA, ERR_UNSUPPORTED, ERR_TIMEOUT, ERR_BUSY, ERR_STATE, \
    ERR_CANCELLED = range(9)
STATUS_NAMES = ["OK", "INVALID", "NOMEM", "CUDA", "UNSUPPORTED", "TIMEOUT", "BUSY", "STATE",
                "CANCELLED"]
TSP, QAP, KNAPSACK, GAP, CVRPTW = range(5)
ENC_PERM, ENC_BINARY, ENC_INTEGER = range(3)
MODEL_ENCODING = {TSP: ENC_PERM, QAP: ENC_PERM, KNAPSACK: ENC_BINARY, GAP: ENC_INTEGER,
                  CVRPTW: ENC_PERM}

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)


class cgo_problem_desc(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("encoding", ctypes.c_int32),
                ("model", ctypes.c_int32), ("n", ctypes.c_int32),
                ("mat0", ctypes.c_void_p), ("mat1", ctypes.c_void_p),
                ("vec0", ctypes.c_void_p), ("vec1", ctypes.c_void_p),
                ("vec2", ctypes.c_void_p), ("vec3", ctypes.c_void_p),
                ("capacity", ctypes.c_int64), ("lb", ctypes.c_int32), ("ub", ctypes.c_int32),
                ("m", ctypes.c_int32), ("vehicles", ctypes.c_int32),
                ("penalty0", ctypes.c_int64), ("penalty1", ctypes.c_int64),
                ("pointers_on_device", ctypes.c_int32), ("instance_tag", ctypes.c_uint32),
                ("weight_distance", ctypes.c_int64), ("weight_vehicles", ctypes.c_int64),
                ("weight_longest", ctypes.c_int64),
                ("lex_n", ctypes.c_int32), ("lex_obj", ctypes.c_int32 * 3),
                ("lex_tol", ctypes.c_int64 * 3)]


# CVRPTW objectives of the lexicographic mode (cgo_problem_desc.lex_obj)
LEX_DISTANCE, LEX_VEHICLES, LEX_LONGEST = 0, 1, 2


class cgo_params(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("population", ctypes.c_int32),
                ("candidates", ctypes.c_int32), ("generations", ctypes.c_int64),
                ("op_mask", ctypes.c_uint32), ("op_w0_q16", ctypes.c_uint32 * NOPS),
                ("k_w0_q16", ctypes.c_uint32 * 3), ("T0_q32", ctypes.c_uint64),
                ("alpha_q32", ctypes.c_uint64), ("aos_interval", ctypes.c_uint32),
                ("ema_alpha_q16", ctypes.c_uint32), ("w_floor_q16", ctypes.c_uint32),
                ("w_cap_q16", ctypes.c_uint32), ("op_cap_q16", ctypes.c_uint32 * NOPS),
                ("stag_limit", ctypes.c_uint32), ("elite_period", ctypes.c_uint32),
                ("init_oversample", ctypes.c_uint32), ("init_heuristic", ctypes.c_uint32),
                ("islands", ctypes.c_uint32), ("migrate_period", ctypes.c_uint32),
                ("migrate_strategy", ctypes.c_uint32), ("migrate_n", ctypes.c_uint32),
                ("cross_q16", ctypes.c_uint32), ("row_w0_q16", ctypes.c_uint32 * NROW),
                ("row_cap_q16", ctypes.c_uint32 * NROW)]


class cgo_state(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("population", ctypes.c_int32),
                ("length", ctypes.c_int32), ("generation", ctypes.c_int64),
                ("T_q32", ctypes.c_uint64), ("w_op_q16", ctypes.c_uint32 * NOPS),
                ("w_k_q16", ctypes.c_uint32 * 3), ("stag", ctypes.c_uint32),
                ("elite_prev", ctypes.c_int64), ("u_op", ctypes.c_uint32 * NOPS),
                ("v_op", ctypes.c_uint32 * NOPS), ("u_k", ctypes.c_uint32 * 3),
                ("v_k", ctypes.c_uint32 * 3), ("cur", _i32p), ("best_sol", _i32p),
                ("cost", _i64p), ("best_cost", _i64p), ("w_row_q16", ctypes.c_uint32 * NROW),
                ("u_row", ctypes.c_uint32 * NROW), ("v_row", ctypes.c_uint32 * NROW)]


class cgo_server_cfg(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("max_slots", ctypes.c_int32),
                ("hbm_budget_bytes", ctypes.c_int64), ("smem_budget_bytes", ctypes.c_int64),
                ("slice_generations", ctypes.c_int64), ("max_queued", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("slice_by_model", ctypes.c_int64 * 5)]


class cgo_server_info(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("queued", ctypes.c_int32),
                ("active", ctypes.c_int32), ("buckets", ctypes.c_int32),
                ("slices", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("hbm_used_bytes", ctypes.c_int64)]


class cgo_launch(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("warps_per_cta", ctypes.c_int32),
                ("warps_per_member", ctypes.c_int32), ("staging", ctypes.c_int32),
                ("gens_in_flight", ctypes.c_int32)]


_LIB = None
_LOCK = threading.Lock()


def lib() -> ctypes.CDLL:
    """Load (building first if needed) the in-tree CUDA library."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            path = _build.LIB
            if os.environ.get("CGO_NO_BUILD") != "1":
                path = _build.build()
            if not os.path.exists(path):
                raise ImportError("libcgo.so is not built (run __graft_entry__.build())")
            L = ctypes.CDLL(path)
            P, c = ctypes.POINTER, ctypes
            vp = c.c_void_p
            sigs = {
                "cgo_problem_create": ([P(cgo_problem_desc), P(vp)], c.c_int),
                "cgo_problem_destroy": ([vp], c.c_int),
                "cgo_params_default": ([vp, P(cgo_params)], c.c_int),
                "cgo_set_launch": ([vp, P(cgo_launch)], c.c_int),
                "cgo_get_launch": ([vp, P(cgo_launch)], c.c_int),
                "cgo_solve": ([vp, P(cgo_params), c.c_uint64, vp], c.c_int),
                "cgo_solve_continue": ([vp, c.c_int64, vp], c.c_int),
                "cgo_best": ([vp, _i32p, c.c_int32, _i64p], c.c_int),
                "cgo_solution_length": ([vp, _i32p], c.c_int),
                "cgo_best_rows": ([vp, _i32p, c.c_int32, _i32p, c.c_int32, _i32p, _i64p], c.c_int),
                "cgo_state_get": ([vp, P(cgo_state)], c.c_int),
                "cgo_op_counts": ([vp, P(c.c_uint64), c.c_int32], c.c_int),
                "cgo_state_export": ([vp, vp, c.c_size_t, P(c.c_size_t)], c.c_int),
                "cgo_state_import": ([vp, P(cgo_params), c.c_uint64, vp, c.c_size_t], c.c_int),
                "cgo_state_set": ([vp, P(cgo_params), c.c_uint64, P(cgo_state)], c.c_int),
                "cgo_solve_batch": ([P(vp), P(cgo_params), P(c.c_uint64), c.c_int32, vp], c.c_int),
                "cgo_last_error": ([], c.c_char_p),
                "cgo_version": ([], c.c_char_p),
                "cgo_kernel_launches": ([P(c.c_uint64)], c.c_int),
                "cgo_gather_peak": ([c.c_int32, c.c_int32, P(c.c_double), P(c.c_double)], c.c_int),
                "cgo_debug_inject": ([vp, c.c_int32, c.c_int64], c.c_int),
                "cgo_last_kernel_time": ([vp, P(c.c_double), _i64p], c.c_int),
                "cgo_solve_static": ([P(cgo_problem_desc), P(cgo_params), c.c_uint64, vp, vp, vp],
                                     c.c_int),
                "cgo_server_create": ([P(cgo_server_cfg), P(vp)], c.c_int),
                "cgo_submit": ([vp, vp, P(cgo_params), c.c_uint64, P(c.c_uint64)], c.c_int),
                "cgo_wait": ([vp, c.c_uint64, c.c_int32, _i64p, P(c.c_double)], c.c_int),
                "cgo_server_stats": ([vp, P(cgo_server_info)], c.c_int),
                "cgo_server_destroy": ([vp], c.c_int),
                "cgo_cancel": ([vp, c.c_uint64], c.c_int),
            }
            for name, (args, res) in sigs.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _LIB = L
    return _LIB


class CgoError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().cgo_last_error().decode()
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__("%s: CGO_ERR_%s: %s" % (where, name, msg))


def check(status: int, where: str) -> None:
    if status != OK:
        raise CgoError(status, where)


def gather_peak(kind: int, log2_elements: int) -> tuple[float, float]:
    """(gathers/s, kernel ms) of the random-gather microbenchmark: kind 0
    shared memory (16-bit entries), kind 1 global memory (32-bit entries)."""
    g, ms = ctypes.c_double(0), ctypes.c_double(0)
    check(lib().cgo_gather_peak(int(kind), int(log2_elements), ctypes.byref(g), ctypes.byref(ms)),
          "cgo_gather_peak")
    return float(g.value), float(ms.value)


def kernel_launches() -> int:
    """Kernels the library has launched in this process so far."""
    v = ctypes.c_uint64(0)
    check(lib().cgo_kernel_launches(ctypes.byref(v)), "cgo_kernel_launches")
    return int(v.value)


# ------------------------------------------------------------------ params
PARAM_MAP = [("P", "population"), ("C", "candidates"), ("G", "generations"),
             ("op_mask", "op_mask"), ("w_op", "op_w0_q16"), ("w_k", "k_w0_q16"),
             ("T0", "T0_q32"), ("alpha", "alpha_q32"), ("U", "aos_interval"),
             ("ema_a", "ema_alpha_q16"), ("w_floor", "w_floor_q16"), ("w_cap", "w_cap_q16"),
             ("op_cap", "op_cap_q16"), ("stag_limit", "stag_limit"),
             ("elite_period", "elite_period"), ("init_oversample", "init_oversample"),
             ("init_heuristic", "init_heuristic"), ("islands", "islands"),
             ("migrate_period", "migrate_period"), ("migrate_strategy", "migrate_strategy"),
             ("migrate_n", "migrate_n"), ("cross_q16", "cross_q16")]


# per-slot lists of the dict (NOPS_ALL entries) and the two C arrays they fill
SLOT_ARRAYS = {"op_w0_q16": "row_w0_q16", "op_cap_q16": "row_cap_q16"}


def params_struct(d: dict) -> cgo_params:
    q = cgo_params()
    q.struct_size = ctypes.sizeof(cgo_params)
    for i in range(NROW):
        q.row_cap_q16[i] = 65536
    for k, f in PARAM_MAP:
        if k not in d:
            continue
        v = d[k]
        if isinstance(v, (list, tuple, np.ndarray)):
            arr, row = getattr(q, f), getattr(q, SLOT_ARRAYS[f]) if f in SLOT_ARRAYS else None
            for i, x in enumerate(v):
                if i < len(arr):
                    arr[i] = int(x)
                else:
                    row[i - len(arr)] = int(x)
        else:
            setattr(q, f, int(v))
    return q


def params_dict(q: cgo_params) -> dict:
    d = {}
    for k, f in PARAM_MAP:
        v = getattr(q, f)
        d[k] = list(v) if hasattr(v, "__len__") else int(v)
        if f in SLOT_ARRAYS:
            d[k] += list(getattr(q, SLOT_ARRAYS[f]))
    return d


def _ptr(a, keep, device):
    if a is None:
        return None
    if device:
        return int(a.data_ptr())
    x = np.ascontiguousarray(np.asarray(a, dtype=np.int32).reshape(-1))
    keep.append(x)
    return x.ctypes.data


class Problem:
    """A cgo_problem handle built from an instance dict."""

    def __init__(self, inst: dict, on_device: bool = False):
        L = lib()
        keep = []
        d = cgo_problem_desc()
        d.struct_size = ctypes.sizeof(cgo_problem_desc)
        d.model = int(inst["model"])
        d.encoding = MODEL_ENCODING[d.model]
        d.n = int(inst["n"])
        for f in ("mat0", "mat1", "vec0", "vec1", "vec2", "vec3"):
            setattr(d, f, _ptr(inst.get(f), keep, on_device))
        d.capacity = int(inst.get("capacity", 0))
        d.lb = int(inst.get("lb", 0))
        d.ub = int(inst.get("ub", 0))
        d.m = int(inst.get("m", 0))
        d.vehicles = int(inst.get("vehicles", 0))
        d.penalty0 = int(inst.get("penalty0", 0))
        d.penalty1 = int(inst.get("penalty1", 0))
        d.weight_distance = int(inst.get("weight_distance", 0))
        d.weight_vehicles = int(inst.get("weight_vehicles", 0))
        d.weight_longest = int(inst.get("weight_longest", 0))
        # lexicographic mode: [(objective, tolerance), ...] in priority order
        lex = list(inst.get("lexicographic", ()))
        d.lex_n = len(lex)
        for i, (obj, tol) in enumerate(lex[:3]):
            d.lex_obj[i] = int(obj)
            d.lex_tol[i] = int(tol)
        d.pointers_on_device = 1 if on_device else 0
        d.instance_tag = int(inst.get("tag", 0)) & 0xFFFFFFFF
        h = ctypes.c_void_p()
        check(L.cgo_problem_create(ctypes.byref(d), ctypes.byref(h)), "cgo_problem_create")
        self.h = h
        self.inst = inst
        n = ctypes.c_int32()
        check(L.cgo_solution_length(h, ctypes.byref(n)), "cgo_solution_length")
        self.length = n.value

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().cgo_problem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def default_params(self) -> dict:
        q = cgo_params()
        check(lib().cgo_params_default(self.h, ctypes.byref(q)), "cgo_params_default")
        return params_dict(q)

    def set_launch(self, warps: int = 0, staging: int = 0, wpm: int = 0, ns: int = 0):
        """Launch override (0 = automatic): warps per CTA, staging mode,
        warps per member generation, generations in flight."""
        l = cgo_launch(ctypes.sizeof(cgo_launch), warps, wpm, staging, ns)
        check(lib().cgo_set_launch(self.h, ctypes.byref(l)), "cgo_set_launch")

    def get_launch(self) -> tuple[int, int, int, int]:
        """(warps per CTA, warps per member generation, staging, generations
        in flight) of the last solve."""
        l = cgo_launch()
        check(lib().cgo_get_launch(self.h, ctypes.byref(l)), "cgo_get_launch")
        return l.warps_per_cta, l.warps_per_member, l.staging, l.gens_in_flight

    def solve(self, params: dict, seed: int, stream=None):
        q = params_struct(params)
        check(lib().cgo_solve(self.h, ctypes.byref(q), int(seed), _stream(stream)), "cgo_solve")
        return self

    def solve_continue(self, generations: int, stream=None):
        check(lib().cgo_solve_continue(self.h, int(generations), _stream(stream)),
              "cgo_solve_continue")
        return self

    def best(self) -> tuple[np.ndarray, int]:
        sol = np.zeros(self.length, np.int32)
        c = ctypes.c_int64()
        check(lib().cgo_best(self.h, sol.ctypes.data_as(_i32p), self.length, ctypes.byref(c)),
              "cgo_best")
        return sol, c.value

    def best_rows(self) -> tuple[list, int]:
        """The elite as rows (CVRPTW: one list of customers per route)."""
        n = int(self.inst["n"])
        rows = int(self.inst.get("vehicles", 1)) if int(self.inst["model"]) == CVRPTW else 1
        flat = np.zeros(max(n, self.length), np.int32)
        lens = np.zeros(rows, np.int32)
        cnt, c = ctypes.c_int32(), ctypes.c_int64()
        check(lib().cgo_best_rows(self.h, flat.ctypes.data_as(_i32p), len(flat),
                                  lens.ctypes.data_as(_i32p), rows, ctypes.byref(cnt),
                                  ctypes.byref(c)), "cgo_best_rows")
        out, o = [], 0
        for L in lens[:cnt.value]:
            out.append(flat[o:o + L].tolist())
            o += int(L)
        return out, c.value

    def state(self) -> dict:
        s = cgo_state()
        s.struct_size = ctypes.sizeof(cgo_state)
        check(lib().cgo_state_get(self.h, ctypes.byref(s)), "cgo_state_get")
        P, n = s.population, s.length
        arr = dict(cur=np.zeros((P, n), np.int32), best_sol=np.zeros((P, n), np.int32),
                   cost=np.zeros(P, np.int64), best_cost=np.zeros(P, np.int64))
        s.cur = arr["cur"].ctypes.data_as(_i32p)
        s.best_sol = arr["best_sol"].ctypes.data_as(_i32p)
        s.cost = arr["cost"].ctypes.data_as(_i64p)
        s.best_cost = arr["best_cost"].ctypes.data_as(_i64p)
        check(lib().cgo_state_get(self.h, ctypes.byref(s)), "cgo_state_get")
        arr.update(P=P, len=n, g=s.generation, T=s.T_q32,
                   w_op=list(s.w_op_q16) + list(s.w_row_q16),
                   w_k=list(s.w_k_q16), stag=s.stag, elite_prev=s.elite_prev,
                   u_op=list(s.u_op) + list(s.u_row), v_op=list(s.v_op) + list(s.v_row),
                   u_k=list(s.u_k), v_k=list(s.v_k))
        return arr

    def export_state(self) -> bytes:
        """The search state as a versioned byte buffer (cgo_state_export)."""
        used = ctypes.c_size_t()
        lib().cgo_state_export(self.h, None, 0, ctypes.byref(used))    # sizes the buffer
        buf = ctypes.create_string_buffer(used.value)
        check(lib().cgo_state_export(self.h, buf, used.value, ctypes.byref(used)), "cgo_state_export")
        return buf.raw[:used.value]

    def import_state(self, params: dict, seed: int, blob: bytes):
        q = params_struct(params)
        buf = ctypes.create_string_buffer(blob, len(blob))
        check(lib().cgo_state_import(self.h, ctypes.byref(q), int(seed), buf, len(blob)),
              "cgo_state_import")

    def op_counts(self) -> dict:
        """Operator and k-level counts over every generation of the solve so far."""
        n = NOPS_ALL
        out = (ctypes.c_uint64 * (2 * n + 6))()
        check(lib().cgo_op_counts(self.h, out, 2 * n + 6), "cgo_op_counts")
        v = list(out)
        return dict(u_op=v[0:n], v_op=v[n:2 * n], u_k=v[2 * n:2 * n + 3],
                    v_k=v[2 * n + 3:2 * n + 6])

    def set_state(self, params: dict, seed: int, st: dict):
        s = cgo_state()
        s.struct_size = ctypes.sizeof(cgo_state)
        s.population, s.length, s.generation, s.T_q32 = st["P"], st["len"], st["g"], st["T"]
        rows = {"w_op_q16": "w_row_q16", "u_op": "u_row", "v_op": "v_row"}
        for f_py, f_c in (("w_op", "w_op_q16"), ("w_k", "w_k_q16"), ("u_op", "u_op"),
                          ("v_op", "v_op"), ("u_k", "u_k"), ("v_k", "v_k")):
            arr = getattr(s, f_c)
            for i, x in enumerate(st[f_py]):
                if i < len(arr):
                    arr[i] = int(x)
                else:
                    getattr(s, rows[f_c])[i - len(arr)] = int(x)
        s.stag, s.elite_prev = st["stag"], st["elite_prev"]
        keep = {k: np.ascontiguousarray(st[k], dtype=np.int32 if k in ("cur", "best_sol")
                                        else np.int64) for k in ("cur", "best_sol", "cost",
                                                                 "best_cost")}
        s.cur = keep["cur"].ctypes.data_as(_i32p)
        s.best_sol = keep["best_sol"].ctypes.data_as(_i32p)
        s.cost = keep["cost"].ctypes.data_as(_i64p)
        s.best_cost = keep["best_cost"].ctypes.data_as(_i64p)
        q = params_struct(params)
        check(lib().cgo_state_set(self.h, ctypes.byref(q), int(seed), ctypes.byref(s)),
              "cgo_state_set")

    def last_kernel_time(self) -> tuple[float, int]:
        """(milliseconds, generations) of the last evolve-kernel launch."""
        ms = ctypes.c_double()
        g = ctypes.c_int64()
        check(lib().cgo_last_kernel_time(self.h, ctypes.byref(ms), ctypes.byref(g)),
              "cgo_last_kernel_time")
        return ms.value, g.value

    def inject(self, what: int, value: int):
        check(lib().cgo_debug_inject(self.h, int(what), int(value)), "cgo_debug_inject")


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return int(stream.cuda_stream)
    return int(stream)


def solve_batch(problems: list, params: list, seeds: list, stream=None) -> None:
    n = len(problems)
    hs = (ctypes.c_void_p * n)(*[p.h.value for p in problems])
    qs = (cgo_params * n)(*[params_struct(d) for d in params])
    ss = (ctypes.c_uint64 * n)(*[int(s) for s in seeds])
    check(lib().cgo_solve_batch(hs, qs, ss, n, _stream(stream)), "cgo_solve_batch")


def version() -> str:
    return lib().cgo_version().decode()


class Server:
    """A cgo_server: continuous batching of solve requests."""

    def __init__(self, max_slots: int = 1024, hbm_budget_bytes: int = 64 << 30,
                 smem_budget_bytes: int = 0, slice_generations: int = 2000, max_queued: int = 0,
                 slice_by_model: dict | None = None):
        """slice_by_model: {model: generations per slice} for the models whose
        requests should advance further (or less far) per slice than
        slice_generations."""
        per = [0] * 5
        for m, v in (slice_by_model or {}).items():
            per[int(m)] = int(v)
        cfg = cgo_server_cfg(ctypes.sizeof(cgo_server_cfg), max_slots, hbm_budget_bytes,
                             smem_budget_bytes, slice_generations, max_queued, 0,
                             (ctypes.c_int64 * 5)(*per))
        h = ctypes.c_void_p()
        check(lib().cgo_server_create(ctypes.byref(cfg), ctypes.byref(h)), "cgo_server_create")
        self.h = h

    def submit(self, prob: "Problem", params: dict, seed: int) -> int:
        q = params_struct(params)
        t = ctypes.c_uint64()
        check(lib().cgo_submit(self.h, prob.h, ctypes.byref(q), int(seed), ctypes.byref(t)),
              "cgo_submit")
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1) -> tuple[int, float]:
        c = ctypes.c_int64()
        lat = ctypes.c_double()
        check(lib().cgo_wait(self.h, int(ticket), int(timeout_ms), ctypes.byref(c),
                             ctypes.byref(lat)), "cgo_wait")
        return c.value, lat.value

    def cancel(self, ticket: int):
        check(lib().cgo_cancel(self.h, int(ticket)), "cgo_cancel")

    def stats(self) -> dict:
        i = cgo_server_info()
        i.struct_size = ctypes.sizeof(cgo_server_info)
        check(lib().cgo_server_stats(self.h, ctypes.byref(i)), "cgo_server_stats")
        return dict(queued=i.queued, active=i.active, buckets=i.buckets, slices=i.slices,
                    completed=i.completed, hbm_used_bytes=i.hbm_used_bytes)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().cgo_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
