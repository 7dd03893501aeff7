"""The C-ABI library loads and exports every entry point the header
declares; the ctypes structs match the C layout (no GPU needed)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cgo.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cgo_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("cgo_problem_create", "cgo_problem_destroy", "cgo_params_default", "cgo_solve",
                 "cgo_best", "cgo_solve_batch", "cgo_state_get", "cgo_state_set",
                 "cgo_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2603_19163_gb300 import cgo
    L = cgo.lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    assert cgo.version().startswith("cgo")


def test_ctypes_layout_matches_c():
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    from paper_2603_19163_gb300 import cgo
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "cgo.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(cgo_problem_desc), sizeof(cgo_params),
         sizeof(cgo_state), sizeof(cgo_launch));
  printf("%zu %zu %zu %zu\n", offsetof(cgo_params, generations), offsetof(cgo_params, T0_q32),
         offsetof(cgo_params, op_cap_q16), offsetof(cgo_state, cur));
  printf("%zu %zu\n", offsetof(cgo_problem_desc, capacity), offsetof(cgo_problem_desc, instance_tag));
  printf("%zu %zu %u %u\n", offsetof(cgo_problem_desc, lex_n), offsetof(cgo_problem_desc, lex_tol),
         CGO_DESC_SIZE_V1, CGO_DESC_SIZE_V2);
  printf("%zu %zu %u %u\n", sizeof(cgo_server_cfg), offsetof(cgo_server_cfg, slice_by_model),
         CGO_SERVER_CFG_SIZE_V1, CGO_SERVER_CFG_SIZE_V2);
  return 0;
}
"""
    d = os.path.join(ROOT, "tests", "_build")
    os.makedirs(d, exist_ok=True)
    c = os.path.join(d, "layout.c")
    exe = os.path.join(d, "layout")
    open(c, "w").write(src)
    subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), c, "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    want = [ctypes.sizeof(cgo.cgo_problem_desc), ctypes.sizeof(cgo.cgo_params),
            ctypes.sizeof(cgo.cgo_state), ctypes.sizeof(cgo.cgo_launch),
            cgo.cgo_params.generations.offset, cgo.cgo_params.T0_q32.offset,
            cgo.cgo_params.op_cap_q16.offset, cgo.cgo_state.cur.offset,
            cgo.cgo_problem_desc.capacity.offset, cgo.cgo_problem_desc.instance_tag.offset,
            cgo.cgo_problem_desc.lex_n.offset, cgo.cgo_problem_desc.lex_tol.offset,
            cgo.cgo_problem_desc.weight_longest.offset, cgo.cgo_problem_desc.lex_n.offset,
            ctypes.sizeof(cgo.cgo_server_cfg), cgo.cgo_server_cfg.slice_by_model.offset,
            cgo.cgo_server_cfg.max_queued.offset, cgo.cgo_server_cfg.slice_by_model.offset]
    assert [int(x) for x in out] == want


def test_errors_are_reported_without_a_gpu_call():
    from paper_2603_19163_gb300 import cgo
    L = cgo.lib()
    h = ctypes.c_void_p()
    d = cgo.cgo_problem_desc()
    d.struct_size = 3          # wrong size: rejected before any CUDA call
    assert L.cgo_problem_create(ctypes.byref(d), ctypes.byref(h)) == cgo.ERR_INVALID
    assert b"struct_size" in L.cgo_last_error()
    assert L.cgo_solve(None, None, 0, None) == cgo.ERR_INVALID


def test_server_config_checked_without_a_gpu_call():
    """cgo_server_create validates its configuration before any CUDA call:
    a negative per-model slice length, an unknown struct size."""
    from paper_2603_19163_gb300 import cgo
    L = cgo.lib()
    h = ctypes.c_void_p()
    per = (ctypes.c_int64 * 5)(0, 0, 0, -1, 0)
    cfg = cgo.cgo_server_cfg(ctypes.sizeof(cgo.cgo_server_cfg), 2, 1 << 30, 0, 100, 0, 0, per)
    assert L.cgo_server_create(ctypes.byref(cfg), ctypes.byref(h)) == cgo.ERR_INVALID
    assert b"slice_by_model" in L.cgo_last_error() and not h.value
    cfg = cgo.cgo_server_cfg(ctypes.sizeof(cgo.cgo_server_cfg) - 8, 2, 1 << 30, 0, 100, 0, 0)
    assert L.cgo_server_create(ctypes.byref(cfg), ctypes.byref(h)) == cgo.ERR_INVALID
    assert b"struct_size" in L.cgo_last_error()


def test_launch_counter_without_a_gpu():
    from paper_2603_19163_gb300 import cgo
    L = cgo.lib()
    assert L.cgo_kernel_launches(None) == cgo.ERR_INVALID
    before = cgo.kernel_launches()
    assert before >= 0
    assert cgo.kernel_launches() == before      # nothing launched in between


def test_gather_peak_rejects_bad_sizes_without_a_gpu():
    from paper_2603_19163_gb300 import cgo
    L = cgo.lib()
    g = ctypes.c_double(0)
    assert L.cgo_gather_peak(0, 17, ctypes.byref(g), None) == cgo.ERR_INVALID   # > 128 KB shared
    assert L.cgo_gather_peak(1, 29, ctypes.byref(g), None) == cgo.ERR_INVALID
    assert L.cgo_gather_peak(2, 12, ctypes.byref(g), None) == cgo.ERR_INVALID
    assert L.cgo_gather_peak(0, 12, None, None) == cgo.ERR_INVALID


def test_earlier_struct_sizes():
    """The structs before the row level was appended: their sizeof (tail
    padding included) is what CGO_PARAMS_SIZE_V1 / CGO_STATE_SIZE_V1 give."""
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    src = r"""
#include <stdio.h>
#include "cgo.h"
typedef struct {
  uint32_t struct_size; int32_t population, candidates; int64_t generations; uint32_t op_mask;
  uint32_t op_w0_q16[8], k_w0_q16[3]; uint64_t T0_q32, alpha_q32;
  uint32_t aos_interval, ema_alpha_q16, w_floor_q16, w_cap_q16, op_cap_q16[8], stag_limit,
      elite_period, init_oversample, init_heuristic, islands, migrate_period, migrate_strategy,
      migrate_n, cross_q16;
} params_v1;
typedef struct {
  uint32_t struct_size; int32_t population, length; int64_t generation; uint64_t T_q32;
  uint32_t w_op_q16[8], w_k_q16[3], stag; int64_t elite_prev;
  uint32_t u_op[8], v_op[8], u_k[3], v_k[3]; int32_t *cur, *best_sol; int64_t *cost, *best_cost;
} state_v1;
int main(void) {
  printf("%zu %u %zu %u\n", sizeof(params_v1), CGO_PARAMS_SIZE_V1, sizeof(state_v1), CGO_STATE_SIZE_V1);
  return 0;
}
"""
    d = os.path.join(ROOT, "tests", "_build")
    os.makedirs(d, exist_ok=True)
    c, exe = os.path.join(d, "v1.c"), os.path.join(d, "v1")
    open(c, "w").write(src)
    subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), c, "-o", exe], check=True)
    a, b, x, y = (int(v) for v in subprocess.run([exe], capture_output=True, text=True,
                                                   check=True).stdout.split())
    assert a == b and x == y
