"""Build the cgo CUDA library (libcgo.so) in-tree with nvcc for sm_103a.

The library is plain C ABI (include/cgo.h); the Python binding loads it with
ctypes.  Translation units are compiled in parallel, then linked.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libcgo.so")
# Kernel units: cgo_kernels.cu compiled again with CGO_UNIT defined, each
# instantiating a share of the kernel sets, so that they compile in parallel
# (cgo_kernels.cu itself keeps the host code and the benchmark's TSP set).
# Entry: object name, the population-step code compiled in (0 none, 1
# crossover, 2 island migration and crossover), then the sets as (name,
# model, int16 matrix, evolve shape mask, batch shape mask); the names are
# those declared in cgo_kernels.cu.  Batched solves use the sets 0 and 2;
# the crossover-only sets hold single-solve kernels.  CVRPTW's kernels are
# the slowest to compile and are spread over several units.
ALL_E, ALL_B, NO_B = "0xFFu", "0x7u", "0u"
UNITS = [
    ("x_cvrptw_a", 2, [("x_cvrptw_a", "CVRPTW", "false", "0x03u", NO_B)]),
    ("x_cvrptw_b", 2, [("x_cvrptw_b", "CVRPTW", "false", "0x0Cu", NO_B)]),
    ("x_cvrptw_c", 2, [("x_cvrptw_c", "CVRPTW", "false", "0x30u", NO_B)]),
    ("x_cvrptw_d", 2, [("x_cvrptw_d", "CVRPTW", "false", "0u", "0x3u")]),
    ("x_cvrptw_e", 2, [("x_cvrptw_e", "CVRPTW", "false", "0u", "0x4u")]),
    ("c_cvrptw_a", 1, [("c_cvrptw_a", "CVRPTW", "false", "0x03u", NO_B)]),
    ("c_cvrptw_b", 1, [("c_cvrptw_b", "CVRPTW", "false", "0x0Cu", NO_B)]),
    ("c_cvrptw_c", 1, [("c_cvrptw_c", "CVRPTW", "false", "0x30u", NO_B)]),
    ("p_cvrptw_a", 0, [("p_cvrptw_a", "CVRPTW", "false", "0x03u", NO_B)]),
    ("p_cvrptw_b", 0, [("p_cvrptw_b", "CVRPTW", "false", "0x0Cu", NO_B)]),
    ("p_cvrptw_c", 0, [("p_cvrptw_c", "CVRPTW", "false", "0x30u", NO_B)]),
    ("p_cvrptw_d", 0, [("p_cvrptw_d", "CVRPTW", "false", "0xC0u", NO_B)]),
    ("p_cvrptw_e", 0, [("p_cvrptw_e", "CVRPTW", "false", "0u", ALL_B)]),
    ("x_atsp16", 2, [("x_atsp16", "ATSP", "true", ALL_E, ALL_B)]),
    ("x_atsp32", 2, [("x_atsp32", "ATSP", "false", ALL_E, ALL_B)]),
    ("c_atsp", 1, [("c_atsp16", "ATSP", "true", ALL_E, NO_B),
                   ("c_atsp32", "ATSP", "false", ALL_E, NO_B)]),
    ("p_atsp", 0, [("p_atsp16", "ATSP", "true", ALL_E, ALL_B),
                   ("p_atsp32", "ATSP", "false", ALL_E, ALL_B)]),
    ("x_qap", 2, [("x_qap", "QAP", "false", ALL_E, ALL_B)]),
    ("c_qap", 1, [("c_qap", "QAP", "false", ALL_E, NO_B)]),
    ("p_qap", 0, [("p_qap", "QAP", "false", ALL_E, ALL_B)]),
    ("x_gap", 2, [("x_gap", "GAP", "false", ALL_E, ALL_B)]),
    ("c_gap", 1, [("c_gap", "GAP", "false", ALL_E, NO_B)]),
    ("p_gap", 0, [("p_gap", "GAP", "false", ALL_E, ALL_B)]),
    ("x_knapsack", 2, [("x_knapsack", "KNAPSACK", "false", ALL_E, ALL_B)]),
    ("c_knapsack", 1, [("c_knapsack", "KNAPSACK", "false", ALL_E, NO_B)]),
    ("p_knapsack", 0, [("p_knapsack", "KNAPSACK", "false", ALL_E, ALL_B)]),
    ("x_tsp16", 2, [("x_tsp16", "TSP", "true", ALL_E, ALL_B)]),
    ("x_tsp32", 2, [("x_tsp32", "TSP", "false", ALL_E, ALL_B)]),
    ("c_tsp", 1, [("c_tsp16", "TSP", "true", ALL_E, NO_B),
                  ("c_tsp32", "TSP", "false", ALL_E, NO_B)]),
    ("p_tsp32", 0, [("p_tsp32", "TSP", "false", ALL_E, ALL_B)]),
]
SOURCES = ["cgo_kernels.cu", "cgo_api.cu", "cgo_server.cu", "cgo_peaks.cu"]


def _unit_defines(xf, sets):
    # one value per definition (nvcc splits a definition's value at commas)
    d = ["-DCGO_UNIT=1", "-DCGO_UNIT_XF=%d" % xf]
    for i, (name, model, t16, em, bm) in enumerate(sets, 1):
        d += ["-DCGO_UNIT_S%d_%s=%s" % (i, k, v)
              for k, v in (("NAME", name), ("MODEL", model), ("T16", t16), ("EM", em), ("BM", bm))]
    return d
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the cgo library needs the CUDA toolkit")


def _flags(extra=()):
    return ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
            "-I" + INC, "-I" + CSRC, *extra]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INC, "cgo.h"),
                                                                 __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_info else []

    jobs = [("unit_%s.o" % name, "cgo_kernels.cu", _unit_defines(xf, sets))
            for name, xf, sets in UNITS]
    jobs += [(src.replace(".cu", ".o"), src, []) for src in SOURCES]

    def compile_one(job):
        name, src, defs = job
        obj = os.path.join(OUT_DIR, name)
        cmd = [cc, *_flags(extra), *defs, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s (%s):\n%s" % (src, name, r.stderr))
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max(1, min(len(jobs), 2 * (os.cpu_count() or 8)))) as ex:
        results = list(ex.map(compile_one, jobs))
    if verbose or ptxas_info:
        for _, err in results:
            print(err)
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results], "-cudart", "shared"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc link failed:\n%s" % r.stderr)
    os.replace(tmp, LIB)
    # every build compiles all units again: the objects are not kept
    for o, _ in results:
        try:
            os.remove(o)
        except OSError:
            pass
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose=True, ptxas_info="-v" in sys.argv))
