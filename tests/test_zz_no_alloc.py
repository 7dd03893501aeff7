"""The allocation-free TSP entry point (cgo_solve_static).

Some callers cannot allocate device memory (their code runs where
cudaMalloc is not allowed, or their GPU memory budget is fixed once the
process has started).  cgo_solve_static serves them: the caller passes
device inputs and outputs, and the library works in a fixed device array of
its own instead of allocating.  This file checks, through the C ABI, that
two calls in a row give the same elite solution and cost as cgo_solve +
cgo_best (exactly: the search is integer), and that a request larger than
the array is refused before any GPU work.  It is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import instances as I
from helpers import params_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_19163_gb300 import cgo
    return torch, cgo


def _desc(cgo, n, d_ptr, tag):
    d = cgo.cgo_problem_desc()
    d.struct_size = ctypes.sizeof(cgo.cgo_problem_desc)
    d.encoding = cgo.ENC_PERM
    d.model = cgo.TSP
    d.n = n
    d.mat0 = d_ptr
    d.pointers_on_device = 1
    d.instance_tag = tag
    return d


def _static_solve(torch, cgo, inst, params, seed):
    n = inst["n"]
    D = torch.from_numpy(np.ascontiguousarray(inst["mat0"])).cuda()
    out_sol = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    out_cost = torch.zeros(1, dtype=torch.int64, device="cuda")
    d = _desc(cgo, n, D.data_ptr(), inst.get("tag", 0))
    q = cgo.params_struct(params)
    rc = cgo.lib().cgo_solve_static(ctypes.byref(d), ctypes.byref(q), seed, out_sol.data_ptr(),
                                    out_cost.data_ptr(), None)
    return rc, out_sol.cpu().numpy(), int(out_cost.cpu().item())


def test_static_solve_matches_cgo_solve_twice(env):
    torch, cgo = env
    cases = [
        (I.tsp_clustered(442, 0), dict(P=128, C=128, G=300, op_mask=0b1110), 1),
        (I.tsp_uniform(60, 5), dict(P=16, C=64, G=500), 7),
    ]
    for inst, over, seed in cases:
        p = params_for(inst, **over)
        prob = cgo.Problem(inst)
        prob.solve(p, seed)
        want_sol, want_cost = prob.best()
        rc, sol, cost = _static_solve(torch, cgo, inst, p, seed)
        assert rc == cgo.OK, cgo.lib().cgo_last_error()
        assert cost == want_cost
        assert np.array_equal(sol, want_sol)


def test_static_solve_rejects_the_pool_start(env):
    torch, cgo = env
    inst = I.tsp_uniform(30, 3)
    for over in (dict(init_oversample=2), dict(init_heuristic=1), dict(cross_q16=30000)):
        p = params_for(inst, P=8, C=32, G=5, **over)
        rc, _, _ = _static_solve(torch, cgo, inst, p, 1)
        assert rc == cgo.ERR_UNSUPPORTED


def test_static_solve_rejects_oversized_requests(env):
    torch, cgo = env
    inst = I.tsp_uniform(2100, 9)                # 2n^2 alone exceeds the array
    p = params_for(inst, P=8, C=32, G=1)
    rc, _, _ = _static_solve(torch, cgo, inst, p, 1)
    assert rc == cgo.ERR_INVALID
    assert b"scratch" in cgo.lib().cgo_last_error()


def test_static_solve_refuses_an_asymmetric_matrix(env):
    # the fixed array holds the triangle of a symmetric matrix; cgo_solve
    # takes the asymmetric case
    torch, cgo = env
    inst = I.tsp_asym(30, 4)
    p = params_for(inst, P=8, C=32, G=5)
    rc, _, _ = _static_solve(torch, cgo, inst, p, 1)
    assert rc == cgo.ERR_UNSUPPORTED
    assert b"symmetric" in cgo.lib().cgo_last_error()
