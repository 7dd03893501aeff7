"""Failure paths made on the host (nothing here faults, traps or hangs the
GPU): device allocations that fail (an injected out-of-memory on the n-th
allocation), a bounded submit queue, and cancelled requests.  After each
failure the library keeps working and later results equal the plain solve."""
import time

import pytest

import instances as I
from helpers import assert_same_state, oracle_run, params_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cgo():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_19163_gb300 import cgo as C
    C.lib()
    yield C
    C.lib().cgo_debug_inject(None, 4, 0)


def inject_alloc_failure(C, nth):
    C.check(C.lib().cgo_debug_inject(None, 4, nth), "inject")


def test_problem_creation_survives_failed_allocations(cgo):
    inst = I.cvrptw(20, 400, vehicles=4, capacity=80)
    for nth in (1, 2, 3):
        inject_alloc_failure(cgo, nth)
        with pytest.raises(cgo.CgoError) as e:
            cgo.Problem(inst)
        assert e.value.status == cgo.ERR_NOMEM
    inject_alloc_failure(cgo, 0)
    prob = cgo.Problem(inst)
    p = params_for(inst, P=6, C=64, G=15)
    prob.solve(p, 3)
    assert_same_state(prob.state(), oracle_run(inst, p, 3, 15), "after failed creations")


def test_solve_survives_a_failed_state_allocation(cgo):
    inst = I.tsp_uniform(40, 401)
    prob = cgo.Problem(inst)
    p = params_for(inst, P=8, C=64, G=20)
    for nth in (1, 3, 6):
        inject_alloc_failure(cgo, nth)
        with pytest.raises(cgo.CgoError) as e:
            prob.solve(p, 5)
        assert e.value.status == cgo.ERR_NOMEM
        with pytest.raises(cgo.CgoError):        # no state was left behind
            prob.best()
    inject_alloc_failure(cgo, 0)
    prob.solve(p, 5)
    assert_same_state(prob.state(), oracle_run(inst, p, 5, 20), "after failed allocations")


def long_request(cgo):
    """A request that stays resident for many slices."""
    inst = dict(I.tsp_uniform(300, 402), tag=77)
    prob = cgo.Problem(inst)
    return prob, params_for(inst, P=32, C=128, G=3_000_000)


def wait_until(pred, limit=30.0):
    t0 = time.time()
    while not pred():
        assert time.time() - t0 < limit, "condition not reached"
        time.sleep(0.005)


def test_bounded_queue_and_cancellation(cgo):
    srv = cgo.Server(max_slots=1, slice_generations=500, max_queued=2)
    try:
        big, bp = long_request(cgo)
        t_big = srv.submit(big, bp, 1)
        wait_until(lambda: srv.stats()["active"] == 1 and srv.stats()["queued"] == 0)
        small = [(dict(I.knapsack(60 + 10 * i, 403 + i), tag=i), None) for i in range(3)]
        probs = [cgo.Problem(x) for x, _ in small]
        params = [params_for(x, P=6, C=64, G=21) for x, _ in small]
        t0 = srv.submit(probs[0], params[0], 11)
        t1 = srv.submit(probs[1], params[1], 12)
        with pytest.raises(cgo.CgoError) as e:       # two already wait for admission
            srv.submit(probs[2], params[2], 13)
        assert e.value.status == cgo.ERR_BUSY
        # a queued request cancelled: it ends at once and its handle is free
        srv.cancel(t1)
        with pytest.raises(cgo.CgoError) as e:
            srv.wait(t1, -1)
        assert e.value.status == cgo.ERR_CANCELLED
        probs[1].solve(params[1], 12)                # the handle works again
        assert_same_state(probs[1].state(), oracle_run(small[1][0], params[1], 12, 21), "after cancel")
        # the queue has room again
        t2 = srv.submit(probs[2], params[2], 13)
        # the resident request cancelled: retired at the next slice boundary
        srv.cancel(t_big)
        with pytest.raises(cgo.CgoError) as e:
            srv.wait(t_big, -1)
        assert e.value.status == cgo.ERR_CANCELLED
        with pytest.raises(cgo.CgoError):
            big.best()                               # no search state kept
        with pytest.raises(cgo.CgoError) as e:
            srv.cancel(t_big)                        # forgotten after the wait
        assert e.value.status == cgo.ERR_INVALID
        # the others run to the end and equal the oracle
        for t, pr, q, (x, _), seed in ((t0, probs[0], params[0], small[0], 11),
                                       (t2, probs[2], params[2], small[2], 13)):
            srv.wait(t, -1)
            assert_same_state(pr.state(), oracle_run(x, q, seed, 21), "served after cancel")
    finally:
        srv.close()


def test_admission_allocation_failure_fails_one_request(cgo):
    srv = cgo.Server(max_slots=4, slice_generations=500)
    try:
        inst = dict(I.gap(40, 410, m=5), tag=3)
        prob = cgo.Problem(inst)
        p = params_for(inst, P=8, C=64, G=25)
        inject_alloc_failure(cgo, 1)                 # the request's state at admission
        t = srv.submit(prob, p, 9)
        with pytest.raises(cgo.CgoError) as e:
            srv.wait(t, -1)
        assert e.value.status == cgo.ERR_NOMEM
        inject_alloc_failure(cgo, 0)
        t = srv.submit(prob, p, 9)                   # the server carries on
        srv.wait(t, -1)
        assert_same_state(prob.state(), oracle_run(inst, p, 9, 25), "after a failed admission")
    finally:
        inject_alloc_failure(cgo, 0)
        srv.close()


def test_earlier_server_config_size(cgo):
    import ctypes
    cfg = cgo.cgo_server_cfg(cgo.cgo_server_cfg.max_queued.offset, 2, 1 << 30, 0, 100, 0, 0)
    h = ctypes.c_void_p()
    cgo.check(cgo.lib().cgo_server_create(ctypes.byref(cfg), ctypes.byref(h)), "create")
    cgo.lib().cgo_server_destroy(h)
    cfg.struct_size = 7
    assert cgo.lib().cgo_server_create(ctypes.byref(cfg), ctypes.byref(h)) == cgo.ERR_INVALID
