"""Shared test helpers: parameter presets and exact state comparison."""
import numpy as np

import oracle as O

STATE_ARRAYS = ("cur", "best_sol", "cost", "best_cost")
STATE_SCALARS = ("P", "len", "g", "T", "w_op", "w_k", "stag", "elite_prev", "u_op", "v_op",
                 "u_k", "v_k")


def params_for(inst, **over):
    """The oracle's defaults for `inst`, with overrides; G defaults to 0."""
    p = O.default_params(inst)
    p["G"] = 0
    ops = over.pop("ops", None)
    if ops is not None:
        w = [0] * O.NOPS
        for o in ops:
            w[o] = 65536 // len(ops)
        p["w_op"] = w
        p["op_mask"] = sum(1 << o for o in ops)
    p.update(over)
    return p


def assert_same_state(g, o, where=""):
    """Bit-exact equality of a GPU state and an oracle state."""
    for k in STATE_SCALARS:
        assert g[k] == o[k], "%s: %s differs: gpu %r oracle %r" % (where, k, g[k], o[k])
    for k in STATE_ARRAYS:
        a, b = np.asarray(g[k]), np.asarray(o[k])
        assert a.shape == b.shape, "%s: %s shape" % (where, k)
        if not (a == b).all():
            bad = np.argwhere(a != b)[:5].tolist()
            raise AssertionError("%s: %s differs at %s" % (where, k, bad))


def oracle_run(inst, params, seed, G, threads=0):
    return O.solve(inst, params, seed, G, threads=threads)


def assert_same_counts(prob, o, where=""):
    """Operator and k-level counts over the whole solve (cgo_op_counts) equal
    the oracle's, and the k-level counts add up to P x C x G."""
    g = prob.op_counts()
    for k in ("u_op", "v_op", "u_k", "v_k"):
        assert g[k] == o["op_counts"][k], "%s: %s gpu %r oracle %r" % (where, k, g[k], o["op_counts"][k])
