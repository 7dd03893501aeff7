"""Oracle pins for islands and migration (Sec. 3.4.3).

Hand-built states with ties check the choice of sources and targets of each
strategy; a run with migration must equal the run without it followed by one
migration step at the end of the migrating generation (after the AOS update,
before elite injection)."""
import numpy as np
import pytest

import instances as I
import oracle as O
from helpers import params_for


def crafted(P=8, length=3):
    cur = np.array([np.roll(np.arange(length), q) for q in range(P)], np.int32)
    best = cur[::-1].copy()
    cost = np.array([50, 70, 70, 10, 90, 20, 90, 30], np.int64)[:P]
    best_cost = np.array([40, 5, 60, 10, 80, 5, 15, 30], np.int64)[:P]
    return dict(cur=cur, best_sol=best, cost=cost, best_cost=best_cost, g=10)


def params(strategy, islands=2, n=1):
    inst = I.tsp_uniform(3, 1)
    p = O.default_params(inst)
    p.update(islands=islands, migrate_period=10, migrate_strategy=strategy, migrate_n=n)
    return p


def expect_replace(st, target, source):
    st["cur"][target] = st["_bsol"][source]
    st["cost"][target] = st["_bcost"][source]
    if st["_bcost"][source] < st["best_cost"][target]:
        st["best_cost"][target] = st["_bcost"][source]
        st["best_sol"][target] = st["_bsol"][source]


def snapshot(st):
    e = {k: np.array(v, copy=True) if isinstance(v, np.ndarray) else v for k, v in st.items()}
    e["_bsol"], e["_bcost"] = st["best_sol"].copy(), st["best_cost"].copy()
    return e


def test_ring_two_islands_with_ties():
    st = crafted()
    got = O.migrate(params(0), st)
    e = snapshot(st)
    # island 0 = members 0-3: best (lowest best cost, lowest index) is 1 (5);
    # worst (highest cost, lowest index) is 1 or 2 at 70 -> 1
    # island 1 = members 4-7: best is 5 (5), worst is 4 or 6 at 90 -> 4
    expect_replace(e, 4, 1)      # island 0's best to island 1's worst
    expect_replace(e, 1, 5)      # island 1's best to island 0's worst
    for k in ("cur", "best_sol", "cost", "best_cost"):
        assert (got[k] == e[k]).all(), k


def test_top_n_every_island():
    st = crafted()
    got = O.migrate(params(1, islands=2, n=2), st)
    e = snapshot(st)
    # population's two best by (best cost, index): 1 (5), 5 (5)
    # island 0 worst two: 1 (70), 2 (70); island 1: 4 (90), 6 (90)
    for tgt, src in ((1, 1), (2, 5), (4, 1), (6, 5)):
        expect_replace(e, tgt, src)
    for k in ("cur", "best_sol", "cost", "best_cost"):
        assert (got[k] == e[k]).all(), k


@pytest.mark.parametrize("g,kind", [(10, "ring"), (20, "top")])
def test_hybrid_alternates(g, kind):
    st = dict(crafted(), g=g)
    got = O.migrate(params(2, islands=2, n=1), st)
    want = O.migrate(params(0 if kind == "ring" else 1, islands=2, n=1), st)
    for k in ("cur", "best_sol", "cost", "best_cost"):
        assert (got[k] == want[k]).all(), k


def test_invalid_island_parameters():
    st = crafted()
    for bad in (dict(islands=3), dict(migrate_strategy=1, migrate_n=5), dict(migrate_strategy=4)):
        p = params(0)
        p.update(bad)
        with pytest.raises(ValueError):
            O.migrate(p, st)


@pytest.mark.parametrize("strategy,n", [(0, 1), (1, 2), (2, 1)])
def test_run_with_migration_is_run_then_migrate(strategy, n):
    inst = I.tsp_uniform(20, 3)
    base = params_for(inst, P=12, C=32, U=5, elite_period=0)
    mig = dict(base, islands=3, migrate_period=5, migrate_strategy=strategy, migrate_n=n)
    plain = O.solve(inst, base, 7, 5)
    with_m = O.solve(inst, mig, 7, 5)
    want = O.migrate(mig, plain)
    for k in ("cur", "best_sol", "cost", "best_cost"):
        assert (with_m[k] == want[k]).all(), k
    assert with_m["w_op"] == plain["w_op"] and with_m["T"] == plain["T"]
