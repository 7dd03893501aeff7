"""Pin of the oracle's search generation against generations worked by hand
(tests/golden/generation.json): Alg. "evolve" (Sec. 3.2.3) for every member,
the AOS statistics and Eq. "ema" (Sec. 4.2.2), the stagnation rule
(Sec. 4.2.3), cooling and the plain random start.

The fixture lists, for each candidate, its Philox words, the roulette that
gives k (from word r3 of step 0) and each operator (word r0 of its step), the
decoded positions, the array after every step, the full cost edge by edge
and the delta; then the argmin (lowest index among the minimum deltas), the
acceptance draw and the state after the generation.  The oracle's state must
equal it exactly.  The second group of tests checks that the fixture tells
apart the plausible misreadings of the step: counting only the winner's
operators, ties going to the highest index, k drawn from word r0.
"""
import json
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "generation.json")
CASES = json.load(open(GOLDEN))["cases"]
TSP_CASE, GAP_CASE = CASES


def _instance(case):
    d = dict(case["instance"])
    for f in ("mat0", "mat1", "vec0"):
        if f in d:
            d[f] = np.array(d[f], np.int32)
    return d


def _params(case):
    inst = _instance(case)
    p = O.default_params(inst)
    p.update(case["params"])
    return inst, p


def _state(case, G):
    inst, p = _params(case)
    if G == 0:
        return O.Solver(inst, p, case["seed"]).state()
    return O.solve(inst, p, case["seed"], G)


# ------------------------------------------------------------ oracle vs hand
def test_tsp_start_population():
    st = _state(TSP_CASE, 0)
    for m in TSP_CASE["init"]:
        assert st["cur"][m["member"]].tolist() == m["start"]
        assert int(st["cost"][m["member"]]) == m["cost"]["total"]
    assert st["stag"] == 0
    assert st["elite_prev"] == min(m["cost"]["total"] for m in TSP_CASE["init"])


@pytest.mark.parametrize("G", [1, 2])
def test_tsp_state_after_generation(G):
    st = _state(TSP_CASE, G)
    want = TSP_CASE["after_generation_%d" % G]
    assert st["cur"].tolist() == want["cur"]
    assert st["cost"].tolist() == want["cost"]
    assert st["best_cost"].tolist() == want["best_cost"]
    assert st["best_sol"].tolist() == want["best_sol"]
    for k in ("u_op", "v_op", "u_k", "v_k"):
        assert st[k] == want[k], k
    assert st["T"] == want["T"]
    if G == 2:
        assert st["w_op"] == want["w_op"]
        assert st["w_k"] == want["w_k"]
        assert st["stag"] == want["stag"]
        assert st["elite_prev"] == want["elite_prev"]


def test_gap_generation():
    st0 = _state(GAP_CASE, 0)
    assert st0["cur"][0].tolist() == GAP_CASE["init"]["start"]
    assert int(st0["cost"][0]) == GAP_CASE["init"]["cost"]["total"]
    st = _state(GAP_CASE, 1)
    want = GAP_CASE["after_generation_1"]
    assert st["cur"].tolist() == want["cur"]
    assert st["cost"].tolist() == want["cost"]
    for k in ("u_op", "v_op", "u_k", "v_k"):
        assert st[k] == want[k], k


# -------------------------------------------- the fixture is self-consistent
@pytest.mark.parametrize("case", CASES, ids=["tsp", "gap"])
def test_fixture_arithmetic(case):
    for gen in case["generations"]:
        for cd in gen["candidates"]:
            assert cd["delta"] == cd["cost"]["total"] - gen["start_cost"]
            assert len(cd["steps"]) == cd["k"]["value"]
            assert cd["result"] == cd["steps"][-1]["after"]
            for roul in [cd["k"]] + [s["op"] for s in cd["steps"]]:
                r = roul["r"]
                assert roul["thresholds"][roul["pick"]] > r
                assert roul["pick"] == 0 or roul["thresholds"][roul["pick"] - 1] <= r
        deltas = [cd["delta"] for cd in gen["candidates"]]
        assert gen["min_delta"] == min(deltas)
        assert gen["tied"] == [c for c, d in enumerate(deltas) if d == min(deltas)]
        assert gen["winner"] == gen["tied"][0]


def _counts(gens, only_winner=False):
    u, v, uk, vk = [0] * O.NOPS, [0] * O.NOPS, [0] * 3, [0] * 3
    for gen in gens:
        for cd in gen["candidates"]:
            if only_winner and cd["c"] != gen["winner"]:
                continue
            imp = int(cd["delta"] < 0)
            for s in cd["steps"]:
                u[s["op"]["pick"]] += 1
                v[s["op"]["pick"]] += imp
            uk[cd["k"]["value"] - 1] += 1
            vk[cd["k"]["value"] - 1] += imp
    return u, v, uk, vk


# ------------------------------------- the fixture catches plausible mistakes
def test_counts_cover_every_candidate_not_only_the_winner():
    g1 = TSP_CASE["generations"][:2]
    want = TSP_CASE["after_generation_1"]
    assert list(_counts(g1)) == [want["u_op"], want["v_op"], want["u_k"], want["v_k"]]
    assert list(_counts(g1, only_winner=True)) != [want["u_op"], want["v_op"], want["u_k"], want["v_k"]]


def test_a_tie_decides_the_next_solution():
    # an accepted generation whose tied candidates lead to different arrays:
    # ties going to the highest index would leave another solution
    hits = [gen for gen in TSP_CASE["generations"]
            if gen["acceptance"]["accepted"] and len(gen["tied"]) > 1
            and gen["candidates"][gen["tied"][0]]["result"] != gen["candidates"][gen["tied"][-1]]["result"]]
    assert hits
    gen = hits[0]
    want = TSP_CASE["after_generation_%d" % (gen["generation"] + 1)]["cur"][gen["member"]]
    assert want == gen["candidates"][gen["tied"][0]]["result"]
    assert want != gen["candidates"][gen["tied"][-1]]["result"]


def test_k_from_r3_is_distinguishable_from_r0():
    for case in CASES:
        ks = [(cd["k"]["value"], cd["k_if_drawn_from_r0"])
              for gen in case["generations"][:2] for cd in gen["candidates"]]
        assert any(a != b for a, b in ks)
        # the k-level counts after generation 1 would differ
        u_k = [0, 0, 0]
        for _, b in ks:
            u_k[b - 1] += 1
        assert u_k != case["after_generation_1"]["u_k"]


def test_acceptance_cases_far_from_the_boundary():
    seen = set()
    for gen in TSP_CASE["generations"]:
        acc = gen["acceptance"]
        if gen["min_delta"] > 0:
            assert abs(gen["min_delta"] - acc["T_times_E"]) > 0.5
            seen.add(acc["accepted"])
    assert seen == {True, False}  # one worsening move taken, one refused
