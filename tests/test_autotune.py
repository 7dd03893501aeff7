"""Host logic of the autotuner (no GPU): trial shapes and the serving-population rule."""
from paper_2603_19163_gb300.autotune import Autotuner, population_for_load, slices_by_class


def test_population_rule_keeps_everything_at_the_top_when_it_fits():
    P, load = population_for_load({"a": 1e10, "b": 1e10}, {"a": 0.5, "b": 0.5}, 10.0, 1000, 128)
    assert P == {"a": 32, "b": 32} and load < 0.8


def test_population_rule_steps_down_the_heaviest_class_first():
    rate = {"fast": 2e10, "slow": 2e8}
    share = {"fast": 0.85, "slow": 0.15}
    P, load = population_for_load(rate, share, 200.0, 20000, 128)
    # the slow class dominates the load, so it reaches the bottom of the
    # ladder before the fast one moves
    assert P["slow"] == 8
    assert P["fast"] in (32, 16, 8)
    loads = {c: 200 * share[c] * P[c] * 128 * 20000 / rate[c] for c in rate}
    assert abs(sum(loads.values()) - load) < 1e-9


def test_population_rule_reports_overload_at_the_bottom():
    P, load = population_for_load({"x": 1e6}, {"x": 1.0}, 1000.0, 20000, 128)
    assert P == {"x": 8} and load > 0.8


def test_solve_shapes_cover_deep_generations_only_where_they_run():
    t = Autotuner()
    shapes = t.solve_shapes(dict(C=128))
    assert (12, 4, 1, 3) in shapes and (16, 4, 1, 4) in shapes and (8, 4, 1, 2) in shapes
    assert all(s[3] <= 2 or (s[1] == 4 and s[0] == 4 * s[3]) for s in shapes)
    assert all(s[3] <= 2 for s in t.solve_shapes(dict(C=128, cross_q16=100)))
    assert all(s[3] == 1 for s in t.solve_shapes(dict(C=300)))


def test_batch_populations_fit_the_l2_working_set():
    import instances as I
    from paper_2603_19163_gb300.autotune import batch_populations, instance_data_bytes, state_bytes
    mix = I.batch_mix(64, 0)
    big, total = batch_populations(mix, 1 << 40)
    assert set(big.values()) == {64} and total > 0            # everything fits: the top
    small, total = batch_populations(mix, 1 << 20)
    assert set(small.values()) == {8}                          # nothing fits: the bottom
    data = sum(instance_data_bytes(x) for x in mix)
    mid, total = batch_populations(mix, data + 3 * (total - data))
    assert total <= data + 3 * (total - data)
    # the class with the most state is cut first: knapsack (n up to 2000) before GAP
    assert mid[2] <= mid[3]
    # the working set adds every instance's state at its class's population
    lens = [(int(x["model"]), int(x["n"])) for x in mix]
    assert total == data + sum(state_bytes(n, mid[m]) for m, n in lens)


def test_slice_rule_keeps_the_slowest_class_at_the_base_slice():
    # per request and generation: a 1e9 / (8 x 128), b 1e8 / (8 x 128), c 4e9 / (32 x 128)
    rate = {"a": 1e9, "b": 1e8, "c": 4e9}
    pops = {"a": 8, "b": 8, "c": 32}
    assert slices_by_class(rate, pops, 128, 20000, 2000, 50000) == {"a": 20000, "b": 2000, "c": 20000}
    assert slices_by_class(rate, pops, 128, 20000, 2000, 6000) == {"a": 6000, "b": 2000, "c": 6000}
    # off: every class at the base slice
    assert slices_by_class(rate, pops, 128, 20000, 2000, 0) == {"a": 2000, "b": 2000, "c": 2000}


def test_slice_rule_weighs_the_population():
    # equal batch rates, but b's requests carry four times the members
    rate = {"a": 1e9, "b": 1e9}
    assert slices_by_class(rate, {"a": 8, "b": 32}, 128, 20000, 2000, 20000) == {"a": 20000, "b": 2000}
