"""Host logic of the variant optimizer (no GPU): the paper's variant-space
counts and Algorithm 1 on synthetic cost functions."""
import itertools
import math

from paper_1709_00700_gb300 import autotune


def test_paper_variant_space_counts():
    # Section 9.2.2: 4 + 28 = 32 projection variants, 896 aggregation variants
    assert len(autotune.paper_space("project")) == 32
    assert sum(v["exec"] == "single" for v in autotune.paper_space("project")) == 4
    agg = autotune.paper_space("aggregate")
    assert len(agg) == 896
    assert sum(v["agg"] == "local" for v in agg) == 2 ** 4 * 7 * 7
    assert len({autotune.variant_key(v) for v in agg}) == 896


def _dims():
    return [("a", [0, 1, 2]), ("b", ["x", "y"]), ("c", [10, 20, 30, 40])]


def test_feature_wise_finds_separable_optimum_in_one_sweep():
    w = {"a": [3.0, 1.0, 2.0], "b": {"x": 5.0, "y": 0.5}, "c": {10: 4, 20: 3, 30: 0.1, 40: 2}}
    calls = []

    def cost(v):
        calls.append(v)
        return w["a"][v["a"]] + w["b"][v["b"]] + w["c"][v["c"]]

    v, t, n = autotune.feature_wise(cost, _dims(), q=5)
    best = min(autotune.enumerate_space(_dims()), key=cost)
    assert v == best and math.isclose(t, cost(best))
    # first sweep finds it (1 + 2 + 1 + 3 new configurations); the second sweep
    # tries the other values of a and b around it (2 + 1 new), changes nothing
    # and ends the loop
    assert n == 10


def test_feature_wise_stops_at_q_sweeps_and_keeps_ties_first():
    def cost(v):
        return 1.0  # everything ties: the first value of each dimension stays

    v, t, n = autotune.feature_wise(cost, _dims(), q=3)
    assert v == {"a": 0, "b": "x", "c": 10}


def test_feature_wise_revisits_a_dimension_after_a_later_one_changed():
    # b's best value depends on c, which is swept after b: the second sweep
    # must move b
    def cost(v):
        pen_b = 0.0 if (v["b"] == "y") == (v["c"] == 40) else 0.5
        return {0: 3.0, 1: 2.0, 2: 1.0}[v["a"]] + pen_b + (40 - v["c"]) / 10

    v, t, _ = autotune.feature_wise(cost, _dims(), q=4)
    assert v == {"a": 2, "b": "y", "c": 40}
    v1, _, _ = autotune.feature_wise(cost, _dims(), q=1)
    assert v1 == {"a": 2, "b": "x", "c": 40}  # one sweep is not enough


def test_feature_wise_stops_in_a_local_optimum():
    # a and b must change together to reach the optimum (2, y): one value at a
    # time never gets there, as coordinate descent does
    def cost(v):
        pen = 0.0 if (v["a"] == 2) == (v["b"] == "y") else 5.0
        return {0: 3.0, 1: 2.0, 2: 1.0}[v["a"]] + pen + v["c"] / 100

    v, t, _ = autotune.feature_wise(cost, _dims(), q=4)
    assert v == {"a": 1, "b": "x", "c": 10}
    best = min(autotune.enumerate_space(_dims()), key=cost)
    assert best == {"a": 2, "b": "y", "c": 10} and cost(best) < t


def test_feature_wise_failed_dimension_keeps_value():
    def cost(v):
        return math.inf if v["c"] != 10 else {0: 2.0, 1: 1.0, 2: 3.0}[v["a"]]

    v, t, _ = autotune.feature_wise(cost, _dims(), q=3)
    assert v["c"] == 10 and v["a"] == 1


def test_feature_ordering_restricts_and_orders():
    seen = []

    def cost(v):
        seen.append(tuple(sorted(v)))
        return v.get("c", 0)

    v, _, _ = autotune.feature_wise(cost, _dims(), q=1, order=["c", "a"])
    assert set(v) == {"c", "a"}


def test_exhaustive_and_db_resume(tmp_path):
    db = autotune.TimingDB(str(tmp_path / "t.jsonl"))
    n = [0]

    def cost(v):
        n[0] += 1
        return v["a"] * 10 + (v["b"] == "y") + v["c"] / 100

    best, ms, all_ms, _ = autotune.exhaustive(cost, _dims(), db, "q1")
    assert best == {"a": 0, "b": "x", "c": 10} and n[0] == 24 and len(all_ms) == 24
    db2 = autotune.TimingDB(str(tmp_path / "t.jsonl"))
    best2, ms2, _, _ = autotune.exhaustive(cost, _dims(), db2, "q1")
    assert best2 == best and n[0] == 24  # all timings came from the database


def test_algorithm_1_searches_the_probe_order_dimension():
    # a synthetic cost: block 512 is best, and only two probe orders have a compiled shape
    from paper_1709_00700_gb300 import autotune, workloads
    plan = workloads.star_plan()
    dims = [("block", [256, 512, 1024]), autotune.probe_order_dim(plan)]
    good = {(0, 1, 2, 3): 2.0, (1, 0, 3, 2): 1.5}

    def cost(v):
        return good.get(tuple(v["probe_order"]), float("inf")) * (1.0 if v["block"] == 512 else 1.3)

    v, c, n = autotune.feature_wise(cost, dims)
    assert v == {"block": 512, "probe_order": (1, 0, 3, 2)} and c == 1.5
    assert n <= 3 + 24 + 3 + 24
