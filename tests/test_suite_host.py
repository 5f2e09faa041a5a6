"""Host logic of the variant-selection suite (no GPU)."""
import math

from paper_1709_00700_gb300 import autotune, suite


def test_query_generator_hits_its_targets():
    qs = suite.make_queries(300, seed=5)
    fams = [q["family"] for q in qs]
    assert fams.count("filter") == fams.count("grouped") == fams.count("star") == 100
    assert all(1_000_000 <= q["rows"] <= 300_000_000 for q in qs)
    for q in qs:
        if q["family"] == "filter":
            got = q["A"] / 100 * (q["B1"] - q["B0"] + 1) / 100
            assert abs(math.log(got / q["sel_target"])) < 0.7


def test_grids_have_uniform_keys_and_algorithm1_runs_on_lookups():
    for g, grid in suite.GRIDS.items():
        keys = set(grid[0])
        assert all(set(v) == keys for v in grid)
        assert len({autotune.variant_key(v) for v in grid}) == len(grid)
    grid = suite.GRIDS["filter_aggregate"]
    # a synthetic timing table whose best configuration is known
    train = [{"id": i} for i in range(3)]
    timings = {i: {autotune.variant_key(v): 1.0 + (v["pred"] == "predicated") + (v["access"] == "chunked")
                   + 0.1 * (v["items_per_thread"] == 1) + 0.01 * (v["block"] == 256) + 0.001 * v["prefetch"]
                   for v in grid} for i in range(3)}
    v = suite.algorithm1_config(train, timings, grid)
    assert v == {"pred": "branch", "access": "grid", "items_per_thread": 4, "block": 512, "prefetch": 0,
                 "first_items": 1}
