"""A small variant-selection suite end to end on the GPU: random queries of
the three families, exhaustive timing, Algorithm 1 per family, and the cost
model trained with its own kernels and assessed on held-out queries."""
import math

import numpy as np
import pytest

from oracle import oracle
from paper_1709_00700_gb300 import autotune, datagen, pv, suite, workloads

pytestmark = pytest.mark.gpu


def test_small_suite_runs_and_picks_from_the_grid():
    ctx = pv.Context(0)
    s = suite.run(ctx, n_queries=24, max_rows=2_000_000, min_rows=200_000, reps=2,
                  candidates=((300, 2, 2e-3), (200, 1, 3e-3)), log=None)
    ctx.close()
    assert s["held_out"] == 5 and s["train"] == 19
    assert len(s["validation"]) == 2 and s["chosen"]["epochs"] in (300, 200)
    assert s["loss_history"][-1] < s["loss_history"][0]
    for p in s["per_query"]:
        grid = [autotune.variant_key(v) for v in suite.GRIDS[p["family"]]]
        assert autotune.variant_key(p["pick"]) in grid
        assert p["best_ms"] <= p["pick_ms"] and p["best_ms"] <= p["config_ms"]
        assert math.isfinite(p["pick_ms"])
    assert 0.0 <= s["mlp_within_10pct"] <= 1.0


def test_confirm_retimes_the_held_out_candidates():
    ctx = pv.Context(0)
    data = suite.SuiteData(ctx, 2_000_000)
    ex = suite.explore(ctx, 12, 2_000_000, 200_000, reps=2, log=None, data=data)
    s = suite.assess(ctx, ex, candidates=((200, 1, 3e-3),))
    c = suite.confirm(data, ex, s, reps=3, log=None)
    ctx.close()
    assert c["reps"] == 3 and len(c["per_query"]) == len(s["per_query"])
    for r in c["per_query"]:
        assert r["pick_ratio"] >= 1.0 and r["config_ratio"] >= 1.0 and math.isfinite(r["pick_ratio"])
    assert 0.0 <= c["mlp_within_10pct"] <= 1.0


def test_online_tuner_learns_from_its_own_runs():
    """The run-time tuner learns from the queries it runs: after the stream,
    its network predicts the times it observed (the chosen variants and, with
    shadow runs, the runner-ups) better than the seed network left as it was."""
    ctx = pv.Context(0)
    data = suite.SuiteData(ctx, 2_000_000)
    ex = suite.explore(ctx, 40, 2_000_000, 200_000, reps=2, log=None, data=data)
    for top in (1, 3):
        r = suite.online_experiment(ctx, ex, n_seed=10, tail=10, seed_epochs=300, ensemble=1, every=5, steps=200,
                                    explore=0.0, observe_top=top)
        assert r["stream"] == 30 and r["updates"] == 6
        assert r["observations"] == 30 * top and r["shadow_runs_per_query"] == top - 1
        assert r["online_fit_mse"] < r["static_fit_mse"], r
        assert 0.0 <= r["online_within_10pct"] <= 1.0 and r["online_geomean"] >= 1.0
    ctx.close()


def test_graph_experiment_results_equal_eager_and_oracle():
    """The CUDA-graph experiment: 64 small queries replayed as one graph keep
    their eager results (asserted inside), and the star join's four builds
    plus its probe replayed as one graph equal the eager run (asserted
    inside) and the oracle on the same tables."""
    rows = 200_000
    ctx = pv.Context(0)
    r = suite.graph_experiment(ctx, n_queries=8, rows=rows, reps=3, star_results=True)
    ctx.close()
    want = oracle.run(workloads.star_plan(), datagen.star_schema(rows))["cols"]
    got = r["star_cols"]
    assert len(got) == len(want) and len(want[0]) > 10
    for g, w in zip(got, want):
        assert np.array_equal(g, w)


def test_network_gains_over_algorithm1_on_held_out_queries():
    """What the trained network gains over the method without it: on a seeded
    suite of 150 random queries (120 to train on, 30 held out), the per-query
    picks of the network (trained with libpv's kernels) are within 10% of the
    exhaustive best at least as often as Algorithm 1's per-family
    configuration (Section 8.3), and lose less in geometric mean."""
    ctx = pv.Context(0)
    s = suite.run(ctx, n_queries=150, max_rows=8_000_000, min_rows=500_000, reps=2,
                  candidates=((3000, 3, 2e-3),), log=None)
    ctx.close()
    assert s["held_out"] == 30 and s["train"] == 120
    assert s["mlp_within_10pct"] >= s["alg1_within_10pct"], s
    assert s["mlp_geomean_slowdown"] < s["alg1_geomean_slowdown"], s
