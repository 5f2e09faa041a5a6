"""A small variant-selection suite end to end on the GPU: random queries of
the three families, exhaustive timing, Algorithm 1 per family, and the cost
model trained with its own kernels and assessed on held-out queries."""
import math

import pytest

from paper_1709_00700_gb300 import autotune, pv, suite

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
    ctx = pv.Context(0)
    data = suite.SuiteData(ctx, 2_000_000)
    ex = suite.explore(ctx, 30, 2_000_000, 200_000, reps=2, log=None, data=data)
    r = suite.online_experiment(ctx, ex, n_seed=10, tail=10, seed_epochs=200, ensemble=1, every=4, steps=50)
    ctx.close()
    assert r["stream"] == 20 and r["updates"] == 5
    assert 0.0 <= r["online_within_10pct"] <= 1.0 and r["online_geomean"] >= 1.0 and r["static_geomean"] >= 1.0
