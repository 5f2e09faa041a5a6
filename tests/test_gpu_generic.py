"""The generic (interpreted) kernels against the oracle: every pipeline
program of Table 1's operations within pv.h's limits runs on the GPU.

The 300 random plans that pin the oracle against the nested-loop brute force
(tests/test_oracle_pins.py) run here through libpv: filters on int32, uint8
and int64 columns, zero to two probes into build tables with two payload
columns each (slots holding the build row, payloads gathered), group keys of
zero to three parts (fact columns and payloads), one to four SUM / COUNT /
MIN / MAX aggregates over products of up to three terms (constants over
payloads too), and projections of up to three values, on tables of 0 to 40
rows.  Each plan runs under several variants and build-table kinds, and the
benchmark workloads run on the generic kernels at ragged sizes, all bit-exact
(projections: multi pass in input order, single pass as a multiset)."""
import random

import numpy as np
import pytest

from oracle import oracle
from paper_1709_00700_gb300 import datagen, pv, workloads
from tests.gpu_util import assert_same, register
from tests.test_oracle_pins import _random_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = pv.Context(0)
    yield c
    c.close()


def _variants(plan, seed):
    if "project" in plan:
        return [dict(exec="multi", interp=1, items_per_thread=1 + seed % 2 * 3),
                dict(exec="single", interp=1, pred="predicated"),
                dict(exec="multi")]
    if plan.get("group_by"):
        ht = ("perfect", "linear", "cuckoo")[seed % 3]
        return [dict(agg="global", ht=ht, exec="multi" if ht == "cuckoo" else "single", interp=1),
                dict(agg="local", ht="linear", interp=1, pred="predicated"),
                dict(agg="local", ht="perfect", interp=1, block=128),
                dict(agg="global", ht="linear", exec="multi", interp=1)]
    return [dict(interp=1), dict(interp=1, pred="predicated", block=64)]


@pytest.mark.parametrize("chunk", range(10))
def test_random_plans_match_the_oracle(ctx, chunk):
    ran = 0
    for seed in range(30 * chunk, 30 * chunk + 30):
        plan, tables = _random_case(random.Random(seed))
        register(ctx, tables)
        w = oracle.run(plan, tables)["cols"]
        build = ("linear", "cuckoo", "perfect")[(seed // 3) % 3]
        for kw in _variants(plan, seed):
            try:
                got = ctx.query(plan, pv.variant(**kw), pv.ht_variant(build))
            except pv.PVError as e:
                # a CTA-local perfect array holds at most 192 KB (a documented limit)
                if e.status == -2 and kw.get("agg") == "local" and kw.get("ht") == "perfect":
                    continue
                raise
            ordered = "project" not in plan or kw.get("exec") == "multi"
            assert_same(got, w, ordered=ordered, ctxmsg=f"seed {seed} {build} {kw} {plan}")
            ran += 1
    assert ran >= 60


@pytest.mark.parametrize("n", [0, 1, 4097, 100_003])
def test_workloads_on_the_generic_kernels(ctx, n):
    """The benchmark workloads' plans forced onto the generic kernels."""
    cases = [({"t": datagen.table_filter_agg(n, seed=n + 11)}, workloads.filter_agg_plan()),
             ({"t": datagen.table_filter_agg(n, seed=n + 11)}, workloads.filter_project_plan()),
             ({"li": datagen.table_lowcard_groups(n, seed=n + 12)}, workloads.lowcard_plan()),
             ({"kv": datagen.table_keyval(n, 1000, "zipf", seed=n + 13)}, workloads.keyval_plan(val_lt=500_000)),
             ({"k3": datagen.table_keys3(n, seed=n + 14)}, workloads.keys3_plan())]
    if n > 0:
        cases += [(datagen.star_schema(n, seed=n + 15), workloads.star_plan({"d_a": 60, "d_b": 50, "d_c": 30})),
                  (datagen.star3_schema(n, seed=n + 16), workloads.star3_plan())]
    for tables, plan in cases:
        register(ctx, tables)
        w = oracle.run(plan, tables)["cols"]
        if "project" in plan:
            kws = [dict(exec="multi", interp=1), dict(exec="single", interp=1)]
        elif plan.get("group_by"):
            kws = [dict(agg="global", ht="perfect", interp=1), dict(agg="local", ht="linear", interp=1),
                   dict(agg="global", ht="cuckoo", exec="multi", interp=1, pred="predicated")]
        else:
            kws = [dict(interp=1), dict(interp=1, pred="predicated")]
        for kw in kws:
            got = ctx.query(plan, pv.variant(**kw), pv.ht_variant("perfect"))
            assert_same(got, w, ordered="project" not in plan or kw["exec"] == "multi", ctxmsg=f"n={n} {kw} {plan}")


def test_generic_only_parts(ctx):
    """Parts no compiled shape takes: an int64 probe key, a constant term over
    a payload, a two-part group key with a 64-bit part (coded in mixed radix)."""
    rng = np.random.default_rng(5)
    n = 50_001
    dim = {"key": rng.permutation(1000).astype(np.int32), "g": rng.integers(-20, 20, 1000).astype(np.int32),
           "h": rng.integers(0, 7, 1000).astype(np.uint8)}
    fact = {"fk": rng.integers(-10, 1010, n).astype(np.int64), "a": rng.integers(0, 5, n).astype(np.int32),
            "v": rng.integers(-1000, 1000, n).astype(np.int64)}
    tables = {"f": fact, "d": dim}
    register(ctx, tables)
    base = {"fact": "f", "builds": [{"table": "d", "key": "key", "filters": [["g", "ge", -15]], "payload": ["g", "h"]}],
            "probes": [{"build": 0, "fk": "fk"}]}
    plans = [dict(base, group_by=["v", "a"], aggs=[["sum", [["x_plus_c", ["payload", 0, 0], 7], ["x", "v"]]],
                                                    ["count"], ["min", [["c_minus_x", ["payload", 0, 1], 3]]]]),
             dict(base, group_by=[["payload", 0, 1]], aggs=[["max", [["x", "v"]]], ["count"]]),
             dict(base, aggs=[["sum", [["x", ["payload", 0, 1]], ["x", "a"]]], ["count"]]),
             dict(base, project=[["payload", 0, 1], "v", ["payload", 0, 0]])]
    for plan in plans:
        w = oracle.run(plan, tables)["cols"]
        for build in ("perfect", "linear"):
            for kw in (dict(agg="global", ht="linear"), dict(exec="multi")):
                got = ctx.query(plan, pv.variant(**kw), pv.ht_variant(build))
                assert_same(got, w, ordered="project" not in plan or kw.get("exec") == "multi",
                            ctxmsg=f"{build} {kw} {plan}")
