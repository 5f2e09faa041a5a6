"""Pins of the CPU oracle against things other than itself.

* closed forms on lattice tables (computed with Python integers from the
  lattice definition, never by running a pipeline);
* hand-worked fixtures under tests/golden/ (worked example of Section 7.3 and
  the pipeline programs of Table 2);
* a pure-Python nested-loop brute force (CROSS_JOIN + FILTER semantics,
  linear-scan grouping) on many tiny random inputs;
* invariants that hold at any size (group sums add up to the ungrouped sum,
  counts equal the number of predicate-true rows, threads do not change the
  result);
* error and edge cases (duplicate build key, empty input, overflow flag).
"""
import glob
import json
import os
import random

import numpy as np
import pytest

from oracle import oracle
from paper_1709_00700_gb300 import datagen, workloads
from tests import bruteforce

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _tables_from_json(spec):
    return {t: {c: np.array(v["values"], dtype=v["dtype"]) for c, v in cols.items()}
            for t, cols in spec.items()}


def _as_lists(res):
    return [list(map(int, c)) for c in res["cols"]]


@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(GOLDEN, "*.json"))))
def test_golden_fixture(path):
    with open(path) as f:
        g = json.load(f)
    if "plan" not in g:
        pytest.skip("not a plan fixture")
    res = oracle.run(g["plan"], _tables_from_json(g["tables"]))
    assert res["kind"] == g["expected"]["kind"]
    assert _as_lists(res) == g["expected"]["cols"]


@pytest.mark.parametrize("m", [1, 3])
def test_lattice_filter_aggregate_closed_form(m):
    # a = i mod 100, b = (i div 100) mod 100, price = 100 + i, i < 10^4 m.
    # WHERE a < 10 AND 20 <= b <= 40: in each block q of 10^4 rows the rows
    # i = 10^4 q + 100 b + a with a in [0,10), b in [20,40] qualify.
    t = {"t": datagen.table_lattice(m)}
    res = oracle.run(workloads.filter_agg_plan(), t)
    count = 210 * m
    sum_q = m * (m - 1) // 2
    total = (100 * count + 10_000 * sum_q * 210 + 100 * sum(range(20, 41)) * 10 * m
             + sum(range(10)) * 21 * m)
    assert _as_lists(res) == [[total], [count]]
    assert not res["overflow"]


def test_lattice_projection_is_input_order():
    t = {"t": datagen.table_lattice(1)}
    res = oracle.run(workloads.filter_project_plan(), t)
    rows = [100 * b + a for b in range(20, 41) for a in range(10)]
    assert _as_lists(res) == [[r % 100 for r in rows], [100 + r for r in rows]]


@pytest.mark.parametrize("g,n", [(7, 1000), (10, 10_000), (1, 5), (64, 63)])
def test_grouped_lattice_closed_form(g, n):
    # key = i mod G, val = i: group k holds i = k + G j, j < J_k = ceil((n-k)/G).
    kv = {"key": (np.arange(n) % g).astype(np.int32), "val": np.arange(n, dtype=np.int64)}
    res = oracle.run(workloads.keyval_plan(), {"kv": kv})
    ks = [k for k in range(g) if k < n]
    j = [(n - k + g - 1) // g for k in ks]
    sums = [k * jk + g * jk * (jk - 1) // 2 for k, jk in zip(ks, j)]
    assert _as_lists(res) == [ks, sums, j]


@pytest.mark.parametrize("spans,m", [((3, 4, 5), 7), ((2, 1, 9), 3), ((5, 5, 1), 1)])
def test_three_part_key_lattice_closed_form(spans, m):
    # Row i = q + P*j (P = A*B*C, j < m) has parts (q mod A, (q div A) mod B,
    # q div AB) offset by (-1, 10, 1992) and val = i: every one of the P groups
    # holds m rows, with SUM(val) = m*q + P*m*(m-1)/2.
    A, B, C = spans
    P = A * B * C
    i = np.arange(P * m)
    q = i % P
    k3 = {"a": (q % A - 1).astype(np.int32), "b": ((q // A) % B + 10).astype(np.int32),
          "c": (q // (A * B) + 1992).astype(np.int32), "val": i.astype(np.int64)}
    got = sorted(zip(*_as_lists(oracle.run(workloads.keys3_plan(), {"k3": k3}))))
    want = sorted((qq % A - 1, (qq // A) % B + 10, qq // (A * B) + 1992, m * qq + P * m * (m - 1) // 2, m)
                  for qq in range(P))
    assert got == want


def test_product_aggregates_closed_form():
    # disc = i mod 11, tax = i mod 9 (every (disc, tax) pair m times over
    # 99 m rows, by the Chinese remainder theorem), price = P, qty = 2;
    # (k1, k2) = (i mod 2, (i div 2) mod 2) is irrelevant to the ungrouped totals.
    m, P = 4, 1234
    n = 99 * m
    i = np.arange(n)
    li = {"date": np.full(n, datagen.DAY0, np.int32),
          "k1": (65 + i % 2).astype(np.uint8), "k2": (88 + (i // 2) % 2).astype(np.uint8),
          "qty": np.full(n, 2, np.int64), "price": np.full(n, P, np.int64),
          "disc": (i % 11).astype(np.int64), "tax": (i % 9).astype(np.int64)}
    plan = workloads.lowcard_plan()
    plan = dict(plan, group_by=[])
    res = _as_lists(oracle.run(plan, {"li": li}))
    s_disc, s_tax = sum(range(11)), sum(range(9))
    expect = [2 * n, P * n, 9 * m * s_disc, 11 * m * s_tax,
              P * 9 * m * (1100 - s_disc),
              P * m * (1100 - s_disc) * (900 + s_tax),
              2 * P * n, n]
    assert res == [[e] for e in expect]


def test_lowcard_groups_partition_the_total():
    t = {"li": datagen.table_lowcard_groups(20_000, seed=5)}
    plan = workloads.lowcard_plan()
    g = oracle.run(plan, t)
    u = oracle.run(dict(plan, group_by=[]), t)
    assert g["kind"] == "grouped" and len(g["cols"][0]) == 4
    for j in range(8):
        assert int(g["cols"][2 + j].sum()) == int(u["cols"][j][0])
    passing = int((t["li"]["date"] <= workloads.LOWCARD_DAY_HI).sum())
    assert int(g["cols"][-1].sum()) == passing
    assert sorted(set(map(int, g["cols"][0]))) == [65, 66]


def test_join_lattice_count():
    # dimension key = i (0..D-1), f = i mod 100, build filter f < t;
    # fact fk = i mod D for n = r D rows: every key is referenced r times.
    D, r, thr = 1234, 3, 37
    dim = {"key": np.arange(D, dtype=np.int32), "f": (np.arange(D) % 100).astype(np.int32)}
    fact = {"fk": (np.arange(D * r) % D).astype(np.int32), "v": np.ones(D * r, np.int64)}
    plan = {"fact": "fact", "builds": [{"table": "dim", "key": "key", "filters": [["f", "lt", thr]],
                                        "payload": []}],
            "probes": [{"build": 0, "fk": "fk"}], "aggs": [["count"]]}
    res = oracle.run(plan, {"fact": fact, "dim": dim})
    keys = (D // 100) * thr + min(D % 100, thr)
    assert _as_lists(res) == [[r * keys]]
    # all filters passing and every FK valid: the join keeps every fact row
    plan["builds"][0]["filters"] = []
    assert _as_lists(oracle.run(plan, {"fact": fact, "dim": dim})) == [[D * r]]


def _random_case(rng: random.Random):
    nf = rng.randint(0, 40)
    nd = [rng.randint(0, 8) for _ in range(2)]
    dims = {}
    for j, m in enumerate(nd):
        keys = rng.sample(range(-5, 15), m)
        dims[f"d{j}"] = {"key": np.array(keys, np.int32),
                         "f": np.array([rng.randint(0, 9) for _ in range(m)], np.int32),
                         "g": np.array([rng.randint(-3, 3) for _ in range(m)], np.int32)}
    fact = {"fk0": np.array([rng.randint(-5, 15) for _ in range(nf)], np.int32),
            "fk1": np.array([rng.randint(-5, 15) for _ in range(nf)], np.int32),
            "a": np.array([rng.randint(-50, 50) for _ in range(nf)], np.int32),
            "u": np.array([rng.randint(0, 255) for _ in range(nf)], np.uint8),
            "v": np.array([rng.randint(-10**6, 10**6) for _ in range(nf)], np.int64)}
    tables = {"f": fact, **dims}
    nprobe = rng.randint(0, 2)
    builds, probes = [], []
    for j in range(nprobe):
        builds.append({"table": f"d{j}", "key": "key",
                       "filters": [["f", rng.choice(["lt", "ge"]), rng.randint(0, 9)]] if rng.random() < .7 else [],
                       "payload": ["g", "f"]})
        probes.append({"build": j, "fk": f"fk{j}"})
    ops = [("lt",), ("le",), ("gt",), ("ge",), ("eq",), ("between",)]
    filters = []
    for _ in range(rng.randint(0, 2)):
        col = rng.choice(["a", "u", "v"])
        op = rng.choice(ops)[0]
        lo = rng.randint(-60, 260) if col != "v" else rng.randint(-10**6, 10**6)
        filters.append([col, "between", lo, lo + rng.randint(0, 200)] if op == "between" else [col, op, lo])
    refs = ["a", "u", "v"] + [["payload", p, i] for p in range(nprobe) for i in range(2)]
    plan = {"fact": "f", "builds": builds, "probes": probes, "filters": filters}
    if rng.random() < 0.25:
        plan["project"] = rng.sample(refs, rng.randint(1, 3))
    else:
        keyable = [r for r in refs if r != "v"]
        plan["group_by"] = rng.sample(keyable, rng.randint(0, min(3, len(keyable))))
        aggs = []
        for _ in range(rng.randint(1, 4)):
            f = rng.choice(["sum", "count", "min", "max"])
            if f == "count":
                aggs.append(["count"])
                continue
            terms = []
            for _ in range(rng.randint(1, 3)):
                k = rng.choice(["x", "x_plus_c", "c_minus_x"])
                r = rng.choice(refs)
                terms.append([k, r] if k == "x" else [k, r, rng.randint(-100, 100)])
            aggs.append([f, terms])
        plan["aggs"] = aggs
    return plan, tables


@pytest.mark.parametrize("seed", range(300))
def test_oracle_matches_nested_loop_bruteforce(seed):
    plan, tables = _random_case(random.Random(seed))
    want = bruteforce.evaluate(plan, tables)
    got = oracle.run(plan, tables)
    assert got["kind"] == want["kind"]
    # an ungrouped MIN/MAX over no rows is undefined; both sides report 0 there
    assert _as_lists(got) == want["cols"]


def test_duplicate_build_key_is_an_error():
    dim = {"key": np.array([1, 2, 1], np.int32)}
    fact = {"fk": np.array([1], np.int32)}
    plan = {"fact": "fact", "builds": [{"table": "dim", "key": "key", "payload": []}],
            "probes": [{"build": 0, "fk": "fk"}], "aggs": [["count"]]}
    with pytest.raises(oracle.OracleError) as e:
        oracle.run(plan, {"fact": fact, "dim": dim})
    assert e.value.code == -6
    # a duplicate removed by the build filter is not a duplicate
    dim["f"] = np.array([0, 0, 1], np.int32)
    plan["builds"][0]["filters"] = [["f", "eq", 0]]
    assert _as_lists(oracle.run(plan, {"fact": fact, "dim": dim})) == [[1]]


def test_empty_inputs():
    t = {"t": {"a": np.zeros(0, np.int32), "b": np.zeros(0, np.int32), "price": np.zeros(0, np.int64)}}
    assert _as_lists(oracle.run(workloads.filter_agg_plan(), t)) == [[0], [0]]
    assert _as_lists(oracle.run(workloads.filter_project_plan(), t)) == [[], []]
    kv = {"kv": {"key": np.zeros(0, np.int32), "val": np.zeros(0, np.int64)}}
    assert _as_lists(oracle.run(workloads.keyval_plan(), kv)) == [[], [], []]


def test_no_row_passes():
    t = {"t": datagen.table_filter_agg(5000, seed=3)}
    res = oracle.run(workloads.filter_agg_plan(a_lt=0), t)
    assert _as_lists(res) == [[0], [0]]


def test_overflow_flag():
    kv = {"kv": {"key": np.zeros(3, np.int32), "val": np.array([2**62, 2**62, 2**62], np.int64)}}
    res = oracle.run(workloads.keyval_plan(), kv)
    assert res["overflow"]
    assert int(res["cols"][1][0]) == bruteforce.wrap(3 * 2**62)
    res = oracle.run(workloads.keyval_plan(), {"kv": {"key": np.zeros(2, np.int32),
                                                      "val": np.array([5, 6], np.int64)}})
    assert not res["overflow"]


@pytest.mark.parametrize("plan_fn,table_fn", [
    (workloads.filter_agg_plan, lambda: {"t": datagen.table_filter_agg(50_000, 11)}),
    (workloads.filter_project_plan, lambda: {"t": datagen.table_filter_agg(50_000, 11)}),
    (workloads.lowcard_plan, lambda: {"li": datagen.table_lowcard_groups(50_000, 12)}),
    (workloads.keyval_plan, lambda: {"kv": datagen.table_keyval(50_000, 1000, "zipf", 13)}),
])
def test_threads_do_not_change_the_result(plan_fn, table_fn):
    t = table_fn()
    a = oracle.run(plan_fn(), t, nthreads=1)
    b = oracle.run(plan_fn(), t, nthreads=4)
    assert _as_lists(a) == _as_lists(b)


def test_star_join_small_matches_bruteforce_on_sample():
    # Full-size star schema shapes with a tiny fact table: the nested loop over
    # the four (filtered) dimensions is still affordable for 40 fact rows.
    s = datagen.star_schema(n=40, seed=21)
    small = {"fact": s["fact"]}
    for name, rows, _ in datagen.STAR_DIMS:
        small[name] = {k: v[: min(rows, 300)] for k, v in s[name].items()}
        # keep every key the fact table references so some rows join
        need = np.unique(s["fact"]["fk_" + name[2:]])
        pos = np.searchsorted(np.sort(s[name]["key"]), need)
        order = np.argsort(s[name]["key"])
        pick = order[pos]
        small[name] = {k: np.concatenate([v[pick], v[:0]]) for k, v in s[name].items()}
    plan = workloads.star_plan({"d_a": 60, "d_b": 60, "d_c": 60, "d_d": 60})
    want = bruteforce.evaluate(plan, small)
    got = oracle.run(plan, small)
    assert _as_lists(got) == want["cols"]
    assert sum(want["cols"][-1]) > 0


@pytest.mark.parametrize("n,seed,regions", [(1203, 3, 3), (2001, 4, 1), (37, 5, 5)])
def test_chain_of_pipelines_matches_brute_force(n, seed, regions):
    """A query of several pipelines (workloads.q5_chain, shaped like TPC-H
    Q5): each step's result becomes a table of the next steps.  The oracle's
    step-by-step evaluation equals the nested-loop brute force composed the
    same way, and the per-region result adds up to the per-nation one."""
    tables = datagen.tpch_schema(n, seed=seed)
    chain = workloads.q5_chain(regions=regions)
    got = oracle.run_chain(chain, tables)
    bt = dict(tables)
    for st, res in zip(chain, got):
        want = bruteforce.evaluate(st["plan"], bt)
        assert res["kind"] == want["kind"]
        assert _as_lists(res) == want["cols"]  # projections in input order, groups by key, on both sides
        bt[st["name"]] = {c: np.asarray(v, dtype=np.int64) for c, v in zip(st["columns"], want["cols"])}
    nat, reg = got[2]["cols"], got[3]["cols"]
    assert int(reg[1].sum()) == int(nat[1].sum()) and int(reg[2].sum()) == int(nat[2].sum())
    assert int(reg[3].sum()) == len(nat[0])  # nations per region
    assert all(int(x) // 5 < regions for x in nat[0])  # only nations of the selected regions
