"""Query plans of the evaluated workloads, as neutral plan dicts (data only).

A plan is the pipeline program(s) of one query (Table 2): optional build
pipelines (FILTER + HASH_PUT on a dimension), then one probe/scan pipeline
(LOOP, FILTER, HASH_PROBE*, ARITHMETIC, then AGGREGATE, HASH_AGGREGATE or
PROJECT).  The format is documented in the Python binding
(``paper_1709_00700_gb300.pv.plan_to_spec``); it carries no arithmetic.
"""
from __future__ import annotations

from . import datagen

# Plain filter-aggregate / filter-project query on the 1M-row table:
#   WHERE a < 10 AND 20 <= b <= 40  -> SUM(price), COUNT(*)  and  (a, price) rows.
def filter_agg_plan(a_lt: int = 10, b_lo: int = 20, b_hi: int = 40) -> dict:
    return {"fact": "t", "filters": [["a", "lt", a_lt], ["b", "between", b_lo, b_hi]],
            "aggs": [["sum", [["x", "price"]]], ["count"]]}


def filter_project_plan(a_lt: int = 10, b_lo: int = 20, b_hi: int = 40) -> dict:
    return {"fact": "t", "filters": [["a", "lt", a_lt], ["b", "between", b_lo, b_hi]],
            "project": ["a", "price"]}


# Low-cardinality grouped aggregation (4 groups, 8 aggregates of fixed-point
# products), shaped like the compute-heavy aggregation pipeline of TPC-H Q1.
LOWCARD_DAY_HI = datagen.DAY0 + 2475


def lowcard_plan(day_hi: int = LOWCARD_DAY_HI) -> dict:
    return {
        "fact": "li",
        "filters": [["date", "le", day_hi]],
        "group_by": ["k1", "k2"],
        "aggs": [
            ["sum", [["x", "qty"]]],
            ["sum", [["x", "price"]]],
            ["sum", [["x", "disc"]]],
            ["sum", [["x", "tax"]]],
            ["sum", [["x", "price"], ["c_minus_x", "disc", 100]]],
            ["sum", [["x", "price"], ["c_minus_x", "disc", 100], ["x_plus_c", "tax", 100]]],
            ["sum", [["x", "qty"], ["x", "price"]]],
            ["count"],
        ],
    }


# High-cardinality grouped aggregation: SUM(val), COUNT(*) GROUP BY key,
# optionally filtered on val (selectivity knob of the random query suite).
def keyval_plan(val_lt: int | None = None) -> dict:
    p = {"fact": "kv", "group_by": ["key"], "aggs": [["sum", [["x", "val"]]], ["count"]]}
    if val_lt is not None:
        p["filters"] = [["val", "lt", val_lt]]
    return p


# Star join shaped like SSB Q4.1: four build pipelines (dimension filter
# f < t, HASH_PUT key with the grouping attribute as payload) and one probe
# pipeline that probes all four and groups on two dimension attributes.
STAR_THRESHOLDS = {"d_a": 20, "d_b": 20, "d_c": 5, "d_d": 10}
STAR_PROBE_ORDER = ("d_c", "d_d", "d_a", "d_b")   # most selective first


def star_plan(thresholds: dict | None = None, order=STAR_PROBE_ORDER) -> dict:
    th = dict(STAR_THRESHOLDS)
    th.update(thresholds or {})
    builds, probes = [], []
    for name in order:
        pay = ["g"] if name in ("d_a", "d_b") else []
        builds.append({"table": name, "key": "key", "filters": [["f", "lt", th[name]]], "payload": pay})
        probes.append({"build": len(builds) - 1, "fk": "fk_" + name[2:]})
    ia, ib = order.index("d_a"), order.index("d_b")
    return {"fact": "fact", "builds": builds, "probes": probes,
            "group_by": [["payload", ia, 0], ["payload", ib, 0]],
            "aggs": [["sum", [["x", "revenue"]]], ["count"]]}


# Grouped aggregation on a composite key of three fact columns:
# SUM(val), COUNT(*) GROUP BY a, b, c.
def keys3_plan() -> dict:
    return {"fact": "k3", "group_by": ["a", "b", "c"], "aggs": [["sum", [["x", "val"]]], ["count"]]}


# Star join shaped like SSB Q3.1: customers and suppliers of one region, the
# years [year_lo, year_hi]; probes in that order (most selective first);
# SUM(revenue) GROUP BY customer nation, supplier nation, year.
STAR3_REGIONS = (2, 2)
STAR3_YEARS = (datagen.STAR3_YEAR0, datagen.STAR3_YEAR0 + 5)


def star3_plan(regions=STAR3_REGIONS, years=STAR3_YEARS) -> dict:
    builds = [{"table": "d_cust", "key": "key", "filters": [["region", "eq", regions[0]]], "payload": ["nation"]},
              {"table": "d_supp", "key": "key", "filters": [["region", "eq", regions[1]]], "payload": ["nation"]},
              {"table": "d_date", "key": "key", "filters": [["year", "between", years[0], years[1]]],
               "payload": ["year"]}]
    return {"fact": "fact", "builds": builds,
            "probes": [{"build": 0, "fk": "fk_cust"}, {"build": 1, "fk": "fk_supp"}, {"build": 2, "fk": "fk_date"}],
            "group_by": [["payload", 0, 0], ["payload", 1, 0], ["payload", 2, 0]],
            "aggs": [["sum", [["x", "revenue"]]]]}


# Filter/aggregate on dictionary-coded part attributes, shaped like the part
# selection of SSB Q2.2: category = c AND brand BETWEEN b0 AND b1 ->
# SUM(price), COUNT(*).  Other string predicates replace the two filters.
def parts_text_plan(filters=(("category", "eq", "MFGR#12"), ("brand", "between", "MFGR#1221", "MFGR#1228"))) -> dict:
    return {"fact": "parts", "filters": [list(f) for f in filters],
            "aggs": [["sum", [["x", "price"]]], ["count"]]}


# A query of several pipelines where later pipelines read earlier results,
# shaped like TPC-H Q5 (Section 9.2.1): revenue of the line items whose order
# falls in one year and whose customer lives in a nation of the first
# `regions` regions, per nation, then per region.  Each step is a pipeline
# program; its result columns become table step["name"] with step["columns"],
# which later steps build hash tables on (a build over a probe pipeline's
# result) or scan (an aggregation over an aggregation):
#   cust:   customers of the selected nations        (probe, PROJECT)
#   ord:    orders of the year by those customers    (build on cust, probe, PROJECT)
#   nat:    line items of those orders, per nation   (build on ord, probe, HASH_AGGREGATE)
#   region: the nations' revenue per region          (probe, HASH_AGGREGATE over nat)
Q5_YEAR = (datagen.DAY0 + 730, datagen.DAY0 + 1094)   # the third year of the order dates


def q5_chain(regions: int = 3, days=Q5_YEAR) -> list:
    sel_nations = {"table": "nation", "key": "n_nationkey", "filters": [["n_regionkey", "lt", regions]],
                   "payload": []}
    return [
        {"name": "cust", "columns": ["custkey", "nation"],
         "plan": {"fact": "customer", "builds": [sel_nations], "probes": [{"build": 0, "fk": "c_nationkey"}],
                  "project": ["c_custkey", "c_nationkey"]}},
        {"name": "ord", "columns": ["orderkey", "nation"],
         "plan": {"fact": "orders", "filters": [["o_orderdate", "between", days[0], days[1]]],
                  "builds": [{"table": "cust", "key": "custkey", "filters": [], "payload": ["nation"]}],
                  "probes": [{"build": 0, "fk": "o_custkey"}], "project": ["o_orderkey", ["payload", 0, 0]]}},
        {"name": "nat", "columns": ["nation", "revenue", "lines"],
         "plan": {"fact": "lineitem",
                  "builds": [{"table": "ord", "key": "orderkey", "filters": [], "payload": ["nation"]}],
                  "probes": [{"build": 0, "fk": "l_orderkey"}], "group_by": [["payload", 0, 0]],
                  "aggs": [["sum", [["x", "l_extendedprice"], ["c_minus_x", "l_discount", 100]]], ["count"]]}},
        {"name": "region", "columns": ["region", "revenue", "lines", "nations", "top_nation_revenue"],
         "plan": {"fact": "nat",
                  "builds": [{"table": "nation", "key": "n_nationkey", "filters": [], "payload": ["n_regionkey"]}],
                  "probes": [{"build": 0, "fk": "nation"}], "group_by": [["payload", 0, 0]],
                  "aggs": [["sum", [["x", "revenue"]]], ["sum", [["x", "lines"]]], ["count"],
                           ["max", [["x", "revenue"]]]]}},
    ]
