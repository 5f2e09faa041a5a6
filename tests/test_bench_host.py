"""Host-side logic of bench.py: the sector-exact byte count of the pipelines
(star joins, filters in front of aggregations and projections) checked
against a row-by-row count on small tables (no GPU)."""
import numpy as np
import pytest

import bench


def _brute_sector_bytes(tables, plan):
    fact = tables[plan["fact"]]
    n = len(next(iter(fact.values())))
    alive = [True] * n
    total = 0

    def count(elem):
        per = 32 // elem
        return 32 * sum(1 for s in range(0, n, per) if any(alive[s:s + per]))

    for i, p in enumerate(plan["probes"]):
        b = plan["builds"][p["build"]]
        dim = tables[b["table"]]
        passing = set()
        for r in range(len(dim[b["key"]])):
            ok = True
            for col, op, *c in b["filters"]:
                v = int(dim[col][r])
                ok &= {"lt": v < c[0], "le": v <= c[0], "ge": v >= c[0], "eq": v == c[0],
                       "between": c[0] <= v <= c[-1]}[op]
            if ok:
                passing.add(int(dim[b["key"]][r]))
        fk = fact[p["fk"]]
        total += fk.itemsize * n if i == 0 else count(fk.itemsize)
        alive = [alive[r] and int(fk[r]) in passing for r in range(n)]
    for a in plan["aggs"]:
        for term in (a[1] if len(a) > 1 else []):
            total += count(fact[term[1]].itemsize)
    return total


@pytest.mark.parametrize("n,seed", [(37, 1), (64, 2), (203, 3), (1, 4)])
def test_star_sector_bytes_matches_row_by_row_count(n, seed):
    rng = np.random.default_rng(seed)
    dims = {}
    for name, rows in (("d1", 11), ("d2", 7)):
        dims[name] = {"key": rng.permutation(rows).astype(np.int32), "f": rng.integers(0, 10, rows).astype(np.int32)}
    fact = {"fk_1": rng.integers(0, 11, n).astype(np.int32), "fk_2": rng.integers(0, 7, n).astype(np.int32),
            "rev": rng.integers(0, 100, n).astype(np.int64)}
    plan = {"fact": "fact",
            "builds": [{"table": "d1", "key": "key", "filters": [["f", "lt", 4]], "payload": []},
                       {"table": "d2", "key": "key", "filters": [["f", "between", 2, 8]], "payload": []}],
            "probes": [{"build": 0, "fk": "fk_1"}, {"build": 1, "fk": "fk_2"}],
            "aggs": [["sum", [["x", "rev"]]], ["count"]]}
    tables = {"fact": fact, **dims}
    assert bench.star_sector_bytes(tables, plan) == _brute_sector_bytes(tables, plan)


def test_star_sector_bytes_bounds():
    from paper_1709_00700_gb300 import datagen, workloads
    s = datagen.star_schema(100_000)
    b = bench.star_sector_bytes(s, workloads.star_plan())
    assert 4 * 100_000 < b < 24 * 100_000


def test_star3_sector_bytes_matches_row_by_row_count():
    # the three-probe join's eq / between build filters, on a small SSB Q3.1-shaped schema
    from paper_1709_00700_gb300 import datagen, workloads
    s = datagen.star3_schema(3_001, seed=6)
    plan = workloads.star3_plan()
    b = bench.star_sector_bytes(s, plan)
    assert b == _brute_sector_bytes(s, plan)
    assert 4 * 3_001 < b < 20 * 3_001


_CMP = {"lt": lambda v, c: v < c[0], "le": lambda v, c: v <= c[0], "gt": lambda v, c: v > c[0],
        "ge": lambda v, c: v >= c[0], "eq": lambda v, c: v == c[0], "between": lambda v, c: c[0] <= v <= c[1]}


def _brute_filter_bytes(fact, plan):
    """Row by row: the first filter column in full, each later column (in order
    of first use, the sink's columns last) in the 32-byte sectors holding a row
    that is alive when it is read, plus 12 bytes per projected (int32, int64) row."""
    n = len(next(iter(fact.values())))
    alive = [True] * n
    order = []
    for p in plan["filters"]:
        if p[0] not in order:
            order.append(p[0])
    sink = [r for r in plan.get("project", [])] + [t[1] for a in plan.get("aggs", []) for t in
                                                     (a[1] if len(a) > 1 else [])]
    total = 0
    for i, col in enumerate(order + [c for c in sink if c not in order]):
        if col in order[:i] or (i >= len(order) and col in sink[:sink.index(col)]):
            continue
        per = 32 // fact[col].itemsize
        total += fact[col].itemsize * n if i == 0 else \
            32 * sum(1 for s in range(0, n, per) if any(alive[s:s + per]))
        for p in plan["filters"]:
            if p[0] == col:
                alive = [alive[r] and _CMP[p[1]](int(fact[col][r]), p[2:]) for r in range(n)]
    out = sum(fact[c].itemsize for c in plan.get("project", []))
    return total + out * sum(alive)


@pytest.mark.parametrize("n,seed,kind", [(1, 5, "aggregate"), (77, 6, "project"), (1003, 7, "aggregate"),
                                         (1003, 8, "project")])
def test_filter_sector_bytes_matches_row_by_row_count(n, seed, kind):
    from paper_1709_00700_gb300 import datagen, workloads
    t = datagen.table_filter_agg(n, seed=seed)
    plan = workloads.filter_agg_plan(30, 10, 60) if kind == "aggregate" else workloads.filter_project_plan(30, 10, 60)
    got = bench.sector_bytes({"t": t}, plan)
    assert got == _brute_filter_bytes(t, plan)
    full = bench.sector_bytes({"t": t}, plan, lazy=False)
    assert got <= full and full == 16 * n + (12 * len([1 for a, b in zip(t["a"], t["b"]) if a < 30 and 10 <= b <= 60])
                                             if kind == "project" else 0)


def test_unfiltered_pipelines_read_every_column_in_full():
    from paper_1709_00700_gb300 import datagen, workloads
    li = datagen.table_lowcard_groups(4_001)
    assert bench.sector_bytes({"k3": datagen.table_keys3(1000)}, workloads.keys3_plan()) == 20 * 1000
    b = bench.sector_bytes({"li": li}, workloads.lowcard_plan())
    assert 37 * 4_001 < b <= 38 * 4_001 + 6 * 32  # partial last sectors count whole
