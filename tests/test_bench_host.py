"""Host-side logic of bench.py: the sector-exact byte count of the star join
checked against a row-by-row count on small tables (no GPU)."""
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
