"""HASH_PROBE order as a variant, pinned with no GPU: every order of a plan's
probes, rewritten by pv.reorder_probes and evaluated by the oracle, gives the
plan's own result once the key columns are put back (pv.restore_key_order)."""
import json
import os

import numpy as np
import pytest

from oracle import oracle
from paper_1709_00700_gb300 import autotune, datagen, pv, workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(cols):
    return sorted(zip(*[[int(v) for v in c] for c in cols]))


def _every_order_agrees(plan, tables):
    want = oracle.run(plan, tables)
    orders = pv.probe_orders(plan)
    for order in orders:
        rp, perm = pv.reorder_probes(plan, order)
        assert [q["fk"] for q in rp["probes"]] == [plan["probes"][o]["fk"] for o in order]
        got = pv.restore_key_order(oracle.run(rp, tables)["cols"], perm)
        if want["kind"] == "project":  # input order, whatever the probe order
            assert [c.tolist() for c in got] == [c.tolist() for c in want["cols"]], order
        else:
            assert _rows(got) == _rows(want["cols"]), order
    return len(orders)


def test_star_join_every_probe_order():
    s = datagen.star_schema(20_000, seed=4)
    assert _every_order_agrees(workloads.star_plan({"d_a": 60, "d_b": 50, "d_c": 30, "d_d": 40}), s) == 24


def test_three_probe_join_every_probe_order():
    s = datagen.star3_schema(20_000, seed=4)
    assert _every_order_agrees(workloads.star3_plan(regions=(1, 3)), s) == 6


@pytest.mark.parametrize("fixture", ["table2_join_group_x.json", "table2_join_group_y.json"])
def test_table2_programs_every_probe_order(fixture):
    g = json.load(open(os.path.join(GOLDEN, fixture)))
    tables = {t: {c: np.array(v["values"], dtype=v["dtype"]) for c, v in cols.items()} for t, cols in g["tables"].items()}
    assert _every_order_agrees(g["plan"], tables) == 2


def test_join_project_of_payloads_every_probe_order():
    s = datagen.star_schema(5_000, seed=8)
    plan = workloads.star_plan({"d_a": 60, "d_b": 50, "d_c": 30, "d_d": 40})
    plan = {k: v for k, v in plan.items() if k not in ("group_by", "aggs")}
    plan["project"] = [["payload", 3, 0], "revenue", ["payload", 2, 0]]
    assert _every_order_agrees(plan, s) == 24


def test_moving_the_grouping_dimensions_keeps_the_compiled_shape():
    # star plan: probes (d_c, d_d, d_a, d_b), grouped on the payloads of probes 2 and 3.  Swapping the
    # payload-less probes, the grouping ones, or both, keeps the keys at positions 2 and 3 (listed
    # by position); the canonical shape is unchanged and only the key columns swap.
    plan = workloads.star_plan()
    for order, perm in (((0, 1, 2, 3), [0, 1]), ((1, 0, 2, 3), [0, 1]), ((0, 1, 3, 2), [1, 0]),
                        ((1, 0, 3, 2), [1, 0])):
        rp, kp = pv.reorder_probes(plan, order)
        assert rp["group_by"] == [["payload", 2, 0], ["payload", 3, 0]] and kp == perm, order
    rp, kp = pv.reorder_probes(plan, (2, 0, 1, 3))  # a grouping dimension probed first: another shape
    assert rp["group_by"] == [["payload", 0, 0], ["payload", 3, 0]]


def test_reorder_rejects_a_non_permutation_and_restores_keys():
    plan = workloads.star_plan()
    with pytest.raises(pv.PVError) as e:
        pv.reorder_probes(plan, (0, 1, 1, 3))
    assert e.value.status == -1
    cols = [np.array([1]), np.array([2]), np.array([30]), np.array([4])]
    assert [int(c[0]) for c in pv.restore_key_order(cols, [1, 0])] == [2, 1, 30, 4]
    assert autotune.probe_order_dim(plan)[0] == "probe_order" and len(autotune.probe_order_dim(plan)[1]) == 24
