"""The exchange step of the row-sharded (multi-GPU) design, on CPU ranks over
gloo: each rank evaluates the plan with the oracle on its slice of the fact
rows (standing in for its GPU), the partial results are all-gathered, and
shard.merge must give the oracle's result on the whole table."""
import os
import socket

import numpy as np
import pytest

from paper_1709_00700_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _cases():
    import json
    from paper_1709_00700_gb300 import datagen, workloads
    kv = {"kv": datagen.table_keyval(30_011, 500, "zipf", seed=3)}
    t = {"t": datagen.table_filter_agg(20_003, seed=5)}
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table2_join_group_y.json")))
    t2 = {n: {c: np.array(v["values"], dtype=v["dtype"]) for c, v in cols.items()} for n, cols in g["tables"].items()}
    only_high = {"fact": "kv", "filters": [["val", "ge", 999_000]],
                 "aggs": [["sum", [["x", "val"]]], ["count"], ["min", [["x", "val"]]], ["max", [["x", "key"]]]]}
    return [
        ("keyval", workloads.keyval_plan(), kv),
        ("keyval_totals_min_max", only_high, kv),  # few rows pass: a rank may have none
        ("lowcard", workloads.lowcard_plan(), {"li": datagen.table_lowcard_groups(25_007, seed=7)}),
        ("filter_agg", workloads.filter_agg_plan(), t),
        ("filter_project", workloads.filter_project_plan(), t),
        ("star", workloads.star_plan({"d_a": 60, "d_b": 50, "d_c": 30, "d_d": 40}), datagen.star_schema(30_001, 9)),
        ("star3", workloads.star3_plan(), datagen.star3_schema(30_001, 9)),
        ("keys3", workloads.keys3_plan(), {"k3": datagen.table_keys3(30_001, seed=2)}),
        ("table2_min_max", g["plan"], t2),
    ]


def _rank_main(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    from oracle import oracle
    dist.init_process_group("gloo")
    out = []
    for name, plan, tables in _cases():
        fact = plan["fact"]
        n = len(next(iter(tables[fact].values())))
        a, b = shard.row_slice(n, rank, world)
        mine = dict(tables)
        mine[fact] = {c: v[a:b] for c, v in tables[fact].items()}
        part = oracle.run(plan, mine)["cols"]
        parts = [None] * world
        dist.all_gather_object(parts, part)
        merged = shard.merge(plan, parts)
        whole = oracle.run(plan, tables)["cols"]
        ok = len(merged) == len(whole) and all(np.array_equal(x, y) for x, y in zip(merged, whole))
        out.append((name, ok))
    dist.destroy_process_group()
    q.put((rank, out))


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_partials_merge_to_the_whole_result(world):
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, results in got:
        bad = [name for name, ok in results if not ok]
        assert not bad, (rank, bad)


def test_row_slices_partition_the_rows():
    for n in (0, 1, 7, 100):
        for world in (1, 2, 3, 8):
            spans = [shard.row_slice(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
            assert max(b - a for a, b in spans) - min(b - a for a, b in spans) <= 1


def test_merge_needs_a_count_for_ungrouped_min_max():
    plan = {"fact": "t", "aggs": [["min", [["x", "v"]]]]}
    with pytest.raises(ValueError):
        shard.merge(plan, [[np.array([1])], [np.array([2])]])


def test_ungrouped_min_max_skip_ranks_without_rows():
    plan = {"fact": "t", "aggs": [["sum", [["x", "v"]]], ["count"], ["min", [["x", "v"]]], ["max", [["x", "v"]]]]}
    empty = [np.array([0]), np.array([0]), np.array([0]), np.array([0])]   # MIN/MAX of no rows read 0
    live = [np.array([-7]), np.array([2]), np.array([-5]), np.array([-2])]
    for parts in ([empty, live], [live, empty], [empty, live, empty]):
        assert [int(c[0]) for c in shard.merge(plan, parts)] == [-7, 2, -5, -2]
    assert [int(c[0]) for c in shard.merge(plan, [empty, empty])] == [0, 0, 0, 0]
