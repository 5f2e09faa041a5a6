"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Every result is int64 fixed point, so the bar is bit-exact equality.
Grouped results are compared after sorting by key (group order is not
defined); single-pass projections after sorting rows (write order is not
defined); multi-pass projections in input order exactly.
"""
import itertools

import numpy as np
import pytest

from paper_1709_00700_gb300 import datagen, pv, workloads
from tests.gpu_util import assert_same, register, want

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    c = pv.Context(0)
    yield c
    c.close()


def run_or_skip(ctx, plan, var, htv=None):
    try:
        return ctx.query(plan, var, htv)
    except pv.PVError as e:
        if e.status == -2:  # no instantiation for this variant (e.g. registers for 1024 threads)
            return None
        raise


SCAN_VARIANTS = [dict(pred=p, access=a, items_per_thread=u, block=b, grid_mult=g)
                 for p, a, u, b, g in itertools.product(["branch", "predicated"], ["grid", "chunked"],
                                                        [1, 2, 4], [64, 256, 1024], [0, 1])]


# ---------------------------------------------------------------- AGGREGATE
@pytest.mark.parametrize("n", [0, 1, 3, 5, 4096, 100_003])
def test_filter_aggregate_all_variants(ctx, n):
    t = {"t": datagen.table_filter_agg(n, seed=n + 1)}
    register(ctx, t)
    plan = workloads.filter_agg_plan()
    w = want(plan, t)
    ran = 0
    for kw in SCAN_VARIANTS:
        got = run_or_skip(ctx, plan, pv.variant(**kw))
        if got is None:
            continue
        ran += 1
        assert_same(got, w, ctxmsg=str(kw))
    assert ran >= len(SCAN_VARIANTS) // 2


def test_filter_aggregate_lattice_closed_form(ctx):
    m = 3
    t = {"t": datagen.table_lattice(m)}
    register(ctx, t)
    got = ctx.query(workloads.filter_agg_plan(), pv.variant())
    count = 210 * m
    total = (100 * count + 10_000 * (m * (m - 1) // 2) * 210 + 100 * sum(range(20, 41)) * 10 * m
             + sum(range(10)) * 21 * m)
    assert [int(got[0][0]), int(got[1][0])] == [total, count]


@pytest.mark.parametrize("a_lt,b_lo,b_hi", [(0, 20, 40), (100, 0, 99), (10, 40, 20), (-5, 0, 10)])
def test_filter_aggregate_degenerate_predicates(ctx, a_lt, b_lo, b_hi):
    t = {"t": datagen.table_filter_agg(20_000, seed=4)}
    register(ctx, t)
    plan = workloads.filter_agg_plan(a_lt, b_lo, b_hi)
    for pred in ("branch", "predicated"):
        assert_same(ctx.query(plan, pv.variant(pred=pred)), want(plan, t), ctxmsg=pred)


def test_lowcard_totals_and_minmax(ctx):
    li = {"li": datagen.table_lowcard_groups(77_777, seed=9)}
    register(ctx, li)
    plan = dict(workloads.lowcard_plan(), group_by=[])
    w = want(plan, li)
    for pred in ("branch", "predicated"):
        assert_same(ctx.query(plan, pv.variant(pred=pred)), w, ctxmsg=pred)
    kv = {"kv": datagen.table_keyval(33_333, 10, seed=3)}
    register(ctx, kv)
    plan = {"fact": "kv", "filters": [["val", "between", 1000, 900_000]],
            "aggs": [["sum", [["x", "val"]]], ["count"], ["min", [["x", "val"]]], ["max", [["x", "val"]]]]}
    for pred in ("branch", "predicated"):
        assert_same(ctx.query(plan, pv.variant(pred=pred)), want(plan, kv), ctxmsg=pred)
    # MIN/MAX over no row read 0, as the oracle reports
    plan["filters"] = [["val", "lt", -1]]
    assert [int(c[0]) for c in ctx.query(plan, pv.variant())] == [0, 0, 0, 0]


# ---------------------------------------------------------------- PROJECT
@pytest.mark.parametrize("n", [0, 2, 7, 4097, 250_001])
def test_filter_project_single_and_multi_pass(ctx, n):
    t = {"t": datagen.table_filter_agg(n, seed=n + 2)}
    register(ctx, t)
    plan = workloads.filter_project_plan()
    w = want(plan, t)
    for kw in SCAN_VARIANTS[::3]:
        for ex in ("single", "multi"):
            got = run_or_skip(ctx, plan, pv.variant(exec=ex, **kw))
            if got is None:
                continue
            assert_same(got, w, ordered=(ex == "multi"), ctxmsg=f"{ex} {kw}")
    # projected columns keep their source types
    res = ctx.run(plan, pv.variant(exec="multi"))
    cols = ctx.fetch(res)
    ctx.free(res)
    assert cols[0].dtype == np.int32 and cols[1].dtype == np.int64


def test_project_golden_example(ctx):
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "select_b_where_a_lt_5.json")))
    tables = {t: {c: np.array(v["values"], dtype=v["dtype"]) for c, v in cols.items()} for t, cols in g["tables"].items()}
    # the compiled projection shape reads (a, b, price); pad the table with a price column
    tables["t"]["price"] = np.arange(8, dtype=np.int64)
    register(ctx, tables)
    plan = {"fact": "t", "filters": [["a", "lt", 5]], "project": ["b", "price"]}
    got = ctx.query(plan, pv.variant(exec="multi"))
    assert list(map(int, got[0])) == g["expected"]["cols"][0]


@pytest.mark.parametrize("ex", ["single", "multi"])
def test_project_output_overflow_is_reported(ctx, ex):
    t = {"t": datagen.table_filter_agg(50_000, seed=5)}
    register(ctx, t)
    plan = dict(workloads.filter_project_plan(), capacity_hint=10)
    with pytest.raises(pv.PVError) as e:
        ctx.query(plan, pv.variant(exec=ex))
    assert e.value.status == -7
    ctx.sync()  # the error word was cleared by the failing fetch


# ---------------------------------------------------------------- HASH_AGGREGATE
GROUP_VARIANTS = [dict(agg=a, ht=h, exec=e, pred=p, access=ac, items_per_thread=u, threads_per_table=tp, hash=hs)
                  for a, h, e, p, ac, u, tp, hs in itertools.product(
                      ["local", "global"], ["linear", "cuckoo", "perfect"], ["single", "multi"],
                      ["branch", "predicated"], ["grid", "chunked"], [1, 2], [0, 1], ["murmur", "multshift"])]


def _grouped_all_variants(ctx, plan, tables, step=1, min_ran=10):
    w = want(plan, tables)
    ran = 0
    for kw in GROUP_VARIANTS[::step]:
        got = run_or_skip(ctx, plan, pv.variant(**kw))
        if got is None:
            continue
        ran += 1
        assert_same(got, w, ctxmsg=str(kw))
    assert ran >= min_ran
    return ran


def test_lowcard_grouped_all_variants(ctx):
    li = {"li": datagen.table_lowcard_groups(60_001, seed=11)}
    register(ctx, li)
    _grouped_all_variants(ctx, workloads.lowcard_plan(), li, min_ran=60)


@pytest.mark.parametrize("n,big,near", [(60_001, 0.001, False), (4_099, 0.3, False), (1_000_003, 0.00001, False),
                                        (300_007, 0.5, True), (2_000_003, 0.01, True)])
def test_lowcard_thread_private_32bit_fields(ctx, n, big, near):
    """Thread-private tables keep the plain-column sums and the count in 32-bit
    fields.  Rows with a value beyond 32 bits or negative (here: quantities
    and prices of a fraction `big` of the rows) go straight to the global
    table; a field whose sum would carry out of 32 bits flushes its exact sum
    into the global table (near: the picked prices lie in [2^31, 2^32), so a
    thread's field overflows every few rows).  All paths, exact against the
    oracle."""
    li = datagen.table_lowcard_groups(n, seed=n)
    rng = np.random.default_rng(n)
    pick = rng.random(n) < big
    if not near:
        li["qty"] = np.where(pick, rng.integers(-2**40, 2**40, n), li["qty"]).astype(np.int64)
    pick = rng.random(n) < big
    hi = 2**32 if near else 2**33
    li["price"] = np.where(pick, rng.integers(2**31, hi, n), li["price"]).astype(np.int64)
    t = {"li": li}
    register(ctx, t)
    w = want(workloads.lowcard_plan(), t)
    for kw in (dict(pred="predicated"), dict(pred="branch"), dict(pred="compacted"),
               dict(pred="predicated", block=1024, grid_mult=1), dict(pred="branch", prefetch=1, block=64),
               dict(pred="predicated", access="staged")):
        kw = dict(kw, agg="local", ht="perfect", threads_per_table=1, items_per_thread=1)
        got = run_or_skip(ctx, workloads.lowcard_plan(), pv.variant(**kw))
        if got is not None:
            assert_same(got, w, ctxmsg=str(kw))


@pytest.mark.parametrize("access", ["grid", "staged"])
def test_lowcard_32bit_fields_with_stale_statistics(ctx, access):
    """The 32-bit-field layout is chosen from the column statistics taken when
    the pipeline is created.  Values written in place afterwards that exceed
    a field's per-row limit (large and negative prices) take the row to the
    global table, still exact; a new pipeline over the changed column reads
    fresh statistics and takes the 64-bit layout."""
    import torch
    n = 400_003
    li = datagen.table_lowcard_groups(n, seed=91)
    dev = {c: torch.from_numpy(np.ascontiguousarray(v)).cuda() for c, v in li.items()}
    ctx.register_table("li", dev)
    plan = workloads.lowcard_plan()
    kw = dict(agg="local", ht="perfect", threads_per_table=1, pred="predicated", access=access, items_per_thread=1)
    res = ctx.run(plan, pv.variant(**kw))
    rng = np.random.default_rng(92)
    pick = rng.random(n) < 0.01
    li["price"] = np.where(pick, rng.integers(-2**33, 2**33, n), li["price"]).astype(np.int64)
    dev["price"].copy_(torch.from_numpy(li["price"]))
    torch.cuda.synchronize()
    ctx.rerun(res)
    w = want(plan, {"li": li})
    got = [c.astype(np.int64) for c in ctx.fetch(res)]
    assert_same(got, w, ordered=False, ctxmsg=f"stale statistics, {access}")
    ctx.free(res)
    ctx.register_table("li", dev)  # fresh handles: fresh statistics
    assert_same(ctx.query(plan, pv.variant(**kw)), w, ctxmsg=f"fresh statistics, {access}")


STAGED = dict(agg="local", ht="perfect", threads_per_table=1, pred="predicated", access="staged",
              items_per_thread=1)


@pytest.mark.parametrize("n", [0, 1, 127, 128, 129, 4096 * 3 + 5, 100_003, 1_000_064])
def test_staged_access_lowcard(ctx, n):
    """TMA-staged chunks of 128 rows (bulk copies into per-warp stages) and the
    plain-loaded partial chunk at the end, with the 32-bit field overflow path
    (a few large values), against the oracle; block sizes change the warps
    per CTA and the chunks per warp."""
    li = datagen.table_lowcard_groups(n, seed=n + 7)
    rng = np.random.default_rng(n)
    pick = rng.random(n) < 0.001
    li["price"] = np.where(pick, rng.integers(2**31, 2**33, n), li["price"]).astype(np.int64)
    t = {"li": li}
    register(ctx, t)
    w = want(workloads.lowcard_plan(), t)
    ran = 0
    for block, gm in ((64, 0), (256, 0), (256, 1), (512, 0)):
        got = run_or_skip(ctx, workloads.lowcard_plan(), pv.variant(**STAGED, block=block, grid_mult=gm))
        if got is not None:
            ran += 1
            assert_same(got, w, ctxmsg=f"staged block {block} grid_mult {gm}")
    assert ran >= 3


@pytest.mark.parametrize("g", [1, 5, 10])
def test_staged_access_keyval(ctx, g):
    kv = {"kv": datagen.table_keyval(300_017, g, "uniform", seed=g + 3)}
    register(ctx, kv)
    for plan in (workloads.keyval_plan(), workloads.keyval_plan(val_lt=300_000)):
        got = ctx.query(plan, pv.variant(**STAGED, block=256))
        assert_same(got, want(plan, kv), ctxmsg=f"staged G={g}")


def test_staged_access_unsupported_forms(ctx):
    li = {"li": datagen.table_lowcard_groups(10_000, seed=3)}
    fa = {"t": datagen.table_filter_agg(10_000, seed=3)}
    register(ctx, li)
    register(ctx, fa)
    plan = workloads.lowcard_plan()
    for kw in (dict(pred="branch"), dict(pred="compacted"), dict(items_per_thread=2), dict(prefetch=1),
               dict(agg="global"), dict(threads_per_table=0), dict(exec="multi")):
        with pytest.raises(pv.PVError) as e:
            ctx.query(plan, pv.variant(**dict(STAGED, **kw)))
        assert e.value.status == -2, kw
    with pytest.raises(pv.PVError) as e:  # not a grouped pipeline
        ctx.query(workloads.filter_agg_plan(), pv.variant(pred="predicated", access="staged", items_per_thread=1))
    assert e.value.status == -2
    ctx.sync()


@pytest.mark.parametrize("g,dist", [(1, "uniform"), (10, "zipf"), (1000, "uniform"), (1000, "zipf"),
                                    (50_000, "uniform")])
def test_keyval_grouped_all_variants(ctx, g, dist):
    kv = {"kv": datagen.table_keyval(120_007, g, dist, seed=g)}
    register(ctx, kv)
    _grouped_all_variants(ctx, workloads.keyval_plan(), kv, step=3, min_ran=20)
    _grouped_all_variants(ctx, workloads.keyval_plan(val_lt=300_000), kv, step=7, min_ran=8)


def test_keyval_negative_and_extreme_keys(ctx):
    rng = np.random.default_rng(5)
    key = rng.choice(np.array([-1, -2, 0, 2**31 - 1, -2**31, 7], np.int32), 10_000)
    kv = {"kv": {"key": key, "val": rng.integers(-10**9, 10**9, 10_000).astype(np.int64)}}
    register(ctx, kv)
    w = want(workloads.keyval_plan(), kv)
    for kw in GROUP_VARIANTS[::5]:
        if kw["ht"] == "perfect":
            continue  # the key domain spans 2^32 values
        got = run_or_skip(ctx, workloads.keyval_plan(), pv.variant(**kw))
        if got is not None:
            assert_same(got, w, ctxmsg=str(kw))


def test_grouped_rerun_is_clean(ctx):
    kv = {"kv": datagen.table_keyval(100_000, 5000, seed=2)}
    register(ctx, kv)
    plan = workloads.keyval_plan()
    w = want(plan, kv)
    for kw in (dict(ht="linear"), dict(ht="cuckoo", exec="multi"), dict(ht="perfect", agg="global")):
        res = ctx.run(plan, pv.variant(**kw))
        for _ in range(3):
            ctx.rerun(res)
        cols = [c.astype(np.int64) for c in ctx.fetch(res)]
        order = np.argsort(cols[0], kind="stable")
        assert_same([c[order] for c in cols], w, ctxmsg=str(kw))
        ctx.free(res)


def test_grouped_table_full_is_reported(ctx):
    kv = {"kv": datagen.table_keyval(50_000, 1000, seed=6)}
    register(ctx, kv)
    plan = dict(workloads.keyval_plan(), capacity_hint=1)
    with pytest.raises(pv.PVError) as e:
        ctx.query(plan, pv.variant(ht="linear", agg="global"))
    assert e.value.status == -3


# ---------------------------------------------------------------- joins
def _star_small(n, seed, lim=None):
    s = datagen.star_schema(n, seed)
    return {"fact": s["fact"], **{d: s[d] for d, _, _ in datagen.STAR_DIMS}}


@pytest.mark.parametrize("build_kind", ["linear", "cuckoo", "perfect"])
@pytest.mark.parametrize("hash_fn", ["murmur", "multshift"])
def test_star_join_all_build_kinds(ctx, build_kind, hash_fn):
    s = _star_small(200_003, seed=31)
    register(ctx, s)
    plan = workloads.star_plan({"d_a": 60, "d_b": 50, "d_c": 30, "d_d": 40})
    w = want(plan, s)
    htv = pv.ht_variant(build_kind, hash_fn)
    ran = 0
    for kw in GROUP_VARIANTS[::6]:
        try:
            got = ctx.query(plan, pv.variant(**kw), htv)
        except pv.PVError as e:
            if e.status == -2:
                continue
            raise
        ran += 1
        assert_same(got, w, ctxmsg=f"{build_kind} {kw}")
    assert ran >= 8


def test_star_join_negative_one_keys_and_payloads(ctx):
    # build key -1 and payloads (-1, -1) exercise both side slots
    d = {}
    for name, rows, g in datagen.STAR_DIMS:
        d[name] = {"key": np.arange(-1, 9, dtype=np.int32), "f": np.zeros(10, np.int32),
                   "g": np.full(10, -1, np.int32)}
        d[name]["g"][5:] = 3
    rng = np.random.default_rng(3)
    fact = {f"fk_{n[2:]}": rng.integers(-2, 10, 20_000).astype(np.int32) for n, _, _ in datagen.STAR_DIMS}
    fact["revenue"] = rng.integers(100, 10**7, 20_000).astype(np.int64)
    tables = {"fact": fact, **d}
    register(ctx, tables)
    plan = workloads.star_plan({k: 100 for k in ("d_a", "d_b", "d_c", "d_d")})
    w = want(plan, tables)
    for kind in ("linear", "cuckoo", "perfect"):
        for kw in (dict(ht="linear"), dict(ht="cuckoo", exec="multi"), dict(ht="perfect"),
                   dict(ht="perfect", agg="global", pred="predicated")):
            got = ctx.query(plan, pv.variant(items_per_thread=1, **kw), pv.ht_variant(kind))
            assert_same(got, w, ctxmsg=f"{kind} {kw}")


@pytest.mark.parametrize("fixture", ["table2_join_group_x.json", "table2_join_group_y.json"])
def test_table2_golden_on_gpu(ctx, fixture):
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", fixture)))
    tables = {t: {c: np.array(v["values"], dtype=v["dtype"]) for c, v in cols.items()} for t, cols in g["tables"].items()}
    register(ctx, tables)
    for kind in ("linear", "cuckoo", "perfect"):
        for kw in (dict(), dict(pred="predicated"), dict(agg="global", ht="perfect")):
            got = ctx.query(g["plan"], pv.variant(items_per_thread=1, **kw), pv.ht_variant(kind))
            assert [list(map(int, c)) for c in got] == g["expected"]["cols"]


@pytest.mark.parametrize("kind", ["linear", "cuckoo", "perfect"])
def test_duplicate_build_key_is_reported(ctx, kind):
    dim = {"key": np.array([1, 2, 3, 2], np.int32)}
    fact = {"fk": np.array([1, 2, 3], np.int32)}
    register(ctx, {"dimdup": dim, "factdup": fact})
    plan = {"fact": "factdup", "builds": [{"table": "dimdup", "key": "key", "payload": []}],
            "probes": [{"build": 0, "fk": "fk"}], "aggs": [["count"]]}
    with pytest.raises(pv.PVError) as e:
        ctx.query(plan, pv.variant(), pv.ht_variant(kind))
    assert e.value.status == -6


def test_join_lattice_count(ctx):
    D, r, thr = 1234, 3, 37
    dim = {"key": np.arange(D, dtype=np.int32), "f": (np.arange(D) % 100).astype(np.int32)}
    fact = {"fk": (np.arange(D * r) % D).astype(np.int32)}
    register(ctx, {"jdim": dim, "jfact": fact})
    plan = {"fact": "jfact", "builds": [{"table": "jdim", "key": "key", "filters": [["f", "lt", thr]], "payload": []}],
            "probes": [{"build": 0, "fk": "fk"}], "aggs": [["count"]]}
    for kind in ("linear", "cuckoo", "perfect"):
        got = ctx.query(plan, pv.variant(), pv.ht_variant(kind))
        assert int(got[0][0]) == r * ((D // 100) * thr + min(D % 100, thr))


# ---------------------------------------------------------------- runtime
def test_shape_without_compiled_kernel_runs_generic(ctx):
    # MAX(b) WHERE a < 3 has no compiled shape: the generic kernels run it; the
    # variant axes they lack (chunked access) are reported, not emulated
    t = {"t": datagen.table_filter_agg(1000, seed=1)}
    register(ctx, t)
    plan = {"fact": "t", "filters": [["a", "lt", 3]], "aggs": [["max", [["x", "b"]]]]}
    assert_same(ctx.query(plan, pv.variant()), want(plan, t))
    with pytest.raises(pv.PVError) as e:
        ctx.query(plan, pv.variant(access="chunked"))
    assert e.value.status == -2


def test_misaligned_column_is_rejected(ctx):
    import ctypes
    import torch
    x = torch.zeros(64, dtype=torch.int32, device="cuda")
    h = ctypes.c_int32()
    st = ctx.lib.pv_register_column(ctx.h, b"t", b"x", 0, ctypes.c_void_p(x.data_ptr() + 4), 10, ctypes.byref(h))
    assert st == -1


def test_watchdog_timeout_then_recovers(ctx):
    lib = ctx.lib
    assert lib.pv_set_timeout_ms(ctx.h, 100) == 0
    assert lib.pv_debug_spin(ctx.h, 1_000_000_000) == 0  # one second of bounded spinning
    assert lib.pv_sync(ctx.h) == -8
    assert lib.pv_set_timeout_ms(ctx.h, 60_000) == 0
    assert lib.pv_sync(ctx.h) == 0


def test_graph_replay_of_reruns(ctx):
    import ctypes
    t = {"t": datagen.table_filter_agg(300_000, seed=12)}
    kv = {"kv": datagen.table_keyval(300_000, 777, seed=13)}
    register(ctx, t)
    register(ctx, kv)
    p1, p2 = workloads.filter_agg_plan(), workloads.keyval_plan()
    r1 = ctx.run(p1, pv.variant())
    r2 = ctx.run(p2, pv.variant(ht="perfect"))
    ctx.sync()
    lib = ctx.lib
    assert lib.pv_l2_flush(ctx.h) == 0
    assert lib.pv_graph_capture_begin(ctx.h) == 0
    for _ in range(4):
        assert lib.pv_l2_flush(ctx.h) == 0
        assert lib.pv_rerun(ctx.h, r1) == 0
        assert lib.pv_rerun(ctx.h, r2) == 0
    g = ctypes.c_int32()
    assert lib.pv_graph_capture_end(ctx.h, ctypes.byref(g)) == 0
    for _ in range(3):
        assert lib.pv_graph_launch(ctx.h, g.value) == 0
    ctx.sync()
    assert_same([c.astype(np.int64) for c in ctx.fetch(r1)], want(p1, t))
    got = [c.astype(np.int64) for c in ctx.fetch(r2)]
    order = np.argsort(got[0])
    assert_same([c[order] for c in got], want(p2, kv))
    ctx.free(g.value)
    ctx.free(r1)
    ctx.free(r2)


def test_cuda_malloc_async_allocator():
    c = pv.Context(0, use_torch_allocator=False)
    t = {"t": datagen.table_filter_agg(10_000, seed=3)}
    register(c, t)
    assert_same(c.query(workloads.filter_agg_plan(), pv.variant()), want(workloads.filter_agg_plan(), t))
    c.close()


def test_rebuild_after_in_place_change_and_in_a_graph(ctx):
    import ctypes
    import torch
    D, r = 1000, 4
    dim = {"key": torch.arange(D, dtype=torch.int32, device="cuda"),
           "f": (torch.arange(D, device="cuda") % 100).to(torch.int32),
           "g": (torch.arange(D, device="cuda") % 7).to(torch.int32)}
    fact = {"fk": (torch.arange(D * r, device="cuda") % D).to(torch.int32),
            "v": torch.ones(D * r, dtype=torch.int64, device="cuda")}
    ctx.register_table("rdim", dim)
    ctx.register_table("rfact", fact)
    plan = {"fact": "rfact", "builds": [{"table": "rdim", "key": "key", "filters": [["f", "lt", 30]], "payload": []}],
            "probes": [{"build": 0, "fk": "fk"}], "aggs": [["count"]]}
    for kind in ("linear", "cuckoo", "perfect"):
        hts = ctx.build_all(plan, pv.ht_variant(kind))
        res = ctx.run(plan, pv.variant(), hts)
        assert int(ctx.fetch(res)[0][0]) == r * 300
        dim["f"].copy_((torch.arange(D, device="cuda") * 7 % 100).to(torch.int32))  # in place
        host = {"rdim": {k: v.cpu().numpy() for k, v in dim.items()},
                "rfact": {k: v.cpu().numpy() for k, v in fact.items()}}
        expect = int(want(plan, host)[0][0])
        ctx.rebuild(hts[0])
        ctx.rerun(res)
        assert int(ctx.fetch(res)[0][0]) == expect
        # the same rebuild + probe recorded as one graph
        dim["f"].copy_((torch.arange(D, device="cuda") % 100).to(torch.int32))
        ctx.sync()
        assert ctx.lib.pv_graph_capture_begin(ctx.h) == 0
        ctx.rebuild(hts[0])
        ctx.rerun(res)
        g = ctypes.c_int32()
        assert ctx.lib.pv_graph_capture_end(ctx.h, ctypes.byref(g)) == 0
        assert ctx.lib.pv_graph_launch(ctx.h, g.value) == 0
        assert int(ctx.fetch(res)[0][0]) == r * 300
        ctx.free(g.value)
        ctx.free(res)
        for h in hts:
            ctx.free(h)


@pytest.mark.parametrize("dim_keys", [
    np.arange(-2**31, -2**31 + 40, dtype=np.int64).astype(np.int32),          # domain at the bottom of int32
    np.arange(-20, 20, dtype=np.int32),                                      # domain straddling zero
    np.arange(2**31 - 40, 2**31, dtype=np.int64).astype(np.int32),           # domain at the top of int32
])
def test_perfect_probe_domain_edges(ctx, dim_keys):
    D = len(dim_keys)
    dim = {"key": dim_keys, "f": (np.arange(D) % 3).astype(np.int32)}
    extremes = np.array([-2**31, -2**31 + 1, 2**31 - 1, 2**31 - 2, 0, -1, 1], dtype=np.int64)
    fk = np.concatenate([extremes, np.asarray(dim_keys, dtype=np.int64)[::3],
                         np.asarray(dim_keys, dtype=np.int64)[:7] - 2**32 + 2**31]).astype(np.int64)
    fk = fk[(fk >= -2**31) & (fk < 2**31)].astype(np.int32)
    fact = {"fk": np.tile(fk, 5)}
    register(ctx, {"edim": dim, "efact": fact})
    plan = {"fact": "efact", "builds": [{"table": "edim", "key": "key", "filters": [["f", "lt", 2]], "payload": []}],
            "probes": [{"build": 0, "fk": "fk"}], "aggs": [["count"]]}
    w = want(plan, {"edim": dim, "efact": fact})
    for kind in ("perfect", "linear", "cuckoo"):
        for pred in ("branch", "predicated"):
            got = ctx.query(plan, pv.variant(pred=pred), pv.ht_variant(kind))
            assert_same(got, w, ctxmsg=f"{kind} {pred}")


def test_int64_build_keys_are_unsupported(ctx):
    dim = {"key": np.arange(2**31 - 5, 2**31 + 5, dtype=np.int64), "f": np.zeros(10, dtype=np.int32)}
    register(ctx, {"i64dim": dim, "i64fact": {"fk": np.arange(10, dtype=np.int32)}})
    plan = {"fact": "i64fact", "builds": [{"table": "i64dim", "key": "key", "filters": [], "payload": []}],
            "probes": [{"build": 0, "fk": "fk"}], "aggs": [["count"]]}
    with pytest.raises(pv.PVError) as e:
        ctx.query(plan, pv.variant(), pv.ht_variant("perfect"))
    assert e.value.status == -2


# ---------------------------------------------------------------- warp pre-aggregation
WARP_AGG_VARIANTS = [dict(kw, warp_agg=1) for kw in GROUP_VARIANTS if kw["threads_per_table"] == 0]


@pytest.mark.parametrize("g,dist", [(1, "uniform"), (7, "zipf"), (1000, "zipf"), (40_000, "uniform")])
def test_warp_preaggregation_keyval(ctx, g, dist):
    kv = {"kv": datagen.table_keyval(90_003, g, dist, seed=100 + g)}
    register(ctx, kv)
    for plan, step in ((workloads.keyval_plan(), 3), (workloads.keyval_plan(val_lt=400_000), 5)):
        w = want(plan, kv)
        ran = 0
        for kw in WARP_AGG_VARIANTS[::step]:
            got = run_or_skip(ctx, plan, pv.variant(**kw))
            if got is None:
                continue
            ran += 1
            assert_same(got, w, ctxmsg=str(kw))
        assert ran >= 8


def test_warp_preaggregation_lowcard(ctx):
    li = {"li": datagen.table_lowcard_groups(50_001, seed=12)}
    register(ctx, li)
    plan = workloads.lowcard_plan()
    w = want(plan, li)
    ran = 0
    for kw in WARP_AGG_VARIANTS[::2]:
        got = run_or_skip(ctx, plan, pv.variant(**kw))
        if got is not None:
            ran += 1
            assert_same(got, w, ctxmsg=str(kw))
    assert ran >= 20


def test_warp_preaggregation_min_max_join(ctx):
    """Table 2's grouped join with SUM, COUNT, MIN and MAX over few groups, so that
    warps hold many rows of one key (MIN/MAX combine as order-preserving codes)."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table2_join_group_y.json")))
    rng = np.random.default_rng(21)
    n1, n2, n3 = 300, 500, 70_001
    t1 = {"a": rng.permutation(n1).astype(np.int32), "x": rng.integers(0, 8, n1).astype(np.int32)}
    t2 = {"b": rng.permutation(n2).astype(np.int32), "y": rng.integers(0, 6, n2).astype(np.int32)}
    t3 = {"c": rng.integers(0, n1, n3).astype(np.int32), "d": rng.integers(0, n2, n3).astype(np.int32),
          "z": rng.integers(0, 5, n3).astype(np.int32), "q": rng.integers(-10**12, 10**12, n3).astype(np.int64)}
    tables = {"T1": t1, "T2": t2, "T3": t3}
    register(ctx, tables)
    w = want(g["plan"], tables)
    assert len(w[0]) >= 3
    for kind in ("linear", "perfect"):
        for kw in (dict(), dict(pred="predicated"), dict(agg="global", ht="perfect"), dict(agg="global"),
                   dict(ht="cuckoo", exec="multi"), dict(agg="local", ht="perfect", pred="predicated")):
            got = ctx.query(g["plan"], pv.variant(items_per_thread=1, warp_agg=1, **kw), pv.ht_variant(kind))
            assert_same(got, w, ctxmsg=f"{kind} {kw}")


# ---------------------------------------------------------------- compacted execution
# items_per_thread: queued rows a lane takes through the row stage at once (1, 2 or 4)
COMPACT_VARIANTS = [dict(agg=a, ht=h, pred="compacted", items_per_thread=u, threads_per_table=tp, warp_agg=wa,
                         block=b, prefetch=pf)
                    for a, h, tp, wa, b, pf, u in itertools.product(["local", "global"], ["linear", "cuckoo", "perfect"],
                                                                    [0, 1], [0, 1], [64, 256, 1024], [0, 1], [1, 2, 4])]


def _compacted(ctx, plan, tables, htv=None, step=1, min_ran=10):
    w = want(plan, tables)
    ran = 0
    for kw in COMPACT_VARIANTS[::step]:
        got = run_or_skip(ctx, plan, pv.variant(**kw), htv)
        if got is None:
            continue
        ran += 1
        assert_same(got, w, ctxmsg=str(kw))
    assert ran >= min_ran
    return ran


def test_compacted_filter_first(ctx):
    li = {"li": datagen.table_lowcard_groups(40_003, seed=13)}
    register(ctx, li)
    _compacted(ctx, workloads.lowcard_plan(day_hi=datagen.DAY0 + 300), li, step=4, min_ran=12)
    for g, dist in ((1000, "zipf"), (50_000, "uniform"), (3, "uniform")):
        kv = {"kv": datagen.table_keyval(70_001, g, dist, seed=40 + g)}
        register(ctx, kv)
        _compacted(ctx, workloads.keyval_plan(val_lt=30_000), kv, step=5, min_ran=8)


@pytest.mark.parametrize("build_kind", ["linear", "cuckoo", "perfect"])
def test_compacted_star_join(ctx, build_kind):
    s = _star_small(150_007, seed=33)
    register(ctx, s)
    for th in ({"d_a": 60, "d_b": 50, "d_c": 30, "d_d": 40}, {"d_a": 20, "d_b": 20, "d_c": 5, "d_d": 10}):
        _compacted(ctx, workloads.star_plan(th), s, pv.ht_variant(build_kind), step=7, min_ran=8)


@pytest.mark.parametrize("build_kind", ["linear", "perfect"])
def test_compacted_two_probe_first_stage(ctx, build_kind):
    """compact_probes = 2: the first two probes run over whole items (both key
    columns read in full) before the survivors are queued; the row stage
    re-probes them only when their payloads are read (the three-probe join's
    group keys), else skips them (the star join's first two dimensions)."""
    s = _star_small(150_007, seed=35)
    register(ctx, s)
    htv = pv.ht_variant(build_kind)
    for th in ({"d_a": 60, "d_b": 50, "d_c": 30, "d_d": 40}, {"d_a": 20, "d_b": 20, "d_c": 5, "d_d": 10}):
        plan = workloads.star_plan(th)
        w = want(plan, s)
        ran = 0
        for kw in COMPACT_VARIANTS[::5]:
            got = run_or_skip(ctx, plan, pv.variant(**kw, compact_probes=2), htv)
            if got is not None:
                ran += 1
                assert_same(got, w, ctxmsg=f"star {th} {kw}")
        assert ran >= 8
    s3 = datagen.star3_schema(120_011, seed=36)
    register(ctx, s3)
    for regions, years in (((2, 2), workloads.STAR3_YEARS), ((0, 4), (1993, 1996))):
        plan = workloads.star3_plan(regions, years)
        w = want(plan, s3)
        for kw in COMPACT_VARIANTS[1::9]:
            got = run_or_skip(ctx, plan, pv.variant(**kw, compact_probes=2), htv)
            if got is not None:
                assert_same(got, w, ctxmsg=f"star3 {regions} {kw}")
    for n in (0, 1, 7, 129):  # empty and ragged fact tables
        sn = _star_small(n, seed=n + 50)
        register(ctx, sn)
        plan = workloads.star_plan({"d_a": 60, "d_b": 50, "d_c": 30, "d_d": 40})
        got = ctx.query(plan, pv.variant(agg="local", ht="perfect", pred="compacted", items_per_thread=2,
                                         compact_probes=2), htv)
        assert_same(got, want(plan, sn), ctxmsg=f"n={n}")


def test_compacted_two_probe_first_stage_unsupported_forms(ctx):
    kv = {"kv": datagen.table_keyval(1000, 10, seed=3)}
    t = {"t": datagen.table_filter_agg(1000)}
    register(ctx, kv)
    register(ctx, t)
    for plan in (workloads.keyval_plan(val_lt=5), workloads.filter_agg_plan(), workloads.filter_project_plan()):
        with pytest.raises(pv.PVError) as e:  # filters first: no probe stage to widen
            ctx.query(plan, pv.variant(pred="compacted", items_per_thread=1, compact_probes=2))
        assert e.value.status == -2
    for kw in (dict(pred="branch", compact_probes=2), dict(pred="compacted", compact_probes=3)):
        with pytest.raises(pv.PVError) as e:
            ctx.query(workloads.keyval_plan(val_lt=5), pv.variant(items_per_thread=1, **kw))
        assert e.value.status == -1
    ctx.sync()


def test_compacted_min_max_join_and_ragged_tables(ctx):
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table2_join_group_y.json")))
    tables = {t: {c: np.array(v["values"], dtype=v["dtype"]) for c, v in cols.items()} for t, cols in g["tables"].items()}
    register(ctx, tables)
    for kind in ("linear", "perfect"):
        for kw in (dict(), dict(agg="global", ht="perfect"), dict(warp_agg=1)):
            got = ctx.query(g["plan"], pv.variant(items_per_thread=1, pred="compacted", **kw), pv.ht_variant(kind))
            assert [list(map(int, c)) for c in got] == g["expected"]["cols"]
    rng = np.random.default_rng(44)
    for n in (0, 1, 5, 1003):
        t3 = {"c": rng.integers(0, 4, n).astype(np.int32), "d": rng.integers(0, 5, n).astype(np.int32),
              "z": rng.integers(0, 5, n).astype(np.int32), "q": rng.integers(-99, 99, n).astype(np.int64)}
        tabs = {"T1": tables["T1"], "T2": tables["T2"], "T3": t3}
        register(ctx, {"T3": t3})
        w = want(g["plan"], tabs)
        for kw in (dict(), dict(agg="global", ht="perfect")):
            got = ctx.query(g["plan"], pv.variant(items_per_thread=1, pred="compacted", **kw), pv.ht_variant("perfect"))
            assert_same(got, w, ctxmsg=f"n={n} {kw}")


@pytest.mark.parametrize("n", [0, 1, 5, 4_097, 200_003])
def test_compacted_two_first_stage_items(ctx, n):
    """first_items = 2: a lane loads two items' filter columns per trip before
    filtering and queueing either.  Ungrouped aggregates, projections (fact
    columns and a probe payload behind a filter), the grouped filter-first
    pipelines (thread-private, CTA-local and global tables, 1, 2 and 4 queued
    rows per lane), empty and ragged tables, against the oracle; probe-first
    pipelines are PV_ERR_UNSUPPORTED and first_items outside compacted mode an
    invalid argument."""
    t = {"t": datagen.table_filter_agg(n, seed=n + 71)}
    register(ctx, t)
    for plan in (workloads.filter_agg_plan(), workloads.filter_agg_plan(a_lt=100, b_lo=0, b_hi=99),
                 workloads.filter_agg_plan(a_lt=0)):
        w = want(plan, t)
        for kw in (dict(items_per_thread=1, block=256), dict(items_per_thread=2, block=512),
                   dict(items_per_thread=2, block=64, grid_mult=1, prefetch=1), dict(items_per_thread=1, block=1024)):
            got = ctx.query(plan, pv.variant(pred="compacted", first_items=2, **kw))
            assert_same(got, w, ctxmsg=f"{plan['filters']} {kw}")
    for plan in (workloads.filter_project_plan(), workloads.filter_project_plan(a_lt=100, b_lo=0, b_hi=99)):
        w = want(plan, t)
        for kw in (dict(items_per_thread=1, block=256), dict(items_per_thread=2, block=512, prefetch=1)):
            got = ctx.query(plan, pv.variant(pred="compacted", exec="single", first_items=2, **kw))
            assert_same(got, w, ordered=False, ctxmsg=f"{plan['filters']} {kw}")
    li = {"li": datagen.table_lowcard_groups(n, seed=n + 72)}
    register(ctx, li)
    plan = workloads.lowcard_plan(day_hi=datagen.DAY0 + 300)
    w = want(plan, li)
    for kw in COMPACT_VARIANTS[::7]:
        got = run_or_skip(ctx, plan, pv.variant(**kw, first_items=2))
        if got is not None:
            assert_same(got, w, ctxmsg=f"lowcard {kw}")
    kv = {"kv": datagen.table_keyval(n, 1000, "zipf", seed=n + 73)}
    register(ctx, kv)
    plan = workloads.keyval_plan(val_lt=30_000)
    w = want(plan, kv)
    for kw in COMPACT_VARIANTS[3::11]:
        got = run_or_skip(ctx, plan, pv.variant(**kw, first_items=2))
        if got is not None:
            assert_same(got, w, ctxmsg=f"keyval {kw}")
    if n:
        s = _star_small(n, seed=n + 74)
        register(ctx, s)
        proj = {"fact": "fact", "filters": [["fk_a", "lt", 1000]],
                "builds": [{"table": "d_b", "key": "key", "filters": [["f", "lt", 40]], "payload": ["g"]}],
                "probes": [{"build": 0, "fk": "fk_b"}], "project": [["payload", 0, 0], "revenue"]}
        for build in ("perfect", "linear"):
            got = ctx.query(proj, pv.variant(pred="compacted", exec="single", items_per_thread=2, first_items=2),
                            pv.ht_variant(build))
            assert_same(got, want(proj, s), ordered=False, ctxmsg=f"filtered join projection {build}")
        with pytest.raises(pv.PVError) as e:  # probe-first: one item per trip only
            ctx.query(workloads.star_plan(), pv.variant(agg="local", ht="perfect", pred="compacted",
                                                        items_per_thread=2, first_items=2))
        assert e.value.status == -2
    for kw in (dict(pred="branch", first_items=2), dict(pred="predicated", first_items=2),
               dict(pred="compacted", first_items=3)):
        with pytest.raises(pv.PVError) as e:
            ctx.query(workloads.filter_agg_plan(), pv.variant(items_per_thread=1, **kw))
        assert e.value.status == -1, kw
    ctx.sync()


def test_l2_fetch_granularity_keeps_results(ctx):
    """pv_set_l2_fetch_bytes changes how much an L2 miss fetches, never what a
    pipeline computes: a join, a compacted projection and the grouped
    benchmark shape at each granularity, against the oracle; the previous
    value comes back and other values are rejected."""
    s = _star_small(100_003, seed=81)
    register(ctx, s)
    t = {"t": datagen.table_filter_agg(100_003, seed=82)}
    register(ctx, t)
    li = {"li": datagen.table_lowcard_groups(100_003, seed=83)}
    register(ctx, li)
    cases = [(workloads.star_plan(), s, pv.variant(agg="local", ht="perfect", pred="compacted", items_per_thread=2,
                                                   block=512), True),
             (workloads.filter_project_plan(), t, pv.variant(pred="compacted", exec="single", items_per_thread=1,
                                                             first_items=2), False),
             (workloads.lowcard_plan(), li, pv.variant(agg="local", ht="perfect", threads_per_table=1,
                                                       pred="predicated", items_per_thread=1), True)]
    wants = [want(plan, tabs) for plan, tabs, _, _ in cases]
    first = ctx.set_l2_fetch_bytes(32)
    try:
        prev = 32
        for nbytes in (64, 128, 32):
            assert ctx.set_l2_fetch_bytes(nbytes) == prev
            prev = nbytes
            for (plan, _, var, ordered), w in zip(cases, wants):
                got = ctx.query(plan, var, pv.ht_variant("perfect"))
                assert_same(got, w, ordered=ordered, ctxmsg=f"l2 fetch {nbytes}: {plan.get('fact')}")
        for bad in (0, 16, 256, -1):
            with pytest.raises(pv.PVError) as e:
                ctx.set_l2_fetch_bytes(bad)
            assert e.value.status == -1
    finally:
        ctx.set_l2_fetch_bytes(first if first in (32, 64, 128) else 64)


def test_compacted_is_unsupported_where_it_does_not_apply(ctx):
    kv = {"kv": datagen.table_keyval(1000, 10, seed=3)}
    register(ctx, kv)
    for plan, kw in ((workloads.keyval_plan(), dict()),                             # nothing to compact on
                     (workloads.keyval_plan(val_lt=5), dict(exec="multi")),         # key pass
                     (workloads.keyval_plan(val_lt=5), dict(access="chunked"))):
        with pytest.raises(pv.PVError) as e:
            ctx.query(plan, pv.variant(pred="compacted", **kw))
        assert e.value.status == -2
    t = {"t": datagen.table_filter_agg(1000)}
    register(ctx, t)
    with pytest.raises(pv.PVError) as e:  # compacted projections are single pass: queues reorder the rows
        ctx.query(workloads.filter_project_plan(), pv.variant(pred="compacted", exec="multi", items_per_thread=1))
    assert e.value.status == -2


@pytest.mark.parametrize("n", [0, 1, 5, 4097, 200_003])
def test_compacted_ungrouped_aggregates(ctx, n):
    t = {"t": datagen.table_filter_agg(n, seed=n + 3)}
    register(ctx, t)
    for plan in (workloads.filter_agg_plan(), workloads.filter_agg_plan(a_lt=100, b_lo=0, b_hi=99),
                 workloads.filter_agg_plan(a_lt=0)):
        w = want(plan, t)
        for kw in (dict(block=64), dict(block=256, prefetch=1), dict(block=1024, grid_mult=1),
                   dict(block=256, items_per_thread=2), dict(block=64, items_per_thread=2, grid_mult=1)):
            kw = dict(dict(items_per_thread=1), **kw)
            got = ctx.query(plan, pv.variant(pred="compacted", **kw))
            assert_same(got, w, ctxmsg=f"{plan['filters']} {kw}")
    kv = {"kv": datagen.table_keyval(n, 50, seed=n + 4)}
    register(ctx, kv)
    plan = {"fact": "kv", "filters": [["val", "lt", 300_000]],
            "aggs": [["sum", [["x", "val"]]], ["count"], ["min", [["x", "val"]]], ["max", [["x", "val"]]]]}
    w = want(plan, kv)
    got = ctx.query(plan, pv.variant(pred="compacted", items_per_thread=1))
    if n:
        assert_same(got, w, ctxmsg="keyval totals")
    else:
        assert int(got[1][0]) == 0 and int(got[0][0]) == 0
    li = {"li": datagen.table_lowcard_groups(n, seed=n + 5)}
    register(ctx, li)
    plan = dict(workloads.lowcard_plan(), group_by=[])
    w = want(plan, li)
    assert_same(ctx.query(plan, pv.variant(pred="compacted", items_per_thread=1)), w, ctxmsg="lowcard totals")


def test_compacted_join_count(ctx):
    D, r, thr = 1234, 3, 37
    dim = {"key": np.arange(D, dtype=np.int32), "f": (np.arange(D) % 100).astype(np.int32)}
    fact = {"fk": (np.arange(D * r) % D).astype(np.int32)}
    register(ctx, {"cjdim": dim, "cjfact": fact})
    plan = {"fact": "cjfact", "builds": [{"table": "cjdim", "key": "key", "filters": [["f", "lt", thr]], "payload": []}],
            "probes": [{"build": 0, "fk": "fk"}], "aggs": [["count"]]}
    for kind in ("linear", "cuckoo", "perfect"):
        got = ctx.query(plan, pv.variant(pred="compacted", items_per_thread=1), pv.ht_variant(kind))
        assert int(got[0][0]) == r * ((D // 100) * thr + min(D % 100, thr))


# ---------------------------------------------------------------- join + project
PROJ_VARIANTS = [dict(exec=e, pred=p, access=a, items_per_thread=u, block=b)
                 for e, p, a, u, b in itertools.product(["single", "multi"], ["branch", "predicated"],
                                                        ["grid", "chunked"], [1, 2, 4], [64, 256])]


@pytest.mark.parametrize("n", [0, 7, 4096, 90_003])
def test_join_project_payloads(ctx, n):
    """PROJECT of a probe's payload beside a fact column, with and without a
    fact filter in front: single pass as a multiset, multi pass in input order."""
    rng = np.random.default_rng(70 + n)
    D = 5000
    dim = {"key": rng.permutation(D).astype(np.int32), "f": rng.integers(0, 100, D).astype(np.int32),
           "g": rng.integers(-1000, 1000, D).astype(np.int32)}
    fact = {"fk": rng.integers(-10, D + 10, n).astype(np.int32), "z": rng.integers(0, 10, n).astype(np.int32),
            "rev": rng.integers(-10**12, 10**12, n).astype(np.int64)}
    register(ctx, {"jpdim": dim, "jpfact": fact})
    build = [{"table": "jpdim", "key": "key", "filters": [["f", "lt", 30]], "payload": ["g"]}]
    plans = [{"fact": "jpfact", "builds": build, "probes": [{"build": 0, "fk": "fk"}],
              "project": [["payload", 0, 0], "rev"]},
             {"fact": "jpfact", "builds": build, "filters": [["z", "lt", 4]], "probes": [{"build": 0, "fk": "fk"}],
              "project": [["payload", 0, 0], "rev"]}]
    tables = {"jpdim": dim, "jpfact": fact}
    for plan in plans:
        w = want(plan, tables)
        for kind in ("perfect", "linear", "cuckoo"):
            ran = 0
            for kw in PROJ_VARIANTS[::3]:
                got = run_or_skip(ctx, plan, pv.variant(**kw), pv.ht_variant(kind))
                if got is None:
                    continue
                ran += 1
                assert_same(got, w, ordered=kw["exec"] == "multi", ctxmsg=f"{kind} {kw}")
            assert ran >= 6
        # result column types: the payload column is int32, the fact column keeps int64
        hts = ctx.build_all(plan, pv.ht_variant("perfect"))
        res = ctx.run(plan, pv.variant(), hts)
        raw = ctx.fetch(res)
        assert raw[0].dtype == np.int32 and raw[1].dtype == np.int64
        ctx.free(res)
        for h in hts:
            ctx.free(h)


# ---------------------------------------------------------------- cluster (distributed shared memory) tables
CLUSTER_VARIANTS = [dict(agg="cluster", ht="perfect", pred=p, access=a, items_per_thread=1, block=b, warp_agg=wa,
                         grid_mult=gm)
                    for p, a, b, wa, gm in itertools.product(["branch", "predicated"], ["grid", "chunked"],
                                                             [128, 512], [0, 1], [0, 1])]


def _cluster(ctx, plan, tables, htv=None, step=1, min_ran=8):
    w = want(plan, tables)
    ran = 0
    for kw in CLUSTER_VARIANTS[::step]:
        got = run_or_skip(ctx, plan, pv.variant(**kw), htv)
        if got is None:
            continue
        ran += 1
        assert_same(got, w, ctxmsg=str(kw))
    assert ran >= min_ran


@pytest.mark.parametrize("g,dist", [(1, "uniform"), (1000, "zipf"), (30_000, "uniform"), (60_000, "zipf")])
def test_cluster_tables_keyval(ctx, g, dist):
    kv = {"kv": datagen.table_keyval(150_007, g, dist, seed=200 + g)}
    register(ctx, kv)
    _cluster(ctx, workloads.keyval_plan(), kv, step=2)
    _cluster(ctx, workloads.keyval_plan(val_lt=200_000), kv, step=5, min_ran=4)


def test_cluster_tables_lowcard_star_and_min_max(ctx):
    li = {"li": datagen.table_lowcard_groups(30_001, seed=14)}
    register(ctx, li)
    _cluster(ctx, workloads.lowcard_plan(), li, step=3, min_ran=5)
    s = _star_small(80_001, seed=35)
    register(ctx, s)
    _cluster(ctx, workloads.star_plan({"d_a": 60, "d_b": 50, "d_c": 30, "d_d": 40}), s, pv.ht_variant("perfect"),
             step=3, min_ran=5)
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table2_join_group_y.json")))
    rng = np.random.default_rng(23)
    n1, n2, n3 = 300, 500, 40_001
    tables = {"T1": {"a": rng.permutation(n1).astype(np.int32), "x": rng.integers(0, 8, n1).astype(np.int32)},
              "T2": {"b": rng.permutation(n2).astype(np.int32), "y": rng.integers(0, 600, n2).astype(np.int32)},
              "T3": {"c": rng.integers(0, n1, n3).astype(np.int32), "d": rng.integers(0, n2, n3).astype(np.int32),
                     "z": rng.integers(0, 5, n3).astype(np.int32),
                     "q": rng.integers(-10**12, 10**12, n3).astype(np.int64)}}
    register(ctx, tables)
    _cluster(ctx, g["plan"], tables, pv.ht_variant("perfect"), step=4, min_ran=3)


def test_cluster_tables_unsupported_cases(ctx):
    kv = {"kv": datagen.table_keyval(10_000, 100, seed=9)}
    register(ctx, kv)
    plan = workloads.keyval_plan()
    for kw in (dict(ht="linear"), dict(ht="cuckoo", exec="multi"), dict(exec="multi"), dict(threads_per_table=1),
               dict(pred="compacted"), dict(items_per_thread=2)):
        with pytest.raises(pv.PVError) as e:
            ctx.query(plan, pv.variant(**dict(dict(agg="cluster", ht="perfect", items_per_thread=1), **kw)))
        assert e.value.status == -2, kw
    big = {"kv": {"key": np.array([0, 10_000_000], np.int32), "val": np.array([1, 2], np.int64)}}
    register(ctx, big)  # a 1e7-slot domain does not fit the shared memory of a cluster
    with pytest.raises(pv.PVError) as e:
        ctx.query(plan, pv.variant(agg="cluster", ht="perfect", items_per_thread=1))
    assert e.value.status == -2


# ---------------------------------------------------------------- three-part group keys
@pytest.mark.parametrize("n,spans,lows", [(0, (16, 64, 7), (0, 0, 1992)), (5, (16, 64, 7), (0, 0, 1992)),
                                          (100_003, (16, 64, 7), (0, 0, 1992)), (60_001, (3, 1, 2), (-7, 5, 0))])
def test_three_part_keys_all_variants(ctx, n, spans, lows):
    k3 = {"k3": datagen.table_keys3(n, spans, lows, seed=n + 3)}
    register(ctx, k3)
    plan = workloads.keys3_plan()
    _grouped_all_variants(ctx, plan, k3, step=3, min_ran=20)
    _cluster(ctx, plan, k3, step=3, min_ran=8)
    for kw in (dict(warp_agg=1, agg="global", ht="perfect", items_per_thread=1),
               dict(warp_agg=1, agg="global", ht="linear", items_per_thread=1),
               dict(agg="local", ht="perfect", items_per_thread=1, block=1024, prefetch=1)):
        assert_same(ctx.query(plan, pv.variant(**kw)), want(plan, k3), ctxmsg=str(kw))


def test_three_part_keys_wide_domain(ctx):
    # 5000^3 = 1.25e11 codes: past 2^32 (64-bit codes in the hash tables),
    # below the 2^40 bound; a perfect array (at most 2^28 slots) is refused
    k3 = {"k3": datagen.table_keys3(80_001, (5000, 5000, 5000), (-2500, 0, 7), seed=5)}
    register(ctx, k3)
    plan = workloads.keys3_plan()
    _grouped_all_variants(ctx, plan, k3, step=5, min_ran=8)
    with pytest.raises(pv.PVError) as e:
        ctx.query(plan, pv.variant(agg="global", ht="perfect", items_per_thread=1))
    assert e.value.status == -2
    # 20001^3 > 2^40 codes: no table kind takes the key
    big = {"k3": {"a": np.array([0, 20_000], np.int32), "b": np.array([0, 20_000], np.int32),
                  "c": np.array([0, 20_000], np.int32), "val": np.array([1, 2], np.int64)}}
    register(ctx, big)
    for kw in (dict(ht="linear"), dict(ht="cuckoo", exec="multi"), dict(ht="perfect", agg="global")):
        with pytest.raises(pv.PVError) as e:
            ctx.query(plan, pv.variant(items_per_thread=1, **kw))
        assert e.value.status == -2, kw


@pytest.mark.parametrize("build_kind", ["linear", "cuckoo", "perfect"])
def test_star3_groups_on_three_payloads(ctx, build_kind):
    s = datagen.star3_schema(150_007, seed=37)
    register(ctx, s)
    htv = pv.ht_variant(build_kind)
    for plan in (workloads.star3_plan(), workloads.star3_plan(regions=(0, 4), years=(1992, 1998))):
        w = want(plan, s)
        assert len(w[0]) > 100
        ran = 0
        for kw in GROUP_VARIANTS[::5]:
            got = run_or_skip(ctx, plan, pv.variant(**kw), htv)
            if got is None:
                continue
            ran += 1
            assert_same(got, w, ctxmsg=f"{build_kind} {kw}")
        assert ran >= 10
        _compacted(ctx, plan, s, htv, step=5, min_ran=10)
        _cluster(ctx, plan, s, htv, step=4, min_ran=6)


# ---------------------------------------------------------------- dictionary-coded strings
def _register_parts(ctx, n, seed):
    from tests.gpu_util import to_device
    codes = datagen.table_parts(n, seed=seed)
    cats, brands = datagen.part_categories(), datagen.part_brands()
    ctx.register_table("parts", to_device({"parts": codes})["parts"], dicts={"category": cats, "brand": brands})
    return {"parts": {"category": datagen.as_text(codes["category"], cats),
                      "brand": datagen.as_text(codes["brand"], brands), "price": codes["price"]}}


# one code range per column (the filter/aggregate shape)
STRING_RANGE_FILTERS = [
    (("category", "eq", "MFGR#12"), ("brand", "between", "MFGR#1221", "MFGR#1228")),
    (("category", "ge", "MFGR#3"), ("brand", "prefix", "MFGR#3")),
    (("category", "lt", "MFGR#2"), ("brand", "like", "MFGR#1%")),
    (("category", "in", ["MFGR#21", "MFGR#22", "MFGR#23"]), ("brand", "gt", "MFGR#2150")),
    (("category", "eq", "MFGR#99"), ("brand", "le", "MFGR#5540")),
]


@pytest.mark.parametrize("n", [0, 5, 100_003])
def test_string_range_predicates(ctx, n):
    text = _register_parts(ctx, n, seed=n + 7)
    for filters in STRING_RANGE_FILTERS:
        plan = workloads.parts_text_plan(filters)
        w = want(plan, text)
        ran = 0
        for kw in SCAN_VARIANTS[::9]:
            got = run_or_skip(ctx, plan, pv.variant(**kw))
            if got is None:
                continue
            ran += 1
            assert_same(got, w, ctxmsg=f"{filters} {kw}")
        assert ran >= 3


@pytest.mark.parametrize("kind", ["linear", "cuckoo", "perfect"])
def test_string_like_and_in_as_semi_joins(ctx, kind):
    text = _register_parts(ctx, 90_001, seed=17)
    for f in (["brand", "like", "MFGR#_2_5"], ["brand", "like", "%9"],
              ["brand", "in", ["MFGR#1101", "MFGR#3340", "MFGR#5540", "nope"]]):
        plan = {"fact": "parts", "filters": [f], "aggs": [["count"]]}
        w = want(plan, text)
        assert int(w[0][0]) > 0
        assert_same(ctx.query(plan, pv.variant(), pv.ht_variant(kind)), w, ctxmsg=f"{kind} {f}")


def test_star3_region_filters_as_strings(ctx):
    from tests.gpu_util import to_device
    s = datagen.star3_schema(120_001, seed=39)
    text = {t: dict(c) for t, c in s.items()}
    for t, cols in to_device(s).items():
        dicts = {"region": datagen.SSB_REGIONS} if t in ("d_cust", "d_supp") else None
        ctx.register_table(t, cols, dicts=dicts)
        if dicts:
            text[t]["region"] = datagen.as_text(s[t]["region"], datagen.SSB_REGIONS)
    for regions in (("ASIA", "ASIA"), ("AFRICA", "MIDDLE EAST")):
        plan = workloads.star3_plan(regions=regions)
        w = want(plan, text)
        assert len(w[0]) > 100
        for kind, kw in (("perfect", dict(agg="global", ht="perfect", pred="compacted", items_per_thread=1, block=512)),
                         ("linear", dict(agg="local", ht="perfect", pred="branch", items_per_thread=1, block=512))):
            assert_same(ctx.query(plan, pv.variant(**kw), pv.ht_variant(kind)), w, ctxmsg=f"{regions} {kind} {kw}")


# ---------------------------------------------------------------- HASH_PROBE order
def test_probe_orders_of_the_star_join(ctx):
    s = _star_small(120_001, seed=41)
    register(ctx, s)
    plan = workloads.star_plan({"d_a": 60, "d_b": 50, "d_c": 30, "d_d": 40})
    w = want(plan, s)
    # the orders that keep the compiled shape: either pair of probes swapped (pv.reorder_probes)
    for order in ((0, 1, 2, 3), (1, 0, 2, 3), (0, 1, 3, 2), (1, 0, 3, 2)):
        for kind, kw in (("perfect", dict(agg="global", ht="perfect", pred="compacted", items_per_thread=1, block=512)),
                         ("linear", dict(agg="local", ht="perfect", pred="branch", items_per_thread=1, block=512))):
            got = ctx.query(plan, pv.variant(**kw), pv.ht_variant(kind), probe_order=order)
            assert_same(got, w, ctxmsg=f"{order} {kind} {kw}")
    # a grouping dimension probed first: no compiled shape, the generic kernels run it
    got = ctx.query(plan, pv.variant(agg="global", ht="perfect", items_per_thread=1), pv.ht_variant("perfect"),
                    probe_order=(2, 0, 1, 3))
    assert_same(got, w, ctxmsg="generic (2, 0, 1, 3)")


# ---------------------------------------------------------------- byte-coded perfect tables
def test_byte_coded_perfect_tables(ctx):
    """A perfect build table whose one payload spans at most 255 values is
    probed through one byte per key; a wider payload keeps the 8-byte slots.
    Both against the oracle, for grouping on the payload and projecting it;
    a rebuild after an in-place change within the recorded payload range
    stays exact, one outside it is reported (the statistics are out of date)."""
    import torch
    D, n = 5000, 200_003
    rng = np.random.default_rng(31)
    key = torch.from_numpy(rng.permutation(D).astype(np.int32)).cuda()
    dim = {"key": key, "f": (key % 10).to(torch.int32), "narrow": (key % 40 + 5).to(torch.int32),
           "wide": (key * 3 - 7000).to(torch.int32)}
    fact = {"fk": torch.from_numpy(rng.integers(-50, D + 50, n).astype(np.int32)).cuda(),
            "v": torch.from_numpy(rng.integers(0, 1000, n).astype(np.int64)).cuda()}
    ctx.register_table("bdim", dim)
    ctx.register_table("bfact", fact)

    def host():
        return {"bdim": {k: v.cpu().numpy() for k, v in dim.items()},
                "bfact": {k: v.cpu().numpy() for k, v in fact.items()}}

    for pay in ("narrow", "wide"):
        build = {"table": "bdim", "key": "key", "filters": [["f", "lt", 7]], "payload": [pay]}
        grouped = {"fact": "bfact", "builds": [build], "probes": [{"build": 0, "fk": "fk"}],
                   "group_by": [["payload", 0, 0]], "aggs": [["sum", [["x", "v"]]], ["count"]]}
        proj = {"fact": "bfact", "builds": [build], "probes": [{"build": 0, "fk": "fk"}],
                "project": [["payload", 0, 0], "v"]}
        for plan, kws in ((grouped, [dict(agg="global", ht="perfect", items_per_thread=1),
                                     dict(agg="local", ht="linear", pred="predicated", items_per_thread=1),
                                     dict(agg="global", ht="linear", pred="predicated", items_per_thread=1)]),
                          (proj, [dict(exec="multi"), dict(exec="single", interp=1)])):
            w = want(plan, host())
            for kw in kws:
                got = ctx.query(plan, pv.variant(**kw), pv.ht_variant("perfect"))
                assert_same(got, w, ordered=plan is grouped or kw.get("exec") == "multi", ctxmsg=f"{pay} {kw}")
    # rebuilds of a byte-coded table
    build = {"table": "bdim", "key": "key", "filters": [["f", "lt", 7]], "payload": ["narrow"]}
    plan = {"fact": "bfact", "builds": [build], "probes": [{"build": 0, "fk": "fk"}],
            "group_by": [["payload", 0, 0]], "aggs": [["sum", [["x", "v"]]], ["count"]]}
    hts = ctx.build_all(plan, pv.ht_variant("perfect"))
    res = ctx.run(plan, pv.variant(agg="global", ht="perfect", items_per_thread=1), hts)
    ctx.sync()
    dim["narrow"].copy_(46 - dim["narrow"])  # the surviving rows' payloads stay within [5, 41]
    ctx.rebuild(hts[0])
    ctx.rerun(res)
    got = ctx.fetch(res)
    order = np.argsort(got[0])
    assert_same([c[order] for c in got], want(plan, host()), ctxmsg="rebuilt")
    dim["narrow"].copy_((key % 300).to(torch.int32))  # outside the first build's payload range
    ctx.rebuild(hts[0])
    with pytest.raises(pv.PVError) as e:
        ctx.sync()
    assert e.value.status == -5
    ctx.free(res)
    ctx.free(hts[0])



@pytest.mark.parametrize("n", [0, 5, 4_099, 300_007])
def test_compacted_projections(ctx, n):
    """Single-pass PROJECT in compacted mode: the first operation's survivors
    queued per warp, one or two per lane, surviving rows staged per warp in
    shared memory and written out 64 or more at a time.
    Filter-first and probe-first plans, projecting fact columns and probe
    payloads, against the oracle as multisets; an output too small is
    reported."""
    t = {"t": datagen.table_filter_agg(n, seed=n + 41)}
    register(ctx, t)
    for plan in (workloads.filter_project_plan(), workloads.filter_project_plan(a_lt=100, b_lo=0, b_hi=99),
                 {"fact": "t", "filters": [["a", "lt", 30]], "project": ["b", "price"]}):
        w = want(plan, t)
        for kw in (dict(items_per_thread=1, block=256), dict(items_per_thread=2, block=512, prefetch=1),
                   dict(items_per_thread=2, block=64, grid_mult=1), dict(items_per_thread=2, block=1024)):
            got = ctx.query(plan, pv.variant(pred="compacted", exec="single", **kw))
            assert_same(got, w, ordered=False, ctxmsg=f"{plan['filters']} {kw}")
    if n:
        s = _star_small(n, seed=n + 42)
        for plan in ({"fact": "fact", "builds": [{"table": "d_b", "key": "key", "filters": [["f", "lt", 40]],
                                                   "payload": ["g"]}],
                      "probes": [{"build": 0, "fk": "fk_b"}], "project": [["payload", 0, 0], "revenue"]},
                     {"fact": "fact", "filters": [["fk_a", "lt", 1000]],
                      "builds": [{"table": "d_b", "key": "key", "filters": [["f", "lt", 40]], "payload": ["g"]}],
                      "probes": [{"build": 0, "fk": "fk_b"}], "project": [["payload", 0, 0], "revenue"]}):
            register(ctx, s)
            w = want(plan, s)
            for build in ("perfect", "linear"):
                for u in (1, 2):
                    got = ctx.query(plan, pv.variant(pred="compacted", exec="single", items_per_thread=u),
                                    pv.ht_variant(build))
                    assert_same(got, w, ordered=False, ctxmsg=f"{build} u={u} {plan}")
        plan = dict(workloads.filter_project_plan(a_lt=100, b_lo=0, b_hi=99), capacity_hint=max(1, n // 3))
        with pytest.raises(pv.PVError) as e:
            ctx.query(plan, pv.variant(pred="compacted", exec="single", items_per_thread=1))
        assert e.value.status == -7
