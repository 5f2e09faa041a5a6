"""Enqueued result fetches (pv_enqueue_fetch, pv_enqueue_fetch_rows) vs the oracle.

pv_enqueue_fetch copies a result's full capacity with copy-engine copies;
pv_enqueue_fetch_rows copies only its live rows with one kernel, into device
memory or page-locked host memory.  Both are checked against the oracle for
ungrouped, projected and grouped results, in page-locked host and device
destinations, and the live-row fetch also inside a CUDA graph.  The live-row
fetch must leave every destination row past the live rows untouched (only
those rows cross to the host), and must refuse pageable host memory.
"""
import ctypes

import numpy as np
import pytest

from paper_1709_00700_gb300 import datagen, pv, workloads
from tests.gpu_util import assert_same, register, want

pytestmark = pytest.mark.gpu

SENTINEL = {np.dtype(np.int32): -0x5A5A5A5A, np.dtype(np.int64): -0x5A5A5A5A5A5A5A5A, np.dtype(np.uint8): 0xA5}


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    c = pv.Context(0)
    yield c
    c.close()


def _cases():
    fa = {"t": datagen.table_filter_agg(100_003, seed=31)}
    kv = {"kv": datagen.table_keyval(70_001, 1000, "uniform", seed=32)}
    return [
        ("aggregate", fa, workloads.filter_agg_plan(), pv.variant(), True),
        ("project multi", fa, workloads.filter_project_plan(), pv.variant(exec="multi"), True),
        ("project single", fa, workloads.filter_project_plan(), pv.variant(exec="single"), False),
        ("grouped", kv, workloads.keyval_plan(), pv.variant(agg="global", ht="linear"), False),
    ]


def _buffers(ctx, res, device):
    import torch
    cols, count = ctx.fetch_buffers(res)
    if device:
        cols = [c.cuda() for c in cols]
        count = count.cuda()
    for c in cols:
        c.fill_(SENTINEL[np.dtype(str(c.dtype).replace("torch.", ""))])
    count.fill_(-1)
    torch.cuda.synchronize()
    return cols, count


def _read(bufs):
    cols, count = bufs
    n = int(count.cpu().item())
    return n, [c.cpu().numpy() for c in cols]


@pytest.mark.parametrize("device", [False, True], ids=["pinned", "device"])
@pytest.mark.parametrize("live_rows", [False, True], ids=["capacity", "live_rows"])
def test_enqueued_fetch_matches_oracle(ctx, device, live_rows):
    for name, tables, plan, var, ordered in _cases():
        register(ctx, tables)
        res = ctx.run(plan, var)
        w = want(plan, tables)
        bufs = _buffers(ctx, res, device)
        ctx.enqueue_fetch(res, bufs, live_rows=live_rows)
        ctx.sync()
        n, cols = _read(bufs)
        assert n == len(w[0]), f"{name}: {n} rows, oracle {len(w[0])}"
        assert_same([c[:n] for c in cols], w, ordered=ordered, ctxmsg=name)
        if live_rows:  # nothing written past the live rows
            for c in cols:
                assert np.all(c[n:] == SENTINEL[c.dtype]), f"{name}: rows past the live rows were written"
        ctx.free(res)


def test_live_row_fetch_in_a_graph(ctx):
    import torch
    t = {"t": datagen.table_filter_agg(200_001, seed=33)}
    register(ctx, t)
    plan = workloads.filter_project_plan()
    res = ctx.run(plan, pv.variant(exec="multi"))
    bufs = _buffers(ctx, res, device=False)
    lib = ctx.lib
    assert lib.pv_graph_capture_begin(ctx.h) == 0
    try:
        ctx.rerun(res)
        ctx.enqueue_fetch(res, bufs, live_rows=True)
    finally:
        g = ctypes.c_int32()
        assert lib.pv_graph_capture_end(ctx.h, ctypes.byref(g)) == 0
    w = want(plan, t)
    for _ in range(2):
        bufs[1].fill_(-1)
        torch.cuda.synchronize()
        assert lib.pv_graph_launch(ctx.h, g.value) == 0
        ctx.sync()
        n, cols = _read(bufs)
        assert_same([c[:n] for c in cols], w, ordered=True, ctxmsg="graph replay")
    ctx.free(g.value)
    ctx.free(res)


def test_live_row_fetch_refuses_pageable_memory(ctx):
    t = {"t": datagen.table_filter_agg(1000, seed=34)}
    register(ctx, t)
    res = ctx.run(workloads.filter_agg_plan(), pv.variant())
    cols, count = ctx.fetch_buffers(res)
    pageable = [np.zeros(c.numel(), dtype=np.int64) for c in cols]
    ptrs = (ctypes.c_void_p * len(cols))(*[a.ctypes.data for a in pageable])
    rows = (ctypes.c_int64 * len(cols))(*[len(a) for a in pageable])
    st = ctx.lib.pv_enqueue_fetch_rows(ctx.h, res, len(cols), ptrs, rows, ctypes.c_void_p(count.data_ptr()))
    assert st == -1
    ctx.sync()
    ctx.free(res)


def test_fetch_refuses_memory_of_the_other_kind(ctx):
    """Device memory passed as a host destination (or the reverse) is refused
    before any copy is issued."""
    import torch
    t = {"t": datagen.table_filter_agg(1000, seed=35)}
    register(ctx, t)
    res = ctx.run(workloads.filter_project_plan(), pv.variant(exec="multi"))
    cols, count = ctx.fetch_buffers(res)
    for on_device, bufs in ((0, ([c.cuda() for c in cols], count.cuda())), (1, (cols, count))):
        dst, cnt = bufs
        ptrs = (ctypes.c_void_p * len(dst))(*[a.data_ptr() for a in dst])
        rows = (ctypes.c_int64 * len(dst))(*[a.numel() for a in dst])
        st = ctx.lib.pv_enqueue_fetch(ctx.h, res, len(dst), ptrs, rows, ctypes.c_void_p(cnt.data_ptr()), on_device)
        assert st == -1, on_device
        st = ctx.lib.pv_fetch_results(ctx.h, res, len(dst), ptrs, rows, on_device)
        assert st == -1, on_device
    torch.cuda.synchronize()
    ctx.sync()
    ctx.free(res)
