"""The allocation-free projection entry point, through the C ABI.

pv_filter_project_noalloc serves callers that cannot allocate device memory
(their device memory belongs to another allocator, or they cannot pay for
cudaMalloc's synchronisation): its scratch is a static device array.  Its
output must equal the multi-pass projection of pv_run_pipeline exactly, and
the oracle's rows in input order, on consecutive calls that reuse the one
scratch array; with too small an output it reports the overflow and keeps
the first rows that fit.  This file is collected last so that a failure here
leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

from oracle import oracle
from paper_1709_00700_gb300 import datagen, pv, workloads

pytestmark = pytest.mark.gpu


def _noalloc(lib, dev, n, bounds, capacity, stream):
    import torch
    out_a = torch.empty(max(capacity, 1), dtype=torch.int32, device="cuda")
    out_p = torch.empty(max(capacity, 1), dtype=torch.int64, device="cuda")
    count = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    status = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    a_lo, a_hi, b_lo, b_hi = bounds
    st = lib.pv_filter_project_noalloc(ctypes.c_void_p(dev["a"].data_ptr()), ctypes.c_void_p(dev["b"].data_ptr()),
                                       ctypes.c_void_p(dev["price"].data_ptr()), n, a_lo, a_hi, b_lo, b_hi,
                                       ctypes.c_void_p(out_a.data_ptr()), ctypes.c_void_p(out_p.data_ptr()),
                                       capacity, ctypes.c_void_p(count.data_ptr()),
                                       ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert st == 0
    stream.synchronize()
    k = int(count.item())
    return int(status.item()), [out_a[:k].cpu().numpy(), out_p[:k].cpu().numpy()]


def test_noalloc_matches_multi_pass_projection_on_consecutive_calls():
    import torch
    n = 300_003
    t = datagen.table_filter_agg(n, seed=77)
    dev = {c: torch.from_numpy(v).cuda() for c, v in t.items()}
    lib = pv.load()
    ctx = pv.Context(0)
    ctx.register_table("t", dev)
    stream = torch.cuda.current_stream()
    # (a < 10 AND 20 <= b <= 40), then (3 <= a <= 60 AND b <= 7): two calls in a row
    for a_lt, (b_lo, b_hi) in ((10, (20, 40)), (None, (-5, 7))):
        if a_lt is not None:
            plan = workloads.filter_project_plan(a_lt, b_lo, b_hi)
            bounds = (-2**63, a_lt - 1, b_lo, b_hi)
        else:
            plan = {"fact": "t", "filters": [["a", "between", 3, 60], ["b", "between", b_lo, b_hi]],
                    "project": ["a", "price"]}
            bounds = (3, 60, b_lo, b_hi)
        res = ctx.run(plan, pv.variant(exec="multi", items_per_thread=4, block=256))
        want = ctx.fetch(res)
        ctx.free(res)
        status, got = _noalloc(lib, dev, n, bounds, n, stream)
        assert status == 0
        assert got[0].dtype == np.int32 and got[1].dtype == np.int64
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
        assert len(want[0]) > 0
        exact = oracle.run(plan, {"t": t})["cols"]  # input order
        assert np.array_equal(got[0].astype(np.int64), exact[0]) and np.array_equal(got[1], exact[1])
    ctx.close()


def test_noalloc_reports_overflow_and_keeps_the_first_rows():
    import torch
    n = 200_001
    t = datagen.table_filter_agg(n, seed=78)
    dev = {c: torch.from_numpy(v).cuda() for c, v in t.items()}
    lib = pv.load()
    stream = torch.cuda.current_stream()
    plan = workloads.filter_project_plan(10, 20, 40)
    exact = oracle.run(plan, {"t": t})["cols"]
    matches = len(exact[0])
    assert matches > 100
    for cap in (matches // 2, 0, matches):
        status, got = _noalloc(lib, dev, n, (-2**63, 9, 20, 40), cap, stream)
        assert status == (-7 if cap < matches else 0)
        assert len(got[0]) == cap  # *out_count = min(matches, capacity)
        assert np.array_equal(got[0].astype(np.int64), exact[0][:cap]) and np.array_equal(got[1], exact[1][:cap])


def test_noalloc_rejects_sizes_beyond_its_maximum():
    lib = pv.load()
    z = ctypes.c_void_p(0)
    too_many = (1 << 28) + 1
    st = lib.pv_filter_project_noalloc(z, z, z, too_many, 0, 1, 0, 1, z, z, 0, z, z, z)
    assert st == -1
