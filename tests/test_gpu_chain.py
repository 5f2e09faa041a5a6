"""A query of several pipelines in which later pipelines read earlier
results (TPC-H Q5 shape, workloads.q5_chain): two builds run over projection
results and the last aggregation runs over a grouped result.  The chain runs
eagerly and as one captured CUDA graph, against the oracle evaluating the
same steps on the host, at a ragged small size and with 60M line items; the
graph is replayed after the inputs change in place, so every build and
pipeline must be recomputed from the new data."""
import numpy as np
import pytest

from oracle import oracle
from paper_1709_00700_gb300 import datagen, pv, workloads
from tests.gpu_util import assert_same

pytestmark = pytest.mark.gpu


def _register(ctx, tables):
    import torch
    dev = {t: {c: torch.from_numpy(np.ascontiguousarray(v)).cuda() for c, v in cols.items()}
           for t, cols in tables.items()}
    for t, cols in dev.items():
        ctx.register_table(t, cols)
    return dev


def _check_steps(chain, got_steps, want_steps, variants):
    for st, got, w in zip(chain, got_steps, want_steps):
        kw = variants.get(st["name"], {})
        ordered = "project" not in st["plan"] or kw.get("exec") == "multi"
        if "group_by" in st["plan"]:  # grouped results: compare sorted by key
            order = np.lexsort(tuple(np.asarray(c) for c in reversed(got[:len(st["plan"]["group_by"])])))
            got = [np.asarray(c)[order] for c in got]
        assert_same(got, w["cols"], ordered=ordered, ctxmsg=f"step {st['name']} {kw}")


def _run(ctx, tables, dev, chain, variants, htv, mutate):
    want = oracle.run_chain(chain, tables, nthreads=oracle.hardware_threads())
    assert len(want[-1]["cols"][0]) > 0
    ch = ctx.run_chain(chain, {k: pv.variant(**v) for k, v in variants.items()}, htv)
    _check_steps(chain, [ch.fetch(i) for i in range(len(chain))], want, variants)
    ch.capture()
    for _ in range(2):
        ch.launch()
    ctx.sync()
    _check_steps(chain, [ch.fetch(i) for i in range(len(chain))], want, variants)
    # new order dates and discounts written in place: the graph recomputes the whole query
    changed = mutate(tables, dev)
    want = oracle.run_chain(chain, changed, nthreads=oracle.hardware_threads())
    ch.launch()
    ctx.sync()
    _check_steps(chain, [ch.fetch(i) for i in range(len(chain))], want, variants)
    generic = [ctx.result_kernel(res)[0] for _, _, res in ch.steps]
    ch.free()
    return generic


def _mutate(seed):
    def f(tables, dev):
        import torch
        o = dict(tables["orders"])
        li = dict(tables["lineitem"])
        n_o, n_l = len(o["o_orderdate"]), len(li["l_discount"])
        o["o_orderdate"] = datagen.uniform_int(seed, 812, n_o, datagen.DAY0, datagen.DAY0 + datagen.TPCH_DAYS,
                                               np.int32)
        li["l_discount"] = datagen.uniform_int(seed, 823, n_l, 0, 11, np.int64)
        dev["orders"]["o_orderdate"].copy_(torch.from_numpy(o["o_orderdate"]))
        dev["lineitem"]["l_discount"].copy_(torch.from_numpy(li["l_discount"]))
        torch.cuda.synchronize()
        return dict(tables, orders=o, lineitem=li)
    return f


COMPILED = {"cust": dict(exec="single", items_per_thread=1), "ord": dict(exec="multi", items_per_thread=2),
            "nat": dict(agg="local", ht="perfect", items_per_thread=1, block=512),
            "region": dict(agg="global", ht="perfect")}
GENERIC = {"cust": dict(exec="multi", interp=1), "ord": dict(exec="single", interp=1, pred="predicated"),
           "nat": dict(agg="global", ht="linear", interp=1), "region": dict(agg="local", ht="linear")}


@pytest.mark.parametrize("variants,build", [(COMPILED, "perfect"), (GENERIC, "linear"), (COMPILED, "cuckoo")])
def test_q5_chain_small(variants, build):
    ctx = pv.Context(0)
    tables = datagen.tpch_schema(100_003, seed=21)
    dev = _register(ctx, tables)
    generic = _run(ctx, tables, dev, workloads.q5_chain(), variants, pv.ht_variant(build), _mutate(22))
    assert generic[-1]  # the last step reads a result: generic kernels
    if variants is COMPILED:
        assert generic[:3] == [False, False, False]  # the compiled shapes of the chain's steps
    ctx.close()


def test_q5_chain_60m_line_items():
    ctx = pv.Context(0)
    tables = datagen.tpch_schema(60_000_000)
    dev = _register(ctx, tables)
    _run(ctx, tables, dev, workloads.q5_chain(), COMPILED, pv.ht_variant("perfect"), _mutate(23))
    ctx.close()
