"""Variant exploration on the GPU (Section 8).

* ``exhaustive``: run every variant of a space and keep the fastest
  ("backtracking" in Table 4);
* ``feature_wise``: Algorithm 1 — start from the first value of every
  dimension, sweep one dimension at a time with the others fixed, keep the
  fastest value, repeat until a sweep changes nothing or q sweeps ran; with
  early termination and feature ordering (Section 8.2);
* ``GraphBatch``: many small pipelines captured once as one CUDA graph and
  replayed without per-launch overhead;
* a JSONL timing database keyed by query and variant, so tuning can resume.

Timing: after one untimed run (allocation), ``reps`` runs each preceded by an
L2 flush, CUDA events on the context stream around the pipeline only; the
median is the variant's time.  A variant whose first timed run exceeds
``cap_factor`` times the best time so far is abandoned (the paper prunes
variants slower than one second, Section 9.1).
"""
from __future__ import annotations

import itertools
import json
import math
import os
import statistics
import time

from . import pv

# Variant dimensions per pipeline kind, in the feature order of Section 8.2
# (execution strategy, degree of parallelism, memory access first).
SPACES = {
    "project": [
        ("exec", ["multi", "single"]),
        ("grid_mult", [0, 1, 2, 4, 8, 16]),
        ("block", [256, 128, 512, 1024]),
        ("access", ["grid", "chunked"]),
        ("pred", ["branch", "predicated"]),
        ("items_per_thread", [4, 2, 1]),
    ],
    "aggregate": [
        ("grid_mult", [0, 1, 2, 4, 8, 16]),
        ("block", [256, 128, 512, 1024]),
        ("access", ["grid", "chunked"]),
        ("pred", ["branch", "predicated"]),
        ("items_per_thread", [2, 4, 1]),
    ],
    "grouped": [
        ("agg", ["local", "global"]),
        ("ht", ["perfect", "linear", "cuckoo"]),
        ("exec", ["single", "multi"]),
        ("threads_per_table", [0, 1]),
        ("grid_mult", [0, 1, 2, 4, 8]),
        ("block", [256, 128, 512]),
        ("access", ["grid", "chunked"]),
        ("pred", ["branch", "predicated"]),
        ("hash", ["murmur", "multshift"]),
        ("items_per_thread", [2, 1]),
    ],
}


def plan_kind(plan: dict) -> str:
    if plan.get("project"):
        return "project"
    return "grouped" if plan.get("group_by") else "aggregate"


def enumerate_space(dims):
    names = [d for d, _ in dims]
    for values in itertools.product(*[v for _, v in dims]):
        yield dict(zip(names, values))


def paper_space(kind: str):
    """The variant space of the paper's evaluation (Section 9.2.2), as an
    enumeration: projection pipelines 2 memory access x 2 predication x
    (single pass at multiplier 1, or multi pass at 7 multipliers) = 32;
    aggregation pipelines 2 x 2 x 2 hash tables x 2 hash functions x
    (local: 7 table multipliers x 7 work-group sizes, or global: 7 work-group
    sizes) = 896."""
    mult = [1, 8, 64, 256, 1024, 16384, 65536]
    wg = [16, 32, 64, 128, 256, 512, 1024]
    out = []
    if kind == "project":
        for acc, pred in itertools.product(["sequential", "coalesced"], ["branched", "predicated"]):
            out.append(dict(access=acc, pred=pred, exec="single", multiplier=1))
            out += [dict(access=acc, pred=pred, exec="multi", multiplier=m) for m in mult]
    elif kind == "aggregate":
        for acc, pred, ht, h in itertools.product(["sequential", "coalesced"], ["branched", "predicated"],
                                                  ["linear", "cuckoo"], ["murmur", "multshift"]):
            out += [dict(access=acc, pred=pred, ht=ht, hash=h, agg="local", tables=m, wg=w)
                    for m, w in itertools.product(mult, wg)]
            out += [dict(access=acc, pred=pred, ht=ht, hash=h, agg="global", wg=w) for w in wg]
    else:
        raise ValueError(kind)
    return out


def variant_key(v: dict) -> str:
    return json.dumps(v, sort_keys=True)


class TimingDB:
    """Append-only JSONL of (query id, variant, ms); reloadable."""

    def __init__(self, path: str | None):
        self.path = path
        self.rows = {}
        if path and os.path.exists(path):
            with open(path) as f:
                for line in f:
                    r = json.loads(line)
                    self.rows[(r["query"], variant_key(r["variant"]))] = r["ms"]

    def get(self, q, v):
        return self.rows.get((q, variant_key(v)))

    def put(self, q, v, ms):
        self.rows[(q, variant_key(v))] = ms
        if self.path:
            with open(self.path, "a") as f:
                f.write(json.dumps({"query": q, "variant": v, "ms": ms}) + "\n")


class Measurer:
    """Times one plan (builds done once) under variants on a Context."""

    def __init__(self, ctx: "pv.Context", plan: dict, build_ht: str = "perfect", reps: int = 5,
                 cap_factor: float = 20.0, flush: bool = True):
        import torch
        self.torch = torch
        self.ctx = ctx
        self.plan = plan
        self.reps = reps
        self.cap_factor = cap_factor
        self.flush = flush
        self.hts = ctx.build_all(plan, pv.ht_variant(build_ht))
        ctx.sync()
        self.best = math.inf
        self.runs = 0

    def close(self):
        for h in self.hts:
            self.ctx.free(h)
        self.hts = []

    def __call__(self, v: dict) -> float:
        """Median ms of the variant; inf when it has no instantiation.  A
        "probe_order" entry runs the probes in that order (pv.reorder_probes;
        the builds are shared)."""
        ctx, torch = self.ctx, self.torch
        v = dict(v)
        order = v.pop("probe_order", None)
        plan = self.plan if order is None else pv.reorder_probes(self.plan, order)[0]
        try:
            res = ctx.run(plan, pv.variant(**v), self.hts)
            ctx.sync()
        except pv.PVError as e:
            if e.status in (-2, -1):
                return math.inf
            raise
        try:
            times = []
            st = ctx.stream
            for i in range(self.reps):
                if self.flush:
                    ctx.lib.pv_l2_flush(ctx.h)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(st)
                ctx.rerun(res)
                b.record(st)
                b.synchronize()
                ms = a.elapsed_time(b)
                times.append(ms)
                if i == 0 and ms > self.cap_factor * self.best:
                    break
            ctx.sync()
        finally:
            ctx.free(res)
        self.runs += 1
        t = statistics.median(times)
        self.best = min(self.best, t)
        return t


def probe_order_dim(plan: dict):
    """HASH_PROBE order as a search dimension: ("probe_order", every order of
    the plan's probes, its own first).  Orders whose rewritten plan has no
    compiled shape measure as inf."""
    return ("probe_order", pv.probe_orders(plan))


def exhaustive(measure, dims, db: TimingDB | None = None, qid: str = ""):
    """Runs every variant; returns (best variant, best ms, {key: ms}, seconds)."""
    t0 = time.perf_counter()
    best, best_ms, all_ms = None, math.inf, {}
    for v in enumerate_space(dims):
        ms = db.get(qid, v) if db else None
        if ms is None:
            ms = measure(v)
            if db:
                db.put(qid, v, ms)
        all_ms[variant_key(v)] = ms
        if ms < best_ms:
            best, best_ms = v, ms
    return best, best_ms, all_ms, time.perf_counter() - t0


def feature_wise(cost, dims, q: int = 3, early_termination: bool = False, order=None):
    """Algorithm 1.  ``cost(v)`` is the execution time of the workload under
    configuration v (lower is better).  Starts from the first value of every
    dimension; for each dimension in turn tries every value with the others
    fixed and keeps the fastest (ties keep the earliest value; a dimension
    whose values all fail keeps its current value); stops when a sweep leaves
    the configuration unchanged or after q sweeps.  Early termination stops
    after the first sweep that finds no faster configuration than the best
    seen so far.  Returns (v, cost(v), number of cost evaluations)."""
    if order is not None:
        dims = [d for d in dims if d[0] in order]
        dims.sort(key=lambda d: order.index(d[0]))
    v = {name: values[0] for name, values in dims}
    cache = {}

    def c(x):
        k = variant_key(x)
        if k not in cache:
            cache[k] = cost(x)
        return cache[k]

    best_seen = c(v)
    for _ in range(q):
        last = dict(v)
        improved = False
        for name, values in dims:
            best_t, best_val = math.inf, None
            for d in values:
                w = dict(v)
                w[name] = d
                t = c(w)
                if t < best_t:
                    best_t, best_val = t, d
            if best_val is not None:
                v[name] = best_val
                if best_t < best_seen:
                    best_seen, improved = best_t, True
        if v == last:
            break
        if early_termination and not improved:
            break
    return v, c(v), len(cache)


class GraphBatch:
    """Captures reruns of many prepared results (e.g. small queries) as one
    CUDA graph on the context stream; ``launch`` replays all of them."""

    def __init__(self, ctx: "pv.Context", results, flush_between: bool = False):
        import ctypes
        self.ctx = ctx
        lib = ctx.lib
        if flush_between:
            ctx._check(lib.pv_l2_flush(ctx.h))
        ctx.sync()
        ctx._check(lib.pv_graph_capture_begin(ctx.h))
        try:
            for r in results:
                if flush_between:
                    ctx._check(lib.pv_l2_flush(ctx.h))
                ctx._check(lib.pv_rerun(ctx.h, r))
        finally:
            g = ctypes.c_int32()
            st = lib.pv_graph_capture_end(ctx.h, ctypes.byref(g))
        ctx._check(st)
        self.g = g.value

    def launch(self):
        self.ctx._check(self.ctx.lib.pv_graph_launch(self.ctx.h, self.g))

    def free(self):
        self.ctx.free(self.g)
