"""Row-sharded execution of one query: the exchange step of the multi-GPU
design.

Each rank runs the same pipeline program (Table 2) on a contiguous slice of
the fact table's rows, while every build pipeline runs whole on every rank
(the dimension tables are small).  The ranks' partial results then merge:

- HASH_AGGREGATE: by group key.  SUM and COUNT add (wrapping mod 2^64 like
  the kernels); MIN and MAX keep the extreme over the ranks where the group
  has rows.
- AGGREGATE: SUM and COUNT add; MIN and MAX are taken over the ranks whose
  COUNT is non-zero, so a plan with MIN or MAX needs a COUNT aggregate.
- PROJECT: concatenation in rank order, which keeps input order.

A box here holds one GPU, so the benchmark runs independent replicas; this
module is the host side of the design, exercised by CPU ranks.
"""
from __future__ import annotations

import numpy as np

_M64 = 1 << 64


def _wrap(v: int) -> int:
    v %= _M64
    return v - _M64 if v >= (1 << 63) else v


def row_slice(n_rows: int, rank: int, world: int) -> tuple:
    """[start, stop) of rank's rows: contiguous slices, the first n_rows mod
    world ranks one row longer."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank outside the world")
    base, extra = divmod(n_rows, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def _combine(func: str, a: int, b: int) -> int:
    if func in ("sum", "count"):
        return _wrap(a + b)
    return min(a, b) if func == "min" else max(a, b)


def merge(plan: dict, parts: list) -> list:
    """The plan's result from the ranks' partial results (parts[r] = rank r's
    int64 result columns on its slice, in the plan's column order).  Grouped
    results come back sorted by key."""
    if not parts:
        raise ValueError("no partial results")
    ncols = len(parts[0])
    if plan.get("project"):
        return [np.concatenate([np.asarray(p[i], dtype=np.int64) for p in parts]) for i in range(ncols)]
    funcs = [a[0] for a in plan.get("aggs", [])]
    nk = len(plan.get("group_by", []))
    if nk == 0:
        extremes = [i for i, f in enumerate(funcs) if f in ("min", "max")]
        if extremes and "count" not in funcs:
            raise ValueError("merging MIN or MAX needs a COUNT aggregate")
        c = funcs.index("count") if "count" in funcs else None
        out = []
        for i, f in enumerate(funcs):
            vals = [int(p[i][0]) for p in parts if f in ("sum", "count") or int(p[c][0]) > 0]
            v = 0
            for j, x in enumerate(vals):
                v = x if j == 0 else _combine(f, v, x)
            out.append(np.array([v], dtype=np.int64))
        return out
    groups = {}
    for p in parts:
        for r in range(len(p[0])):
            key = tuple(int(p[k][r]) for k in range(nk))
            vals = [int(p[nk + i][r]) for i in range(len(funcs))]
            if key in groups:
                groups[key] = [_combine(f, a, b) for f, a, b in zip(funcs, groups[key], vals)]
            else:
                groups[key] = vals
    keys = sorted(groups)
    cols = [np.array([k[i] for k in keys], dtype=np.int64) for i in range(nk)]
    cols += [np.array([groups[k][i] for k in keys], dtype=np.int64) for i in range(len(funcs))]
    return cols
