"""Helpers for the GPU parity tests: device tables, comparisons with the oracle."""
from __future__ import annotations

import numpy as np

from oracle import oracle


def to_device(tables: dict) -> dict:
    import torch
    return {t: {c: torch.from_numpy(np.ascontiguousarray(v)).cuda() for c, v in cols.items()}
            for t, cols in tables.items()}


def register(ctx, tables: dict):
    for t, cols in to_device(tables).items():
        ctx.register_table(t, cols)


def rows_sorted(cols):
    """Lexicographically sorted rows of a list of equal-length columns."""
    if not cols or len(cols[0]) == 0:
        return [np.asarray(c, dtype=np.int64) for c in cols]
    order = np.lexsort(tuple(np.asarray(c) for c in reversed(cols)))
    return [np.asarray(c, dtype=np.int64)[order] for c in cols]


def assert_same(got, want, ordered=True, ctxmsg=""):
    assert len(got) == len(want), f"{ctxmsg}: {len(got)} vs {len(want)} columns"
    if not ordered:
        got, want = rows_sorted(got), rows_sorted(want)
    for i, (g, w) in enumerate(zip(got, want)):
        g = np.asarray(g, dtype=np.int64)
        w = np.asarray(w, dtype=np.int64)
        assert g.shape == w.shape, f"{ctxmsg}: column {i} has {g.shape} rows, oracle {w.shape}"
        if not np.array_equal(g, w):
            bad = np.nonzero(g != w)[0][:5]
            raise AssertionError(f"{ctxmsg}: column {i} differs at rows {bad}: {g[bad]} vs {w[bad]}")


def want(plan, tables, threads=8):
    return oracle.run(plan, tables, nthreads=threads)["cols"]
