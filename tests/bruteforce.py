"""Brute-force evaluation of a neutral plan on tiny tables (pins the oracle).

Independent of the oracle's structure: every join is a nested loop over the
cross product of the fact row with every build table's rows (CROSS_JOIN
followed by FILTER on the equi-join condition, Table 1), and grouping is a
linear scan over a Python list of groups.  Pure Python integers, wrapped to
signed 64 bits after every operation.
"""
from __future__ import annotations

import itertools

import numpy as np

M64 = 1 << 64


def wrap(v: int) -> int:
    v %= M64
    return v - M64 if v >= (1 << 63) else v


def _cell(v):
    """A table cell: text stays text, numbers become Python integers."""
    if isinstance(v, (str, bytes)):
        return v
    if isinstance(v, np.generic) and v.dtype.kind in ("U", "S"):
        return v.item()
    return int(v)


def like(s, pattern) -> bool:
    """SQL LIKE by recursion on the pattern: '%' matches nothing or one more
    character, '_' one character, anything else itself."""
    if not pattern:
        return not s
    if pattern[0] == "%":
        return like(s, pattern[1:]) or (len(s) > 0 and like(s[1:], pattern))
    if s and (pattern[0] == "_" or pattern[0] == s[0]):
        return like(s[1:], pattern[1:])
    return False


def _holds(v, p) -> bool:
    op = p[1]
    if op == "prefix":
        return v[:len(p[2])] == p[2]
    if op == "like":
        return like(v, p[2])
    if op == "in":
        return any(v == x for x in p[2])
    if op == "lt":
        return v < p[2]
    if op == "le":
        return v <= p[2]
    if op == "gt":
        return v > p[2]
    if op == "ge":
        return v >= p[2]
    if op == "eq":
        return v == p[2]
    if op == "between":
        return p[2] <= v <= p[3]
    raise ValueError(op)


class DuplicateBuildKey(Exception):
    pass


def evaluate(plan: dict, tables: dict) -> dict:
    fact = tables[plan["fact"]]
    n = len(next(iter(fact.values())))
    builds = plan.get("builds", [])
    surviving = []
    for b in builds:
        t = tables[b["table"]]
        m = len(t[b["key"]])
        rows = [r for r in range(m) if all(_holds(_cell(t[p[0]][r]), p) for p in b.get("filters", []))]
        keys = [int(t[b["key"]][r]) for r in rows]
        if len(keys) != len(set(keys)):
            raise DuplicateBuildKey()
        surviving.append(rows)
    probes = plan.get("probes", [])

    def value(ref, r, combo):
        if isinstance(ref, str):
            return int(fact[ref][r])
        _, p, i = ref
        b = builds[probes[p]["build"]]
        return int(tables[b["table"]][b["payload"][i]][combo[p]])

    matches = []  # (fact row, tuple of matched build rows per probe)
    for r in range(n):
        for combo in itertools.product(*[surviving[q["build"]] for q in probes]):
            ok = all(_holds(_cell(fact[p[0]][r]), p) for p in plan.get("filters", []))
            for j, q in enumerate(probes):
                b = builds[q["build"]]
                ok = ok and int(fact[q["fk"]][r]) == int(tables[b["table"]][b["key"]][combo[j]])
            if ok:
                matches.append((r, combo))

    if plan.get("project"):
        cols = [[value(ref, r, c) for (r, c) in matches] for ref in plan["project"]]
        return {"kind": "project", "cols": cols}

    aggs = plan["aggs"]

    def agg_value(a, r, combo):
        if a[0] == "count":
            return 1
        v = 1
        for t in a[1]:
            x = value(t[1], r, combo)
            if t[0] == "x":
                tv = x
            elif t[0] == "x_plus_c":
                tv = wrap(x + t[2])
            else:
                tv = wrap(t[2] - x)
            v = wrap(v * tv)
        return v

    def fold(acc, vals):
        out = []
        for a, cur, v in zip(aggs, acc, vals):
            if cur is None:
                out.append(v)
            elif a[0] in ("sum", "count"):
                out.append(wrap(cur + v))
            elif a[0] == "min":
                out.append(min(cur, v))
            else:
                out.append(max(cur, v))
        return out

    keys = plan.get("group_by", [])
    if not keys:
        acc = [None] * len(aggs)
        for r, combo in matches:
            acc = fold(acc, [agg_value(a, r, combo) for a in aggs])
        return {"kind": "ungrouped", "cols": [[0 if v is None else v] for v in acc]}
    groups = []  # list of [key tuple, acc], linear scan
    for r, combo in matches:
        k = tuple(value(ref, r, combo) for ref in keys)
        vals = [agg_value(a, r, combo) for a in aggs]
        for g in groups:
            if g[0] == k:
                g[1] = fold(g[1], vals)
                break
        else:
            groups.append([k, fold([None] * len(aggs), vals)])
    groups.sort(key=lambda g: g[0])
    cols = [[g[0][i] for g in groups] for i in range(len(keys))]
    cols += [[g[1][j] for g in groups] for j in range(len(aggs))]
    return {"kind": "grouped", "cols": cols}
