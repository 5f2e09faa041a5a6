"""Python front end of the CPU oracle (TEST INFRASTRUCTURE ONLY).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this module.  It builds ``liboracle.so`` from ``pv_oracle.cpp`` with
g++, translates a neutral query plan (plain Python dict, described below)
into the oracle's own plan words, and returns the exact result.

Neutral plan (the query written as the pipeline programs of Table 2):

    {
      "fact":    "<fact table name>",
      "builds":  [{"table": t, "key": col, "filters": [pred...], "payload": [col...]}],
      "filters": [pred...],                  # FILTER on the fact table (conjunction)
      "probes":  [{"build": i, "fk": col}],  # HASH_PROBE in this order
      "group_by":[ref...],                   # HASH_AGGREGATE keys (empty: AGGREGATE)
      "aggs":    [agg...],
      "project": [ref...],                   # PROJECT (mutually exclusive with aggs)
    }
    pred = (col, op, c) with op in lt/le/gt/ge/eq, or (col, "between", lo, hi);
           on a column of strings (a numpy str or bytes array) also
           (col, "prefix", s), (col, "like", pattern), (col, "in", [s...])
    ref  = "col" (fact column) or ("payload", probe_index, payload_index)
    agg  = ("count",) or (func, [term...]) with func in sum/min/max and the
           value the product of its terms (ARITHMETIC)
    term = ("x", ref) | ("x_plus_c", ref, c) | ("c_minus_x", ref, c)
"""
from __future__ import annotations

import ctypes
import os
import re
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pv_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

_OPS = {"lt": 0, "le": 1, "gt": 2, "ge": 3, "eq": 4, "between": 5}
_FUNCS = {"sum": 0, "count": 1, "min": 2, "max": 3}
_TERMS = {"x": 0, "x_plus_c": 1, "c_minus_x": 2}
_TYPES = {np.dtype(np.int32): 0, np.dtype(np.int64): 1, np.dtype(np.uint8): 2}
ERRORS = {-1: "ERR_PLAN", -2: "ERR_COLUMN", -6: "ERR_DUP_BUILD_KEY"}


class OracleError(RuntimeError):
    def __init__(self, code: int, msg: str = ""):
        super().__init__(f"oracle error {code} ({ERRORS.get(code, '?')}) {msg}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (plain C++17, no CUDA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.or_run.restype = ctypes.c_int
        lib.or_run.argtypes = [ctypes.POINTER(ctypes.c_int64), ctypes.c_int64,
                               ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int32),
                               ctypes.POINTER(ctypes.c_int64), ctypes.c_int32, ctypes.c_int64,
                               ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)]
        for name in ("or_result_rows",):
            getattr(lib, name).restype = ctypes.c_int64
            getattr(lib, name).argtypes = [ctypes.c_void_p]
        for name in ("or_result_cols", "or_result_kind", "or_result_flags"):
            getattr(lib, name).restype = ctypes.c_int32
            getattr(lib, name).argtypes = [ctypes.c_void_p]
        lib.or_result_copy_col.restype = None
        lib.or_result_copy_col.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
        lib.or_result_free.restype = None
        lib.or_result_free.argtypes = [ctypes.c_void_p]
        lib.or_last_error.restype = ctypes.c_char_p
        lib.or_hardware_threads.restype = ctypes.c_int32
        _lib = lib
    return _lib


def hardware_threads() -> int:
    return int(_load().or_hardware_threads())


class _Encoder:
    def __init__(self, tables):
        self.tables = tables
        self.cols = []      # arrays, contiguous
        self.index = {}     # (table, col) -> index

    def col(self, table, name):
        k = (table, name)
        if k not in self.index:
            a = np.ascontiguousarray(self.tables[table][name])
            if a.dtype not in _TYPES:
                raise TypeError(f"unsupported column dtype {a.dtype} for {table}.{name}")
            self.index[k] = len(self.cols)
            self.cols.append(a)
        return self.index[k]


def _pred_words(enc, table, p):
    col, op = p[0], p[1]
    c0 = int(p[2])
    c1 = int(p[3]) if op == "between" else 0
    return [enc.col(table, col), _OPS[op], c0, c1]


def encode(plan: dict, tables: dict):
    """Neutral plan -> (plan words, encoder holding the referenced columns)."""
    enc = _Encoder(tables)
    fact = plan["fact"]
    w = []
    builds = plan.get("builds", [])
    w.append(len(builds))
    for b in builds:
        w.append(enc.col(b["table"], b["key"]))
        w.append(len(b.get("filters", [])))
        for p in b.get("filters", []):
            w += _pred_words(enc, b["table"], p)
        w.append(len(b.get("payload", [])))
        for c in b.get("payload", []):
            w.append(enc.col(b["table"], c))

    def ref(r):
        if isinstance(r, str):
            return [0, enc.col(fact, r), 0]
        kind, p, i = r
        assert kind == "payload"
        return [1, int(p), int(i)]

    filters = plan.get("filters", [])
    w.append(len(filters))
    for p in filters:
        w += _pred_words(enc, fact, p)
    probes = plan.get("probes", [])
    w.append(len(probes))
    for q in probes:
        w += [int(q["build"]), enc.col(fact, q["fk"])]
    keys = plan.get("group_by", [])
    w.append(len(keys))
    for r in keys:
        w += ref(r)
    aggs = plan.get("aggs", [])
    w.append(len(aggs))
    for a in aggs:
        func = a[0]
        terms = a[1] if len(a) > 1 else []
        w += [_FUNCS[func], len(terms)]
        for t in terms:
            kind = t[0]
            c = int(t[2]) if kind != "x" else 0
            w += [_TERMS[kind]] + ref(t[1]) + [c]
    proj = plan.get("project", [])
    w.append(len(proj))
    for r in proj:
        w += ref(r)
    return np.array(w, dtype=np.int64), enc


# String predicates (FILTER of Table 1 on text attributes; the SQL LIKE of
# Section 9.2.1).  Each is evaluated here on the strings themselves, row by
# row, into a 0/1 int32 column that the plan then filters with "eq 1".
# Strings compare by code point (str) or byte (bytes).
def _like_regex(pattern):
    """SQL LIKE as a regular expression: '%' any run, '_' one character."""
    text = pattern.decode("latin-1") if isinstance(pattern, bytes) else pattern
    body = "".join(".*" if ch == "%" else "." if ch == "_" else re.escape(ch) for ch in text)
    return re.compile(body, re.DOTALL)


def _string_test(p, as_bytes: bool):
    conv = (lambda x: x.encode() if isinstance(x, str) else x) if as_bytes else \
           (lambda x: x.decode() if isinstance(x, bytes) else x)
    op = p[1]
    if op == "like":
        rx = _like_regex(p[2])
        if as_bytes:
            return lambda v: rx.fullmatch(v.decode("latin-1")) is not None
        return lambda v: rx.fullmatch(v) is not None
    if op == "in":
        members = {conv(x) for x in p[2]}
        return lambda v: v in members
    c0 = conv(p[2])
    if op == "lt":
        return lambda v: v < c0
    if op == "le":
        return lambda v: v <= c0
    if op == "gt":
        return lambda v: v > c0
    if op == "ge":
        return lambda v: v >= c0
    if op == "eq":
        return lambda v: v == c0
    if op == "between":
        c1 = conv(p[3])
        return lambda v: c0 <= v <= c1
    if op == "prefix":
        return lambda v: v.startswith(c0)
    raise OracleError(-1, f"bad string predicate {p}")


def _is_text(a) -> bool:
    """Columns of strings: numpy str / bytes arrays, or object arrays (which
    hold nothing but text in a table)."""
    return np.asarray(a).dtype.kind in ("U", "S", "O")


def resolve_string_filters(plan: dict, tables: dict):
    """Returns (plan, tables) in which every predicate on a column of strings
    is replaced by "eq 1" on a 0/1 int32 column holding its value per row."""
    if not any(_is_text(c) for t in tables.values() for c in t.values()):
        return plan, tables
    plan = dict(plan)
    tables = {t: dict(cols) for t, cols in tables.items()}
    made = [0]

    def rewrite(table, preds):
        out = []
        for p in preds:
            col = tables[table].get(p[0])
            if col is None or not _is_text(col):
                out.append(p)
                continue
            a = np.asarray(col)
            test = _string_test(p, a.dtype.kind == "S" or (a.dtype.kind == "O" and len(a) > 0 and isinstance(a[0], bytes)))
            seen = {}
            flags = np.empty(len(a), dtype=np.int32)
            for i, v in enumerate(a.tolist()):
                f = seen.get(v)
                if f is None:
                    f = seen[v] = 1 if test(v) else 0
                flags[i] = f
            name = f"__text{made[0]}"
            made[0] += 1
            tables[table][name] = flags
            out.append([name, "eq", 1])
        return out

    plan["builds"] = [dict(b, filters=rewrite(b["table"], b.get("filters", []))) for b in plan.get("builds", [])]
    plan["filters"] = rewrite(plan["fact"], plan.get("filters", []))
    return plan, tables


def fact_rows(plan: dict, tables: dict) -> int:
    fact = tables[plan["fact"]]
    return len(next(iter(fact.values())))


def run(plan: dict, tables: dict, nthreads: int = 1) -> dict:
    """Evaluate the plan exactly.  Returns {"kind", "cols" (int64 arrays), "overflow"}.

    kind: "ungrouped" (one row, one column per aggregate), "grouped" (key
    columns then aggregate columns, ascending by key), or "project" (projected
    columns in input order)."""
    lib = _load()
    plan, tables = resolve_string_filters(plan, tables)
    words, enc = encode(plan, tables)
    n = len(enc.cols)
    ptrs = (ctypes.c_void_p * max(n, 1))(*[a.ctypes.data for a in enc.cols])
    types = (ctypes.c_int32 * max(n, 1))(*[_TYPES[a.dtype] for a in enc.cols])
    lens = (ctypes.c_int64 * max(n, 1))(*[len(a) for a in enc.cols])
    out = ctypes.c_void_p()
    rc = lib.or_run(words.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(words), ptrs, types,
                    lens, n, fact_rows(plan, tables), int(nthreads), ctypes.byref(out))
    if rc != 0:
        raise OracleError(rc, lib.or_last_error().decode())
    try:
        nrows = lib.or_result_rows(out)
        cols = []
        for c in range(lib.or_result_cols(out)):
            a = np.empty(nrows, dtype=np.int64)
            lib.or_result_copy_col(out, c, a.ctypes.data)
            cols.append(a)
        kind = {0: "ungrouped", 1: "grouped", 2: "project"}[lib.or_result_kind(out)]
        return {"kind": kind, "cols": cols, "overflow": bool(lib.or_result_flags(out) & 1)}
    finally:
        lib.or_result_free(out)


def run_chain(chain: list, tables: dict, nthreads: int = 1) -> list:
    """A query of several pipelines (paper_1709_00700_gb300.workloads.q5_chain
    format): each step's plan is evaluated exactly, and its result columns
    become table step["name"] for the later steps.  Returns every step's
    result, in order."""
    tables = dict(tables)
    out = []
    for step in chain:
        res = run(step["plan"], tables, nthreads=nthreads)
        tables[step["name"]] = dict(zip(step["columns"], res["cols"]))
        out.append(res)
    return out
