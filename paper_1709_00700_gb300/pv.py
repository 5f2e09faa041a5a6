"""Python binding of libpv (argument marshalling only).

The functions ``pv_*`` mirror the C ABI of include/pv.h one to one through
ctypes.  :class:`Context` is a thin convenience layer: it registers torch
CUDA tensors as columns, translates a neutral plan dict (the pipeline
programs of a query, Table 2; format in ``oracle`` and ``workloads``) into
pv_build_spec / pv_pipeline_spec structs, and copies results back.  Every
step of a pipeline runs in libpv's CUDA kernels; there is no CPU path here.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpv.so")

# ---- constants (include/pv.h) ----------------------------------------------
PV_OK = 0
STATUS = {0: "PV_OK", -1: "PV_ERR_INVALID_ARG", -2: "PV_ERR_UNSUPPORTED", -3: "PV_ERR_HT_FULL",
          -4: "PV_ERR_CUCKOO_CYCLE", -5: "PV_ERR_KEY_OUT_OF_RANGE", -6: "PV_ERR_DUP_BUILD_KEY",
          -7: "PV_ERR_OUTPUT_OVERFLOW", -8: "PV_ERR_TIMEOUT", -9: "PV_ERR_CUDA", -10: "PV_ERR_OOM"}
PV_I32, PV_I64, PV_U8 = 0, 1, 2
MAX_PREDS, MAX_PROBES, MAX_KEYS, MAX_AGGS, MAX_TERMS, MAX_PROJ, MAX_PAYLOAD = 4, 4, 3, 8, 3, 4, 4
OPS = {"lt": 0, "le": 1, "gt": 2, "ge": 3, "eq": 4, "between": 5}
FUNCS = {"sum": 0, "count": 1, "min": 2, "max": 3}
TERMS = {"x": 0, "x_plus_c": 1, "c_minus_x": 2}
REF_COL, REF_PAYLOAD = 0, 1
HT = {"linear": 0, "cuckoo": 1, "perfect": 2}
HASH = {"murmur": 0, "multshift": 1}
EXEC = {"single": 0, "multi": 1}
AGG = {"local": 0, "global": 1, "cluster": 2}
PRED = {"branch": 0, "predicated": 1, "compacted": 2}
ACCESS = {"grid": 0, "chunked": 1, "staged": 2}
_NP_OF = {PV_I32: np.int32, PV_I64: np.int64, PV_U8: np.uint8}


class pv_ref(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("a", ctypes.c_int32), ("b", ctypes.c_int32)]


class pv_pred(ctypes.Structure):
    _fields_ = [("col", ctypes.c_int32), ("op", ctypes.c_int32), ("c0", ctypes.c_int64), ("c1", ctypes.c_int64)]


class pv_term(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("x", pv_ref), ("c", ctypes.c_int64)]


class pv_agg(ctypes.Structure):
    _fields_ = [("func", ctypes.c_int32), ("n_terms", ctypes.c_int32), ("terms", pv_term * MAX_TERMS)]


class pv_probe(ctypes.Structure):
    _fields_ = [("ht", ctypes.c_int32), ("fk", ctypes.c_int32)]


class pv_build_spec(ctypes.Structure):
    _fields_ = [("key", ctypes.c_int32), ("n_preds", ctypes.c_int32), ("preds", pv_pred * MAX_PREDS),
                ("n_payload", ctypes.c_int32), ("payload", ctypes.c_int32 * MAX_PAYLOAD)]


class pv_ht_variant(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("hash", ctypes.c_int32), ("cuckoo_k", ctypes.c_int32),
                ("max_evictions", ctypes.c_int32), ("load_factor", ctypes.c_double), ("seed", ctypes.c_uint64)]


class pv_pipeline_spec(ctypes.Structure):
    _fields_ = [("n_preds", ctypes.c_int32), ("preds", pv_pred * MAX_PREDS),
                ("n_probes", ctypes.c_int32), ("probes", pv_probe * MAX_PROBES),
                ("n_keys", ctypes.c_int32), ("keys", pv_ref * MAX_KEYS),
                ("n_aggs", ctypes.c_int32), ("aggs", pv_agg * MAX_AGGS),
                ("n_proj", ctypes.c_int32), ("proj", pv_ref * MAX_PROJ),
                ("capacity_hint", ctypes.c_int64)]


class pv_variant(ctypes.Structure):
    _fields_ = [("exec", ctypes.c_int32), ("agg", ctypes.c_int32), ("pred", ctypes.c_int32),
                ("access", ctypes.c_int32), ("ht", ctypes.c_int32), ("hash", ctypes.c_int32),
                ("block", ctypes.c_int32), ("grid_mult", ctypes.c_int32),
                ("items_per_thread", ctypes.c_int32), ("threads_per_table", ctypes.c_int32),
                ("cuckoo_k", ctypes.c_int32), ("prefetch", ctypes.c_int32), ("warp_agg", ctypes.c_int32),
                ("interp", ctypes.c_int32), ("compact_probes", ctypes.c_int32), ("first_items", ctypes.c_int32),
                ("seed", ctypes.c_uint64)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_P = ctypes.POINTER
_SIGS = {
    "pv_create": (ctypes.c_int32, [_P(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p, ALLOC_FN, FREE_FN, ctypes.c_void_p]),
    "pv_destroy": (ctypes.c_int32, [ctypes.c_void_p]),
    "pv_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "pv_device_info": (ctypes.c_int32, [ctypes.c_void_p, _P(ctypes.c_int32), _P(ctypes.c_int64)]),
    "pv_set_l2_fetch_bytes": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, _P(ctypes.c_int32)]),
    "pv_register_column": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_char_p, ctypes.c_int32,
                                            ctypes.c_void_p, ctypes.c_int64, _P(ctypes.c_int32)]),
    "pv_column_stats": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, _P(ctypes.c_int64), _P(ctypes.c_int64)]),
    "pv_build_hash_table": (ctypes.c_int32, [ctypes.c_void_p, _P(pv_build_spec), _P(pv_ht_variant), _P(ctypes.c_int32)]),
    "pv_rebuild_hash_table": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32]),
    "pv_run_pipeline": (ctypes.c_int32, [ctypes.c_void_p, _P(pv_pipeline_spec), _P(pv_variant), _P(ctypes.c_int32)]),
    "pv_rerun": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32]),
    "pv_sync": (ctypes.c_int32, [ctypes.c_void_p]),
    "pv_set_timeout_ms": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int64]),
    "pv_result_shape": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, _P(ctypes.c_int64), _P(ctypes.c_int32)]),
    "pv_result_col_type": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, _P(ctypes.c_int32)]),
    "pv_fetch_result": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                         ctypes.c_int64, ctypes.c_int32]),
    "pv_free": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32]),
    "pv_result_kernel": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, _P(ctypes.c_int32), ctypes.c_char_p,
                                          ctypes.c_int64]),
    "pv_result_capacity": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, _P(ctypes.c_int64)]),
    "pv_enqueue_fetch": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, _P(ctypes.c_void_p),
                                          _P(ctypes.c_int64), ctypes.c_void_p, ctypes.c_int32]),
    "pv_enqueue_fetch_rows": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, _P(ctypes.c_void_p),
                                               _P(ctypes.c_int64), ctypes.c_void_p]),
    "pv_register_result_column": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_char_p,
                                                   ctypes.c_char_p, _P(ctypes.c_int32)]),
    "pv_graph_capture_begin": (ctypes.c_int32, [ctypes.c_void_p]),
    "pv_graph_capture_end": (ctypes.c_int32, [ctypes.c_void_p, _P(ctypes.c_int32)]),
    "pv_graph_launch": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32]),
    "pv_l2_flush": (ctypes.c_int32, [ctypes.c_void_p]),
    "pv_last_launch_count": (ctypes.c_int32, [ctypes.c_void_p, _P(ctypes.c_int32)]),
    "pv_set_kernel_timing": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32]),
    "pv_kernel_times": (ctypes.c_int32, [ctypes.c_void_p, _P(ctypes.c_float), ctypes.c_int32, _P(ctypes.c_int32)]),
    "pv_debug_spin": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int64]),
    "pv_mlp_forward": (ctypes.c_int32, [ctypes.c_void_p] + [ctypes.c_void_p] * 4 + [ctypes.c_int32, ctypes.c_int32,
                                                                                    ctypes.c_void_p, ctypes.c_void_p]),
    "pv_mlp_backward": (ctypes.c_int32, [ctypes.c_void_p] + [ctypes.c_void_p] * 7 + [ctypes.c_int32, ctypes.c_int32]
                        + [ctypes.c_void_p] * 3),
    "pv_mlp_adam": (ctypes.c_int32, [ctypes.c_void_p] + [ctypes.c_void_p] * 4 + [ctypes.c_int64, ctypes.c_float,
                                                                                 ctypes.c_float, ctypes.c_float,
                                                                                 ctypes.c_float, ctypes.c_int32]),
    "pv_fetch_results": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, _P(ctypes.c_void_p),
                                          _P(ctypes.c_int64), ctypes.c_int32]),
    "pv_atomic_peak": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64,
                                        ctypes.POINTER(ctypes.c_float)]),
    "pv_dict_range": (ctypes.c_int32, [_P(ctypes.c_char_p), ctypes.c_int64, ctypes.c_int32, ctypes.c_char_p,
                                       ctypes.c_char_p, _P(ctypes.c_int64), _P(ctypes.c_int64)]),
    "pv_dict_match": (ctypes.c_int32, [_P(ctypes.c_char_p), ctypes.c_int64, ctypes.c_char_p, _P(ctypes.c_int32),
                                       ctypes.c_int64, _P(ctypes.c_int64)]),
    "pv_filter_project_noalloc": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                                   ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
}
EXPORTS = tuple(_SIGS)

_lib = None


def load(path: str = LIB_PATH):
    """Loads libpv.so.  Raises if it has not been built: there is no fallback."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing; build it with paper_1709_00700_gb300.build.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def __getattr__(name):  # pv_create, pv_run_pipeline, ... resolve to the C functions
    if name.startswith("pv_") and name in _SIGS:
        return getattr(load(), name)
    raise AttributeError(name)


class PVError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def variant(exec="single", agg="local", pred="branch", access="grid", ht="linear", hash="murmur",
            block=256, grid_mult=0, items_per_thread=2, threads_per_table=0, cuckoo_k=3, seed=0,
            prefetch=0, warp_agg=0, interp=0, compact_probes=1, first_items=1) -> pv_variant:
    """A pv_variant from readable names (the variant dimensions of Section 3.3).
    interp=1 runs the pipeline on the generic kernels even when a compiled
    shape matches it.  compact_probes (compacted mode): probes run over whole
    items before the survivors are queued.  first_items (compacted mode):
    items a lane takes through the first stage per trip, their loads in
    flight together."""
    return pv_variant(EXEC[exec], AGG[agg], PRED[pred], ACCESS[access], HT[ht], HASH[hash], block, grid_mult,
                      items_per_thread, threads_per_table, cuckoo_k, prefetch, warp_agg, interp, compact_probes,
                      first_items, seed)


def ht_variant(kind="linear", hash="murmur", cuckoo_k=3, max_evictions=0, load_factor=0.5, seed=0) -> pv_ht_variant:
    return pv_ht_variant(HT[kind], HASH[hash], cuckoo_k, max_evictions, load_factor, seed)


_TORCH_TYPE = None


def _type_of(t) -> int:
    import torch
    m = {torch.int32: PV_I32, torch.int64: PV_I64, torch.uint8: PV_U8}
    if t.dtype not in m:
        raise TypeError(f"unsupported column dtype {t.dtype}")
    return m[t.dtype]


# ---- dictionary-coded strings ------------------------------------------------
STR_OPS = {"lt": 0, "le": 1, "gt": 2, "ge": 3, "eq": 4, "between": 5, "prefix": 6}


class Dictionary:
    """The sorted distinct strings of a dictionary-coded column (a row's code is
    its string's rank), and the host calls that turn string predicates into code
    ranges or code sets (pv_dict_range, pv_dict_match)."""

    def __init__(self, strings):
        self.strings = [x.encode() if isinstance(x, str) else bytes(x) for x in strings]
        self._arr = (ctypes.c_char_p * max(len(self.strings), 1))(*self.strings)
        self.lib = load()

    def __len__(self):
        return len(self.strings)

    def _check(self, st):
        if st != PV_OK:
            raise PVError(st, "string dictionary: not strictly ascending, or a bad predicate")

    def range(self, op: str, s0, s1=None) -> tuple:
        """Inclusive code range of `column op s0` (or s0 <= column <= s1); (1, 0) if empty."""
        lo, hi = ctypes.c_int64(), ctypes.c_int64()
        b0 = s0.encode() if isinstance(s0, str) else bytes(s0)
        b1 = None if s1 is None else (s1.encode() if isinstance(s1, str) else bytes(s1))
        self._check(self.lib.pv_dict_range(self._arr, len(self.strings), STR_OPS[op], b0, b1,
                                           ctypes.byref(lo), ctypes.byref(hi)))
        return lo.value, hi.value

    def match(self, pattern) -> np.ndarray:
        """Ascending codes of the strings matching a SQL LIKE pattern."""
        pat = pattern.encode() if isinstance(pattern, str) else bytes(pattern)
        n = ctypes.c_int64()
        self._check(self.lib.pv_dict_match(self._arr, len(self.strings), pat, None, 0, ctypes.byref(n)))
        out = np.empty(n.value, dtype=np.int32)
        self._check(self.lib.pv_dict_match(self._arr, len(self.strings), pat,
                                           out.ctypes.data_as(_P(ctypes.c_int32)), n.value, ctypes.byref(n)))
        return out

    def codes_of(self, strings) -> np.ndarray:
        """Ascending codes of those of `strings` that are in the dictionary."""
        got = []
        for x in strings:
            lo, hi = self.range("eq", x)
            if lo <= hi:
                got.append(lo)
        return np.unique(np.array(got, dtype=np.int32))

    def decode(self, codes) -> list:
        return [self.strings[int(c)].decode() for c in codes]


def _is_string_pred(p) -> bool:
    return any(isinstance(c, (str, bytes, list, tuple)) for c in p[2:])


def _string_pred_codes(d: Dictionary, p):
    """('range', lo, hi) or ('set', codes) of a string predicate."""
    op = p[1]
    if op == "between":
        return ("range",) + d.range("between", p[2], p[3])
    if op in STR_OPS:
        return ("range",) + d.range(op, p[2])
    if op == "like":
        codes = d.match(p[2])
    elif op == "in":
        codes = d.codes_of(p[2])
    else:
        raise PVError(-1, f"bad string predicate {p}")
    if len(codes) == 0:
        return ("range", 1, 0)
    if int(codes[-1]) - int(codes[0]) + 1 == len(codes):
        return ("range", int(codes[0]), int(codes[-1]))
    return ("set", codes)


def resolve_strings(plan: dict, dicts: dict):
    """Rewrites the string predicates of a plan ([col, op, "text"...] on a column
    registered with a dictionary; dicts maps (table, column) to its Dictionary)
    into predicates on the codes.  Comparisons, BETWEEN and "prefix", and "like" /
    "in" whose codes form one range, become one code range.  Other "like" / "in"
    predicates on the fact table become a semi-join: a build pipeline over the
    matching codes (no payload) and a probe of the column, appended after the
    plan's probes.  Returns (plan, [(set table name, int32 codes)])."""
    import copy
    plan = copy.deepcopy(plan)
    sets = []
    for b in plan.get("builds", []):
        out = []
        for p in b.get("filters", []):
            if (b["table"], p[0]) in dicts and _is_string_pred(p):
                r = _string_pred_codes(dicts[(b["table"], p[0])], p)
                if r[0] == "set":
                    raise PVError(-2, f"build filter {p}: codes that are not one range")
                p = [p[0], "between", r[1], r[2]]
            out.append(p)
        b["filters"] = out
    fact = plan["fact"]
    out = []
    for p in plan.get("filters", []):
        if (fact, p[0]) in dicts and _is_string_pred(p):
            r = _string_pred_codes(dicts[(fact, p[0])], p)
            if r[0] == "range":
                out.append([p[0], "between", r[1], r[2]])
                continue
            name = f"__codes{len(sets)}"
            sets.append((name, r[1]))
            plan.setdefault("builds", []).append({"table": name, "key": "code", "filters": [], "payload": []})
            plan.setdefault("probes", []).append({"build": len(plan["builds"]) - 1, "fk": p[0]})
            continue
        out.append(p)
    plan["filters"] = out
    return plan, sets


# ---- HASH_PROBE order ----------------------------------------------------------
def _remap_ref(r, new_pos):
    if isinstance(r, (list, tuple)) and len(r) == 3 and r[0] == "payload":
        return ["payload", new_pos[int(r[1])], int(r[2])]
    return r


def reorder_probes(plan: dict, order):
    """The plan with its probes run in `order` (a permutation of the probe
    indices): the order of the HASH_PROBE operations as a variant (every order
    gives the same rows).  Payload references follow their probe.  When every
    group key is a payload, the keys are listed by probe position, so orders
    that only move the grouping dimensions reach the same compiled shape.
    Returns (plan, key_perm): new key column j holds original key key_perm[j]."""
    import copy
    probes = plan.get("probes", [])
    order = [int(o) for o in order]
    if sorted(order) != list(range(len(probes))):
        raise PVError(-1, f"probe order {order} is not a permutation of {len(probes)} probes")
    new_pos = {old: new for new, old in enumerate(order)}
    out = copy.deepcopy(plan)
    out["probes"] = [copy.deepcopy(probes[o]) for o in order]
    keys = [_remap_ref(r, new_pos) for r in plan.get("group_by", [])]
    key_perm = list(range(len(keys)))
    if keys and all(isinstance(r, list) and r[0] == "payload" for r in keys):
        key_perm = sorted(key_perm, key=lambda i: (keys[i][1], keys[i][2]))
        keys = [keys[i] for i in key_perm]
    if "group_by" in plan:
        out["group_by"] = keys
    if "aggs" in plan:
        out["aggs"] = [[a[0]] + ([[[t[0], _remap_ref(t[1], new_pos)] + list(t[2:]) for t in a[1]]] if len(a) > 1
                                 else []) for a in plan["aggs"]]
    if "project" in plan:
        out["project"] = [_remap_ref(r, new_pos) for r in plan["project"]]
    return out, key_perm


def restore_key_order(cols, key_perm):
    """Result columns of a reordered plan, with the key columns put back in the
    original plan's order."""
    nk = len(key_perm)
    keys = [None] * nk
    for new, old in enumerate(key_perm):
        keys[old] = cols[new]
    return keys + list(cols[nk:])


def probe_orders(plan: dict) -> list:
    """Every order of the plan's probes, the plan's own first."""
    import itertools
    return [tuple(o) for o in itertools.permutations(range(len(plan.get("probes", []))))]


class Context:
    """One pv_ctx on a dedicated CUDA stream, allocating through torch."""

    def __init__(self, device: int = 0, use_torch_allocator: bool = True):
        import torch
        self.torch = torch
        self.lib = load()
        self.device = device
        self.stream = torch.cuda.Stream(device=device)
        self._alloc_cb, self._free_cb = ALLOC_FN(), FREE_FN()  # NULL: libpv uses cudaMallocAsync
        if use_torch_allocator:
            dev, st = device, self.stream

            def _alloc(nbytes, _user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, st)
                except Exception:  # noqa: BLE001 - reported to C as NULL (PV_ERR_OOM)
                    return None

            def _free(ptr, _user):
                torch.cuda.caching_allocator_delete(ptr)

            self._alloc_cb, self._free_cb = ALLOC_FN(_alloc), FREE_FN(_free)
        h = ctypes.c_void_p()
        self._check(self.lib.pv_create(ctypes.byref(h), device, ctypes.c_void_p(self.stream.cuda_stream),
                                       self._alloc_cb, self._free_cb, None), ctx=None)
        self.h = h
        self.cols = {}      # (table, col) -> handle
        self.keep = {}      # (table, col) -> tensor (borrowed by libpv)
        self.tables = {}    # build key -> ht handle
        self.dicts = {}     # (table, col) -> Dictionary of a dictionary-coded column

    # -- plumbing -------------------------------------------------------------
    def _check(self, st: int, ctx="self"):
        if st != PV_OK:
            msg = "" if ctx is None else self.lib.pv_last_error(self.h).decode()
            raise PVError(st, msg)

    def close(self):
        if getattr(self, "h", None):
            self.lib.pv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def sync(self):
        self._check(self.lib.pv_sync(self.h))

    def device_info(self):
        sm, l2 = ctypes.c_int32(), ctypes.c_int64()
        self._check(self.lib.pv_device_info(self.h, ctypes.byref(sm), ctypes.byref(l2)))
        return sm.value, l2.value

    def set_l2_fetch_bytes(self, nbytes: int) -> int:
        """L2 fetch granularity of this process's CUDA context on the device
        (pv_set_l2_fetch_bytes: 32, 64 or 128); returns the previous value."""
        prev = ctypes.c_int32()
        self._check(self.lib.pv_set_l2_fetch_bytes(self.h, int(nbytes), ctypes.byref(prev)))
        return prev.value

    def last_launch_count(self) -> int:
        n = ctypes.c_int32()
        self._check(self.lib.pv_last_launch_count(self.h, ctypes.byref(n)))
        return n.value

    def set_kernel_timing(self, on: bool):
        self._check(self.lib.pv_set_kernel_timing(self.h, 1 if on else 0))

    def atomic_peak(self, slots: int, words: int, n_updates: int) -> float:
        """Milliseconds of n_updates random-slot updates (pv_atomic_peak)."""
        ms = ctypes.c_float()
        self._check(self.lib.pv_atomic_peak(self.h, slots, words, n_updates, ctypes.byref(ms)))
        return float(ms.value)

    def kernel_times(self) -> list:
        buf = (ctypes.c_float * 64)()
        n = ctypes.c_int32()
        self._check(self.lib.pv_kernel_times(self.h, buf, 64, ctypes.byref(n)))
        return [buf[i] for i in range(min(n.value, 64))]

    # -- columns ----------------------------------------------------------------
    def register_table(self, table: str, cols: dict, dicts: dict | None = None):
        """Registers device tensors (1-D, contiguous) as borrowed columns.  dicts
        maps a column holding int32 codes to its dictionary (sorted distinct
        strings, or a Dictionary): string predicates on it are then resolved by
        query()."""
        torch = self.torch
        for name, d in (dicts or {}).items():
            self.dicts[(table, name)] = d if isinstance(d, Dictionary) else Dictionary(d)
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        for name, t in cols.items():
            if not isinstance(t, torch.Tensor):
                t = torch.from_numpy(np.ascontiguousarray(t)).to(f"cuda:{self.device}")
            assert t.is_cuda and t.is_contiguous() and t.dim() == 1
            h = ctypes.c_int32()
            self._check(self.lib.pv_register_column(self.h, table.encode(), name.encode(), _type_of(t),
                                                    ctypes.c_void_p(t.data_ptr()), t.numel(), ctypes.byref(h)))
            self.cols[(table, name)] = h.value
            self.keep[(table, name)] = t
        return self

    def register_result(self, res: int, table: str, names) -> "Context":
        """Registers the columns of pipeline result `res` as table `table`
        (pv_register_result_column): names[i] for result column i.  A later
        pipeline or build over them reads what the producing pipeline wrote,
        on the device, also when the whole chain is replayed as a graph."""
        for i, name in enumerate(names):
            h = ctypes.c_int32()
            self._check(self.lib.pv_register_result_column(self.h, res, i, table.encode(), name.encode(),
                                                           ctypes.byref(h)))
            self.cols[(table, name)] = h.value
            self.keep.pop((table, name), None)
        return self

    def column_stats(self, table: str, name: str):
        lo, hi = ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.pv_column_stats(self.h, self.cols[(table, name)], ctypes.byref(lo), ctypes.byref(hi)))
        return lo.value, hi.value

    # -- builds -----------------------------------------------------------------
    def _pred(self, table, p) -> pv_pred:
        if _is_string_pred(p) or p[1] not in OPS:
            raise PVError(-1, f"predicate {p} on {table}: string predicates are resolved by query() "
                              "(or resolve_strings) on columns registered with a dictionary")
        c1 = int(p[3]) if p[1] == "between" else 0
        return pv_pred(self.cols[(table, p[0])], OPS[p[1]], int(p[2]), c1)

    def build(self, b: dict, htv: pv_ht_variant) -> int:
        spec = pv_build_spec()
        spec.key = self.cols[(b["table"], b["key"])]
        fl = b.get("filters", [])
        spec.n_preds = len(fl)
        for i, p in enumerate(fl):
            spec.preds[i] = self._pred(b["table"], p)
        pay = b.get("payload", [])
        spec.n_payload = len(pay)
        for i, c in enumerate(pay):
            spec.payload[i] = self.cols[(b["table"], c)]
        h = ctypes.c_int32()
        self._check(self.lib.pv_build_hash_table(self.h, ctypes.byref(spec), ctypes.byref(htv), ctypes.byref(h)))
        return h.value

    # -- pipelines --------------------------------------------------------------
    def spec(self, plan: dict, ht_handles=()) -> pv_pipeline_spec:
        fact = plan["fact"]
        s = pv_pipeline_spec()

        def ref(r) -> pv_ref:
            if isinstance(r, str):
                return pv_ref(REF_COL, self.cols[(fact, r)], 0)
            kind, p, i = r
            assert kind == "payload"
            return pv_ref(REF_PAYLOAD, int(p), int(i))

        fl = plan.get("filters", [])
        s.n_preds = len(fl)
        for i, p in enumerate(fl):
            s.preds[i] = self._pred(fact, p)
        pr = plan.get("probes", [])
        s.n_probes = len(pr)
        for i, q in enumerate(pr):
            s.probes[i] = pv_probe(ht_handles[q["build"]], self.cols[(fact, q["fk"])])
        keys = plan.get("group_by", [])
        s.n_keys = len(keys)
        for i, r in enumerate(keys):
            s.keys[i] = ref(r)
        aggs = plan.get("aggs", [])
        s.n_aggs = len(aggs)
        for i, a in enumerate(aggs):
            terms = a[1] if len(a) > 1 else []
            s.aggs[i].func = FUNCS[a[0]]
            s.aggs[i].n_terms = len(terms)
            for j, t in enumerate(terms):
                c = int(t[2]) if t[0] != "x" else 0
                s.aggs[i].terms[j] = pv_term(TERMS[t[0]], ref(t[1]), c)
        proj = plan.get("project", [])
        s.n_proj = len(proj)
        for i, r in enumerate(proj):
            s.proj[i] = ref(r)
        s.capacity_hint = int(plan.get("capacity_hint", 0))
        return s

    def rebuild(self, ht: int):
        self._check(self.lib.pv_rebuild_hash_table(self.h, ht))

    def build_all(self, plan: dict, htv: pv_ht_variant) -> list:
        return [self.build(b, htv) for b in plan.get("builds", [])]

    def run(self, plan: dict, var: pv_variant, ht_handles=()) -> int:
        s = self.spec(plan, ht_handles)
        h = ctypes.c_int32()
        self._check(self.lib.pv_run_pipeline(self.h, ctypes.byref(s), ctypes.byref(var), ctypes.byref(h)))
        return h.value

    def rerun(self, res: int):
        self._check(self.lib.pv_rerun(self.h, res))

    def fetch(self, res: int) -> list:
        """Result columns as numpy arrays of their result type."""
        n, m = ctypes.c_int64(), ctypes.c_int32()
        self._check(self.lib.pv_result_shape(self.h, res, ctypes.byref(n), ctypes.byref(m)))
        out = []
        for c in range(m.value):
            t = ctypes.c_int32()
            self._check(self.lib.pv_result_col_type(self.h, res, c, ctypes.byref(t)))
            out.append(np.empty(max(n.value, 1), dtype=_NP_OF[t.value]))
        if out:
            ptrs = (ctypes.c_void_p * len(out))(*[a.ctypes.data for a in out])
            rows = (ctypes.c_int64 * len(out))(*[len(a) for a in out])
            self._check(self.lib.pv_fetch_results(self.h, res, len(out), ptrs, rows, 0))
        return [a[: n.value] for a in out]

    def free(self, handle: int):
        self._check(self.lib.pv_free(self.h, handle))

    def fetch_buffers(self, res: int) -> tuple:
        """Page-locked host arrays, one per result column at the result's
        capacity, and a page-locked row count: destinations for enqueue_fetch."""
        import torch
        cap = ctypes.c_int64()
        self._check(self.lib.pv_result_capacity(self.h, res, ctypes.byref(cap)))
        cols = []
        m = self._n_cols(res)
        tmap = {PV_I32: torch.int32, PV_I64: torch.int64, PV_U8: torch.uint8}
        for c in range(m):
            t = ctypes.c_int32()
            self._check(self.lib.pv_result_col_type(self.h, res, c, ctypes.byref(t)))
            cols.append(torch.empty(max(cap.value, 1), dtype=tmap[t.value]).pin_memory())
        return cols, torch.zeros(1, dtype=torch.int64).pin_memory()

    def _n_cols(self, res: int) -> int:
        n, m = ctypes.c_int64(), ctypes.c_int32()
        # the column count needs no synchronisation: it is a property of the plan
        self._check(self.lib.pv_result_shape(self.h, res, ctypes.byref(n), ctypes.byref(m)))
        return m.value

    def enqueue_fetch(self, res: int, bufs: tuple, live_rows: bool = False):
        """pv_enqueue_fetch into fetch_buffers(res): no synchronisation; the
        values are there once the ctx stream has passed this point.  With
        live_rows, pv_enqueue_fetch_rows: a kernel copies only the result's
        live rows (the buffers must be page-locked or device memory)."""
        cols, count = bufs
        ptrs = (ctypes.c_void_p * len(cols))(*[t.data_ptr() for t in cols])
        rows = (ctypes.c_int64 * len(cols))(*[t.numel() for t in cols])
        if live_rows:
            self._check(self.lib.pv_enqueue_fetch_rows(self.h, res, len(cols), ptrs, rows,
                                                       ctypes.c_void_p(count.data_ptr())))
        else:
            on_device = 1 if count.is_cuda else 0
            if any(t.is_cuda != count.is_cuda for t in cols):
                raise ValueError("fetch buffers must all be on the host or all on the device")
            self._check(self.lib.pv_enqueue_fetch(self.h, res, len(cols), ptrs, rows,
                                                  ctypes.c_void_p(count.data_ptr()), on_device))

    def result_kernel(self, res: int) -> tuple:
        """(runs on the generic kernels, canonical shape signature) of a result."""
        g = ctypes.c_int32()
        buf = ctypes.create_string_buffer(1024)
        self._check(self.lib.pv_result_kernel(self.h, res, ctypes.byref(g), buf, len(buf)))
        return bool(g.value), buf.value.decode()

    def run_chain(self, chain: list, variants: dict | None = None, htv: pv_ht_variant | None = None) -> "Chain":
        """Runs a query of several pipelines (workloads.q5_chain format): for
        each step in order, its build pipelines (over registered tables or
        earlier steps' results), then its probe pipeline, whose result columns
        are registered as table step["name"] (pv_register_result_column).
        variants maps a step name to its pv_variant (default: variant()).
        Returns a Chain whose rerun() enqueues every build and pipeline again,
        allocation-free, so the whole query can be captured as one graph."""
        steps = []
        for st in chain:
            hts = self.build_all(st["plan"], htv or ht_variant())
            res = self.run(st["plan"], (variants or {}).get(st["name"], variant()), hts)
            self.register_result(res, st["name"], st["columns"])
            steps.append((st["name"], hts, res))
        return Chain(self, steps)


    def query(self, plan: dict, var: pv_variant, htv: pv_ht_variant | None = None, keep: bool = False,
              probe_order=None):
        """Builds, runs and fetches a whole plan; returns int64 result columns
        (grouped results sorted by key, projections as produced).  probe_order
        runs the probes in that order (reorder_probes); the result keeps the
        plan's column order.  String predicates on dictionary-coded columns are
        resolved first."""
        key_perm = None
        if probe_order is not None:
            plan, key_perm = reorder_probes(plan, probe_order)
        plan, sets = resolve_strings(plan, self.dicts)
        for name, codes in sets:
            self.register_table(name, {"code": codes})
        hts = self.build_all(plan, htv or ht_variant())
        res = self.run(plan, var, hts)
        cols = [c.astype(np.int64) for c in self.fetch(res)]
        if key_perm is not None:
            cols = restore_key_order(cols, key_perm)
        if not keep:
            self.free(res)
            for h in hts:
                self.free(h)
        nk = len(plan.get("group_by", []))
        if nk and cols and len(cols[0]):
            order = np.lexsort(tuple(cols[i] for i in reversed(range(nk))))
            cols = [c[order] for c in cols]
        return cols


class Chain:
    """The table and result handles of a multi-pipeline query run by
    Context.run_chain."""

    def __init__(self, ctx: Context, steps: list):
        self.ctx, self.steps = ctx, steps
        self.graph = None

    def rerun(self):
        """Enqueues every step again: its builds (pv_rebuild_hash_table), then
        its pipeline (pv_rerun).  No allocation, no synchronisation."""
        for _, hts, res in self.steps:
            for h in hts:
                self.ctx.rebuild(h)
            self.ctx.rerun(res)

    def capture(self) -> int:
        """Records rerun() as one CUDA graph (pv_graph_capture_*); returns its handle."""
        ctx = self.ctx
        ctx._check(ctx.lib.pv_graph_capture_begin(ctx.h))
        try:
            self.rerun()
        finally:
            g = ctypes.c_int32()
            ctx._check(ctx.lib.pv_graph_capture_end(ctx.h, ctypes.byref(g)))
        self.graph = g.value
        return self.graph

    def launch(self):
        self.ctx._check(self.ctx.lib.pv_graph_launch(self.ctx.h, self.graph))

    def fetch(self, step: int = -1) -> list:
        """Result columns of a step (the last by default), as produced."""
        return self.ctx.fetch(self.steps[step][2])

    def free(self):
        if self.graph is not None:
            self.ctx.free(self.graph)
            self.graph = None
        for _, hts, res in reversed(self.steps):
            self.ctx.free(res)
            for h in hts:
                self.ctx.free(h)
        self.steps = []
