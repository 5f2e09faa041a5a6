"""Seeded synthetic input tables (counter-based, reproducible row by row).

This module only draws inputs.  It holds none of the query arithmetic: no
predicate, hash function, join or aggregate lives here, so that the CPU oracle
and the CUDA path can both consume the same tables without sharing any code of
the method itself.

Every value is a pure function of (seed, column id, row index):

    state  = mix64(seed_key(seed, col_id) + (row + 1) * GOLDEN)
    u64    = state                       # one SplitMix64 output (Vigna, 2014)

where ``mix64`` is the SplitMix64 output finaliser.  A uniform integer in
[lo, hi) is ``lo + u64 % (hi - lo)``.  Zipf(s) ranks are drawn by inverse CDF
from a 53-bit uniform double.  Any row can therefore be regenerated alone,
and a prefix of a table is the table with fewer rows.

The table recipes follow the workloads the paper evaluates (Section 9.2.1:
projection and aggregation queries on a lineorder-like fact table, a
compute-heavy grouped aggregation like TPC-H Q1, a four-join star query like
SSB Q4.1), with shapes, sizes and value ranges chosen for this library's
configurations; the datasets themselves are not reproduced.
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
DEFAULT_SEED = 1709
_CHUNK = 1 << 22


def _mix64_inplace(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output finaliser applied in place to a uint64 array."""
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def mix64_scalar(x: int) -> int:
    """The same finaliser on one Python int (mod 2**64)."""
    m = (1 << 64) - 1
    z = x & m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


def seed_key(seed: int, col_id: int) -> int:
    """Per-column stream key derived from the global seed."""
    return mix64_scalar(mix64_scalar(seed) ^ ((col_id * 0xD1B54A32D192ED03) & ((1 << 64) - 1)))


def u64_stream(seed: int, col_id: int, n: int, start: int = 0) -> np.ndarray:
    """Rows [start, start+n) of the uint64 stream of one column."""
    out = np.empty(n, dtype=np.uint64)
    key = np.uint64(seed_key(seed, col_id))
    for lo in range(0, n, _CHUNK):
        hi = min(n, lo + _CHUNK)
        z = np.arange(start + lo + 1, start + hi + 1, dtype=np.uint64)
        z *= GOLDEN
        z += key
        out[lo:hi] = _mix64_inplace(z)
    return out


def u64_at(seed: int, col_id: int, row: int) -> int:
    """One element of :func:`u64_stream` (scalar regeneration of any row)."""
    m = (1 << 64) - 1
    return mix64_scalar((seed_key(seed, col_id) + (row + 1) * 0x9E3779B97F4A7C15) & m)


def uniform_int(seed: int, col_id: int, n: int, lo: int, hi: int, dtype=np.int64,
                start: int = 0) -> np.ndarray:
    """Uniform integers in [lo, hi) (hi exclusive), cast to ``dtype``."""
    span = hi - lo
    if span <= 0:
        raise ValueError("empty range")
    u = u64_stream(seed, col_id, n, start)
    u %= np.uint64(span)
    v = u.astype(np.int64)
    v += lo
    return v.astype(dtype, copy=False)


def uniform_double(seed: int, col_id: int, n: int, start: int = 0) -> np.ndarray:
    """53-bit uniform doubles in [0, 1)."""
    u = u64_stream(seed, col_id, n, start)
    u >>= np.uint64(11)
    return u.astype(np.float64) * (1.0 / (1 << 53))


def coprime_multiplier(g: int, start: int = 1000003) -> int:
    a = start
    while math.gcd(a, g) != 1:
        a += 2
    return a % g if g > 1 else 0


def zipf_ranks(seed: int, col_id: int, n: int, g: int, s: float = 1.0, start: int = 0) -> np.ndarray:
    """Zipf(s) ranks in [1, g] by inverse CDF over the g harmonic weights."""
    w = 1.0 / np.power(np.arange(1, g + 1, dtype=np.float64), s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    p = uniform_double(seed, col_id, n, start)
    r = np.searchsorted(cdf, p, side="right") + 1
    np.minimum(r, g, out=r)
    return r.astype(np.int64)


def zipf_keys(seed: int, col_id: int, n: int, g: int, s: float = 1.0, start: int = 0) -> np.ndarray:
    """Zipf(s) keys over the dense domain [0, g): rank r maps to ((r-1)*A + B) mod g
    with A coprime to g, so hot keys are scattered over the domain."""
    r = zipf_ranks(seed, col_id, n, g, s, start) - 1
    a = coprime_multiplier(g)
    b = (g // 3) if g > 2 else 0
    k = (r * a + b) % g if g > 1 else np.zeros_like(r)
    return k.astype(np.int32)


# ---------------------------------------------------------------------------
# Table recipes.  Column ids are fixed per recipe so that any table can be
# regenerated (or extended by rows) deterministically.
# ---------------------------------------------------------------------------

def table_filter_agg(n: int = 1_000_000, seed: int = DEFAULT_SEED) -> dict:
    """Plain filter/aggregate/project table: a, b int32 uniform [0,100);
    price int64 fixed-point uniform [100, 1e7)."""
    return {
        "a": uniform_int(seed, 101, n, 0, 100, np.int32),
        "b": uniform_int(seed, 102, n, 0, 100, np.int32),
        "price": uniform_int(seed, 103, n, 100, 10_000_000, np.int64),
    }


def table_lattice(m: int) -> dict:
    """Lattice table for closed-form checks: n = 10^4 * m rows,
    a = i mod 100, b = (i div 100) mod 100, price = 100 + i."""
    n = 10_000 * m
    i = np.arange(n, dtype=np.int64)
    return {
        "a": (i % 100).astype(np.int32),
        "b": ((i // 100) % 100).astype(np.int32),
        "price": 100 + i,
    }


DAY0 = 8035          # first day number of the date column
NDAYS = 2526         # consecutive day numbers covered


def table_lowcard_groups(n: int = 6_000_000, seed: int = DEFAULT_SEED) -> dict:
    """Low-cardinality grouped-aggregation fact table (compute-heavy
    aggregation like TPC-H Q1): date int32 over 2526 consecutive days; two
    one-byte codes with two values each (4 groups); int64 fixed-point qty
    [1,50], price [100,1e7), discount [0,10] percent, tax [0,8] percent."""
    k1 = uniform_int(seed, 202, n, 0, 2, np.int64)
    k2 = uniform_int(seed, 203, n, 0, 2, np.int64)
    return {
        "date": uniform_int(seed, 201, n, DAY0, DAY0 + NDAYS, np.int32),
        "k1": np.where(k1 == 0, ord("A"), ord("B")).astype(np.uint8),
        "k2": np.where(k2 == 0, ord("X"), ord("Y")).astype(np.uint8),
        "qty": uniform_int(seed, 204, n, 1, 51, np.int64),
        "price": uniform_int(seed, 205, n, 100, 10_000_000, np.int64),
        "disc": uniform_int(seed, 206, n, 0, 11, np.int64),
        "tax": uniform_int(seed, 207, n, 0, 9, np.int64),
    }


def table_keyval(n: int, g: int, dist: str = "uniform", seed: int = DEFAULT_SEED,
                 s: float = 1.0) -> dict:
    """High-cardinality grouped-aggregation table: key int32 over [0, g)
    (uniform or Zipf(s) with scattered hot keys), val int64 uniform [0, 1e6)."""
    if dist == "uniform":
        key = uniform_int(seed, 301, n, 0, g, np.int32)
    elif dist == "zipf":
        key = zipf_keys(seed, 302, n, g, s)
    else:
        raise ValueError(dist)
    return {"key": key, "val": uniform_int(seed, 303, n, 0, 1_000_000, np.int64)}


# Star schema: four dimensions with dense unique keys stored in a shuffled row
# order, a filter attribute f uniform [0,100) (so "f < t" keeps t percent) and,
# for the first two, a grouping attribute g.
STAR_DIMS = (("d_a", 2556, 12), ("d_b", 30_000, 25), ("d_c", 200_000, 0), ("d_d", 20_000, 0))


def star_dimension(name: str, rows: int, groups: int, seed: int = DEFAULT_SEED) -> dict:
    idx = [d[0] for d in STAR_DIMS].index(name) if name in [d[0] for d in STAR_DIMS] else 9
    cid = 400 + 10 * idx
    r = np.arange(rows, dtype=np.int64)
    a = coprime_multiplier(rows, 7919)
    t = {
        "key": ((r * a + 17) % rows).astype(np.int32),
        "f": uniform_int(seed, cid + 1, rows, 0, 100, np.int32),
    }
    if groups:
        t["g"] = uniform_int(seed, cid + 2, rows, 0, groups, np.int32)
    return t


def star_fact(n: int = 60_000_000, seed: int = DEFAULT_SEED) -> dict:
    """Fact table with four int32 foreign keys (uniform over each dimension's
    key domain) and an int64 fixed-point revenue uniform [100, 1e7)."""
    t = {}
    for j, (name, rows, _) in enumerate(STAR_DIMS):
        t["fk_" + name[2:]] = uniform_int(seed, 501 + j, n, 0, rows, np.int32)
    t["revenue"] = uniform_int(seed, 509, n, 100, 10_000_000, np.int64)
    return t


def star_schema(n: int = 60_000_000, seed: int = DEFAULT_SEED) -> dict:
    dims = {name: star_dimension(name, rows, g, seed) for name, rows, g in STAR_DIMS}
    return {"fact": star_fact(n, seed), **dims}


def table_keys3(n: int, spans=(16, 64, 7), lows=(0, 0, 1992), seed: int = DEFAULT_SEED) -> dict:
    """Composite-key table: a, b, c int32 uniform over [low_i, low_i + span_i),
    val int64 uniform over [0, 1e6)."""
    t = {name: uniform_int(seed, 311 + i, n, lo, lo + sp, np.int32)
         for i, (name, lo, sp) in enumerate(zip("abc", lows, spans))}
    t["val"] = uniform_int(seed, 314, n, 0, 1_000_000, np.int64)
    return t


# Three-dimension star schema of the SSB Q3 flight: customer and supplier
# tables carry a nation (25 values) and its region (nation // 5, 5 values), the
# date table one row per day of 7 years with its year.  Row counts are those
# of SSB at scale factor 1 (30,000 customers, 2,000 suppliers, 2,556 days).
STAR3_DIMS = (("d_cust", 30_000), ("d_supp", 2_000), ("d_date", 2_556))
STAR3_YEAR0 = 1992


# Dictionary-coded text attributes shaped like SSB's: part categories
# "MFGR#mk" and brands "MFGR#mkjj" (40 per category), and region names.  Each
# dictionary is sorted, so an attribute's int32 code is its string's rank.
SSB_REGIONS = ("AFRICA", "AMERICA", "ASIA", "EUROPE", "MIDDLE EAST")


def part_categories() -> list:
    return [f"MFGR#{m}{k}" for m in range(1, 6) for k in range(1, 6)]


def part_brands() -> list:
    return [f"MFGR#{m}{k}{j:02d}" for m in range(1, 6) for k in range(1, 6) for j in range(1, 41)]


def table_parts(n: int, seed: int = DEFAULT_SEED) -> dict:
    """category and brand int32 codes (a brand belongs to its category), price int64 uniform [100, 1e7)."""
    cat = uniform_int(seed, 701, n, 0, 25, np.int32)
    brand = (cat.astype(np.int64) * 40 + uniform_int(seed, 702, n, 0, 40, np.int64)).astype(np.int32)
    return {"category": cat, "brand": brand, "price": uniform_int(seed, 703, n, 100, 10_000_000, np.int64)}


def as_text(codes, dictionary) -> np.ndarray:
    """The strings of a dictionary-coded column."""
    return np.asarray(dictionary)[np.asarray(codes)]


def star3_dimension(name: str, seed: int = DEFAULT_SEED) -> dict:
    idx = [d[0] for d in STAR3_DIMS].index(name)
    rows = STAR3_DIMS[idx][1]
    r = np.arange(rows, dtype=np.int64)
    key = ((r * coprime_multiplier(rows, 7919) + 17) % rows).astype(np.int32)
    if name == "d_date":
        year = (STAR3_YEAR0 + np.minimum(r // 365, 6)).astype(np.int32)
        return {"key": key, "year": year}
    nation = uniform_int(seed, 601 + idx, rows, 0, 25, np.int32)
    return {"key": key, "nation": nation, "region": (nation // 5).astype(np.int32)}


def star3_fact(n: int, seed: int = DEFAULT_SEED) -> dict:
    t = {"fk_" + name[2:]: uniform_int(seed, 611 + j, n, 0, rows, np.int32)
         for j, (name, rows) in enumerate(STAR3_DIMS)}
    t["revenue"] = uniform_int(seed, 619, n, 100, 10_000_000, np.int64)
    return t


def star3_schema(n: int = 60_000_000, seed: int = DEFAULT_SEED) -> dict:
    return {"fact": star3_fact(n, seed), **{name: star3_dimension(name, seed) for name, _ in STAR3_DIMS}}


# Order-processing schema shaped like TPC-H's, for the multi-pipeline query
# (Section 9.2.1 runs TPC-H Q5, a chain of joins): 25 nations in 5 regions
# (region = nation // 5); customers, orders and line items in TPC-H's
# proportions (per scale factor 150,000 customers, 1,500,000 orders and about
# 6,000,000 line items); dense keys stored in a shuffled order; foreign keys
# uniform over the referenced keys; order dates uniform over 2,406 days from
# DAY0 (1992-01-01 .. 1998-08-02 in TPC-H); extended price int64 fixed point
# uniform [100, 1e7), discount uniform [0, 10] percent.
TPCH_DAYS = 2406


def tpch_schema(n_lineitem: int, seed: int = DEFAULT_SEED) -> dict:
    n_orders = max(1, n_lineitem // 4)
    n_cust = max(1, n_lineitem // 40)

    def shuffled_keys(rows):
        r = np.arange(rows, dtype=np.int64)
        return ((r * coprime_multiplier(rows, 7919) + 17) % rows).astype(np.int32)

    nation = np.arange(25, dtype=np.int32)
    return {
        "nation": {"n_nationkey": nation, "n_regionkey": (nation // 5).astype(np.int32)},
        "customer": {"c_custkey": shuffled_keys(n_cust), "c_nationkey": uniform_int(seed, 801, n_cust, 0, 25, np.int32)},
        "orders": {"o_orderkey": shuffled_keys(n_orders),
                   "o_custkey": uniform_int(seed, 811, n_orders, 0, n_cust, np.int32),
                   "o_orderdate": uniform_int(seed, 812, n_orders, DAY0, DAY0 + TPCH_DAYS, np.int32)},
        "lineitem": {"l_orderkey": uniform_int(seed, 821, n_lineitem, 0, n_orders, np.int32),
                     "l_extendedprice": uniform_int(seed, 822, n_lineitem, 100, 10_000_000, np.int64),
                     "l_discount": uniform_int(seed, 823, n_lineitem, 0, 11, np.int64)},
    }


# ---------------------------------------------------------------------------
# The same streams computed with torch (on any device), bit-identical to the
# numpy definitions above.  uint64 arithmetic is carried in int64 tensors:
# additions and products wrap alike; right shifts are made logical by masking;
# the unsigned remainder uses u = 2 (u >>> 1) + (u & 1).
# ---------------------------------------------------------------------------
def _i64(x: int) -> int:
    x &= (1 << 64) - 1
    return x - (1 << 64) if x >= (1 << 63) else x


def _shr(z, s: int):
    import torch
    return torch.bitwise_and(torch.bitwise_right_shift(z, s), (1 << (64 - s)) - 1)


def u64_stream_torch(seed: int, col_id: int, n: int, start: int = 0, device="cpu"):
    import torch
    z = torch.arange(start + 1, start + n + 1, dtype=torch.int64, device=device)
    z.mul_(_i64(int(GOLDEN)))
    z.add_(_i64(seed_key(seed, col_id)))
    z.bitwise_xor_(_shr(z, 30))
    z.mul_(_i64(int(_M1)))
    z.bitwise_xor_(_shr(z, 27))
    z.mul_(_i64(int(_M2)))
    z.bitwise_xor_(_shr(z, 31))
    return z


def uniform_int_torch(seed: int, col_id: int, n: int, lo: int, hi: int, dtype=None, start: int = 0, device="cpu"):
    import torch
    span = hi - lo
    u = u64_stream_torch(seed, col_id, n, start, device)
    r = torch.remainder(_shr(u, 1), span).mul_(2).add_(torch.bitwise_and(u, 1)).remainder_(span)
    r.add_(lo)
    return r.to(dtype or torch.int64)


def zipf_keys_torch(seed: int, col_id: int, n: int, g: int, s: float = 1.0, start: int = 0, device="cpu"):
    import torch
    w = 1.0 / np.power(np.arange(1, g + 1, dtype=np.float64), s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = u64_stream_torch(seed, col_id, n, start, device)
    p = _shr(u, 11).to(torch.float64).mul_(1.0 / (1 << 53))
    r = torch.searchsorted(torch.from_numpy(cdf).to(device), p, right=True)
    r = torch.clamp(r + 1, max=g) - 1
    a = coprime_multiplier(g)
    b = (g // 3) if g > 2 else 0
    k = (r * a + b) % g if g > 1 else torch.zeros_like(r)
    return k.to(torch.int32)
