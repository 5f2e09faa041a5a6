"""Dictionary-coded string predicates, pinned with no GPU.

- The C library's host translation (pv_dict_range, pv_dict_match) equals the
  brute-force code set over random sorted dictionaries.
- The oracle's string FILTER, evaluated on the strings themselves, equals the
  brute-force evaluator (its own recursive LIKE matcher).
- The binding's plan rewrite (one code range, or a semi-join over a code
  set) run by the oracle on the code columns gives the oracle's result on the
  strings.
"""
import itertools
import random

import numpy as np
import pytest

from oracle import oracle
from paper_1709_00700_gb300 import build, datagen, pv, workloads
from tests import bruteforce

UNIVERSE = ["".join(t) for n in range(4) for t in itertools.product("abc", repeat=n)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    pv.load()


def _as_lists(res):
    return [[int(v) for v in c] for c in res["cols"]]


@pytest.mark.parametrize("seed", range(60))
def test_dict_range_is_the_brute_force_code_set(seed):
    rng = random.Random(seed)
    d = sorted(rng.sample(UNIVERSE, rng.randint(0, 20)))
    dic = pv.Dictionary(d)
    for _ in range(40):
        op = rng.choice(["lt", "le", "gt", "ge", "eq", "between", "prefix"])
        c0, c1 = rng.choice(UNIVERSE), rng.choice(UNIVERSE)
        lo, hi = dic.range(op, c0, c1 if op == "between" else None)
        got = list(range(lo, hi + 1)) if lo <= hi else []
        want = [i for i, s in enumerate(d) if bruteforce._holds(s, [None, op, c0, c1])]
        assert got == want, (d, op, c0, c1)


@pytest.mark.parametrize("seed", range(60))
def test_dict_match_is_the_brute_force_like(seed):
    rng = random.Random(seed)
    d = sorted(rng.sample(UNIVERSE, rng.randint(0, 25)))
    dic = pv.Dictionary(d)
    for _ in range(40):
        pat = "".join(rng.choice("abc%_") for _ in range(rng.randint(0, 5)))
        want = [i for i, s in enumerate(d) if bruteforce.like(s, pat)]
        assert dic.match(pat).tolist() == want, (d, pat)


def test_dictionary_must_be_strictly_ascending():
    for bad in (["b", "a"], ["a", "a"]):
        with pytest.raises(pv.PVError) as e:
            pv.Dictionary(bad).range("eq", "a")
        assert e.value.status == -1


def _text_case(rng: random.Random):
    nf, nd = rng.randint(0, 40), rng.randint(0, 8)
    words = rng.sample(UNIVERSE, 12)
    dim = {"key": np.array(rng.sample(range(-4, 12), nd), np.int32),
           "t": np.array([rng.choice(words) for _ in range(nd)], dtype=object),
           "g": np.array([rng.randint(-2, 2) for _ in range(nd)], np.int32)}
    fact = {"s": np.array([rng.choice(words) for _ in range(nf)], dtype=object),
            "fk": np.array([rng.randint(-4, 12) for _ in range(nf)], np.int32),
            "k": np.array([rng.randint(0, 2) for _ in range(nf)], np.int32),
            "v": np.array([rng.randint(-1000, 1000) for _ in range(nf)], np.int64)}

    def pred(col):
        op = rng.choice(["lt", "le", "gt", "ge", "eq", "between", "prefix", "like", "in"])
        if op == "between":
            return [col, op, rng.choice(UNIVERSE), rng.choice(UNIVERSE)]
        if op == "like":
            return [col, op, "".join(rng.choice("abc%_") for _ in range(rng.randint(0, 4)))]
        if op == "in":
            return [col, op, rng.sample(UNIVERSE, rng.randint(0, 4))]
        return [col, op, rng.choice(UNIVERSE)]

    plan = {"fact": "f", "filters": [pred("s") for _ in range(rng.randint(0, 2))],
            "aggs": [["count"], ["sum", [["x", "v"]]]]}
    if rng.random() < 0.5:
        plan["builds"] = [{"table": "d", "key": "key", "filters": [pred("t")] if rng.random() < 0.7 else [],
                           "payload": ["g"]}]
        plan["probes"] = [{"build": 0, "fk": "fk"}]
    if rng.random() < 0.6:
        plan["group_by"] = ["k"] if rng.random() < 0.5 or "probes" not in plan else ["k", ["payload", 0, 0]]
    return plan, {"f": fact, "d": dim}


@pytest.mark.parametrize("seed", range(150))
def test_oracle_string_filters_match_bruteforce(seed):
    plan, tables = _text_case(random.Random(seed))
    assert _as_lists(oracle.run(plan, tables)) == bruteforce.evaluate(plan, tables)["cols"]


def _parts(n, seed):
    codes = datagen.table_parts(n, seed=seed)
    cats, brands = datagen.part_categories(), datagen.part_brands()
    text = {"category": datagen.as_text(codes["category"], cats), "brand": datagen.as_text(codes["brand"], brands),
            "price": codes["price"]}
    dicts = {("parts", "category"): pv.Dictionary(cats), ("parts", "brand"): pv.Dictionary(brands)}
    return codes, text, dicts


# (filters, whether the rewrite needs a semi-join)
TEXT_FILTERS = [
    ((("category", "eq", "MFGR#12"), ("brand", "between", "MFGR#1221", "MFGR#1228")), False),
    ((("category", "ge", "MFGR#3"), ("brand", "prefix", "MFGR#3")), False),
    ((("category", "lt", "MFGR#2"), ("brand", "like", "MFGR#1%")), False),           # a LIKE that is one range
    ((("category", "in", ["MFGR#21", "MFGR#22", "MFGR#23"]), ("brand", "gt", "MFGR#2150")), False),
    ((("category", "eq", "MFGR#99"), ("brand", "le", "MFGR#5540")), False),          # a constant not present
    ((("category", "le", "MFGR#55"), ("brand", "like", "MFGR#_2_5")), True),         # 20 scattered codes
    ((("category", "gt", "MFGR#1"), ("brand", "in", ["MFGR#1101", "MFGR#3340", "nope"])), True),
    ((("brand", "like", "%9"),), True),
]


@pytest.mark.parametrize("filters,semi", TEXT_FILTERS)
def test_resolved_plan_on_codes_equals_oracle_on_strings(filters, semi):
    codes, text, dicts = _parts(20_000, seed=5)
    plan = workloads.parts_text_plan(filters)
    rp, sets = pv.resolve_strings(plan, dicts)
    assert all(not pv._is_string_pred(p) for p in rp["filters"])
    assert bool(sets) == semi
    on_codes = oracle.run(rp, {"parts": codes, **{name: {"code": c} for name, c in sets}})
    on_text = oracle.run(plan, {"parts": text})
    assert _as_lists(on_codes) == _as_lists(on_text)
    assert on_text["cols"][1][0] > 0 or filters[0][2] == "MFGR#99"


def test_resolved_build_filters_equal_oracle_on_strings():
    # the SSB Q3.1-shaped join with its region filters written as strings
    n = 30_000
    s = datagen.star3_schema(n, seed=9)
    text = {t: dict(c) for t, c in s.items()}
    dicts = {}
    for d in ("d_cust", "d_supp"):
        text[d]["region"] = datagen.as_text(s[d]["region"], datagen.SSB_REGIONS)
        dicts[(d, "region")] = pv.Dictionary(datagen.SSB_REGIONS)
    plan = workloads.star3_plan(regions=("ASIA", "EUROPE"))
    rp, sets = pv.resolve_strings(plan, dicts)
    assert not sets and rp["builds"][0]["filters"] == [["region", "between", 2, 2]]
    got = oracle.run(rp, s)
    assert _as_lists(got) == _as_lists(oracle.run(plan, text))
    assert _as_lists(got) == _as_lists(oracle.run(workloads.star3_plan(regions=(2, 3)), s))
    with pytest.raises(pv.PVError) as e:  # a code set that is not one range cannot filter a build
        pv.resolve_strings(workloads.star3_plan(regions=("ASIA", "EUROPE")) | {"builds": [
            dict(plan["builds"][0], filters=[["region", "in", ["AFRICA", "EUROPE"]]])] + plan["builds"][1:]}, dicts)
    assert e.value.status == -2
