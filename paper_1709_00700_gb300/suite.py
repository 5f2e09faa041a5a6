"""Variant-selection suite: seeded random queries, exhaustive timing, the
per-workload configuration of Algorithm 1, and the learned per-query pick.

Three query families shaped like the evaluated pipelines (Section 9.2.1):
  filter  -- WHERE a < A AND B0 <= b <= B1 -> SUM(price), COUNT(*) or the
             projection (a, price);
  grouped -- SUM(val), COUNT(*) WHERE val < T GROUP BY key, G groups,
             uniform or Zipf(1) keys;
  star    -- four-probe star join with per-dimension filters, grouped on two
             dimension attributes.
Rows are log-uniform in [min_rows, max_rows], the selectivity log-uniform in
[0.001, 0.9] and the group count log-uniform in [1, 1e7].  The data are
prefixes of one base table per family generated on the GPU (the grouped
family's key column is generated per query).

For every query the whole variant grid of its family is timed (exhaustive
search); the network is trained on the timings of the training queries and
judged on the held-out ones by t(pick) / t(best).  The same held-out queries
run under the per-family configuration Algorithm 1 learns from the training
queries (the method without the network).
"""
from __future__ import annotations

import itertools
import json
import math
import time

import numpy as np

from . import autotune, costmodel, datagen, pv, workloads

SAMPLE_ROWS = 65_536

GRIDS = {
    "filter_aggregate": [dict(pred=p, access=a, items_per_thread=u, block=b, prefetch=f)
                         for p, a, u, b, f in itertools.product(["branch", "predicated"], ["grid", "chunked"],
                                                                [1, 4], [256, 512], [0, 1])] +
                        [dict(pred="compacted", access="grid", items_per_thread=u, block=b, prefetch=f)
                         for u, b, f in itertools.product([1, 2], [256, 512], [0, 1])] +
                        # two items per lane through the first stage, their loads in flight together
                        [dict(pred="compacted", access="grid", items_per_thread=u, block=b, prefetch=0, first_items=2)
                         for u, b in itertools.product([1, 2], [256, 512])],
    "filter_project": [dict(exec=e, pred=p, access=a, items_per_thread=u, block=256, prefetch=f)
                       for e, p, a, u, f in itertools.product(["single", "multi"], ["branch", "predicated"],
                                                              ["grid", "chunked"], [1, 4], [0, 1])] +
                      [dict(exec="single", pred="compacted", access="grid", items_per_thread=u, block=256, prefetch=f)
                       for u, f in itertools.product([1, 2], [0, 1])] +
                      [dict(exec="single", pred="compacted", access="grid", items_per_thread=u, block=256, prefetch=0,
                            first_items=2) for u in (1, 2)],
    "grouped": [dict(s, pred=p, items_per_thread=1, block=256, prefetch=f)
                for s, p, f in itertools.product(
                    [dict(agg="local", ht="perfect"), dict(agg="local", ht="perfect", threads_per_table=1),
                     dict(agg="global", ht="perfect"), dict(agg="local", ht="linear"),
                     dict(agg="global", ht="linear"), dict(agg="global", ht="linear", exec="multi"),
                     dict(agg="global", ht="cuckoo", exec="multi"), dict(agg="local", ht="cuckoo", exec="multi")],
                    ["branch", "predicated"], [0, 1])] +
               # warp pre-aggregation before the global tables (hot keys)
               [dict(s, pred=p, items_per_thread=1, block=256, prefetch=1, warp_agg=1)
                for s, p in itertools.product(
                    [dict(agg="global", ht="perfect"), dict(agg="global", ht="linear"),
                     dict(agg="global", ht="linear", exec="multi"), dict(agg="global", ht="cuckoo", exec="multi")],
                    ["branch", "predicated"])] +
               # rows passing the filter queued per warp, taken 1 or 2 per lane
               [dict(s, pred="compacted", items_per_thread=u, block=256, prefetch=0)
                for s, u in itertools.product([dict(agg="local", ht="perfect"), dict(agg="global", ht="perfect"),
                                               dict(agg="local", ht="linear"), dict(agg="global", ht="linear")],
                                              [1, 2])] +
               [dict(s, pred="compacted", items_per_thread=u, block=256, prefetch=0, first_items=2)
                for s, u in itertools.product([dict(agg="local", ht="perfect"), dict(agg="global", ht="perfect")],
                                              [1, 2])] +
               # perfect array in the distributed shared memory of a cluster of 2 to 16 CTAs
               [dict(agg="cluster", ht="perfect", pred="branch", items_per_thread=1, block=512, prefetch=0,
                     warp_agg=w) for w in (0, 1)] +
               # CTA-local perfect arrays past 113 KB leave room for one CTA per SM: 1024 threads keep it busy
               [dict(agg="local", ht="perfect", pred="branch", items_per_thread=1, block=1024, prefetch=f)
                for f in (0, 1)],
    "star": [dict(s, build=bk, pred=p, items_per_thread=1, block=512, prefetch=f)
             for bk, s, p, f in itertools.product(
                 ["perfect", "linear", "cuckoo"],
                 [dict(agg="local", ht="perfect"), dict(agg="global", ht="perfect"),
                  dict(agg="local", ht="linear"), dict(agg="global", ht="linear")],
                 ["branch", "predicated"], [0, 1])] +
            [dict(s, build=bk, pred="compacted", items_per_thread=u, block=512, prefetch=0)
             for bk, s, u in itertools.product(
                 ["perfect", "linear", "cuckoo"],
                 [dict(agg="local", ht="perfect"), dict(agg="global", ht="perfect"),
                  dict(agg="local", ht="linear"), dict(agg="global", ht="linear")], [1, 2, 4])] +
            # the first two probes over whole items (second key column read in full), then the queue
            [dict(s, build=bk, pred="compacted", items_per_thread=u, block=256, prefetch=0, compact_probes=2)
             for bk, s, u in itertools.product(
                 ["perfect", "linear"], [dict(agg="local", ht="perfect"), dict(agg="global", ht="perfect")], [1, 2])],
}


_DEFAULTS = {"exec": "single", "threads_per_table": 0, "warp_agg": 0, "compact_probes": 1, "first_items": 1}


def _normalize(grid: list) -> list:
    """Same keys in every variant of a grid (missing ones take their default)."""
    keys = []
    for v in grid:
        keys += [k for k in v if k not in keys]
    return [{k: v.get(k, _DEFAULTS.get(k)) for k in keys} for v in grid]


GRIDS = {g: _normalize(v) for g, v in GRIDS.items()}


def grid_key(q: dict) -> str:
    if q["family"] == "filter":
        return "filter_" + q["kind"]
    return q["family"]


def make_queries(n: int = 500, seed: int = 1709, min_rows: int = 1_000_000, max_rows: int = 300_000_000) -> list:
    rng = np.random.default_rng(seed)
    qs = []
    for i in range(n):
        fam = ("filter", "grouped", "star")[i % 3]
        rows = int(math.exp(rng.uniform(math.log(min_rows), math.log(max_rows))))
        rows -= rows % 4
        sel = math.exp(rng.uniform(math.log(0.001), math.log(0.9)))
        q = {"id": i, "family": fam, "rows": rows, "sel_target": sel}
        if fam == "filter":
            q["kind"] = "aggregate" if rng.random() < 0.5 else "project"
            # a < A keeps A %, B0 <= b <= B1 keeps (B1 - B0 + 1) %
            # fraction kept by a, chosen so that b keeps between 1 and 100 percent
            fa = math.exp(rng.uniform(math.log(max(sel, 0.01)), math.log(min(1.0, 100 * sel))))
            A = int(np.clip(round(100 * fa), 1, 100))
            nb = int(np.clip(round(100 * sel / (A / 100)), 1, 100))
            b0 = int(rng.integers(0, 101 - nb))
            q.update(A=A, B0=b0, B1=b0 + nb - 1)
        elif fam == "grouped":
            G = int(math.exp(rng.uniform(0.0, math.log(1e7))))
            q.update(G=max(1, G), dist="zipf" if rng.random() < 0.5 else "uniform",
                     T=int(np.clip(round(sel * 1_000_000), 1, 1_000_000)))
        else:
            # per-dimension thresholds whose product is about the target selectivity
            parts = rng.dirichlet(np.ones(4)) * math.log(sel)
            q["th"] = {d: int(np.clip(round(100 * math.exp(x)), 1, 100))
                       for d, x in zip(("d_a", "d_b", "d_c", "d_d"), parts)}
        qs.append(q)
    return qs


class SuiteData:
    """Base tables on the device and per-query plans over their prefixes."""

    def __init__(self, ctx: "pv.Context", max_rows: int, seed: int = datagen.DEFAULT_SEED):
        import torch
        self.torch = torch
        self.ctx = ctx
        dev = f"cuda:{ctx.device}"
        self.dev = dev
        self.max_rows = max_rows
        self.seed = seed
        u = datagen.uniform_int_torch
        self.filter = {"a": u(seed, 101, max_rows, 0, 100, torch.int32, device=dev),
                       "b": u(seed, 102, max_rows, 0, 100, torch.int32, device=dev),
                       "price": u(seed, 103, max_rows, 100, 10_000_000, torch.int64, device=dev)}
        self.val = u(seed, 303, max_rows, 0, 1_000_000, torch.int64, device=dev)
        self.key = torch.empty(max_rows, dtype=torch.int32, device=dev)
        self.key_of = None
        self.fact = {"fk_" + name[2:]: u(seed, 501 + j, max_rows, 0, rows, torch.int32, device=dev)
                     for j, (name, rows, _) in enumerate(datagen.STAR_DIMS)}
        self.fact["revenue"] = u(seed, 509, max_rows, 100, 10_000_000, torch.int64, device=dev)
        for name, rows, g in datagen.STAR_DIMS:
            d = datagen.star_dimension(name, rows, g, seed)
            ctx.register_table(name, {c: torch.from_numpy(v).to(dev) for c, v in d.items()})

    def _keys(self, q):
        if self.key_of != (q["G"], q["dist"]):
            torch = self.torch
            n = self.max_rows
            if q["dist"] == "uniform":
                k = datagen.uniform_int_torch(self.seed, 301, n, 0, q["G"], torch.int32, device=self.dev)
            else:
                k = datagen.zipf_keys_torch(self.seed, 302, n, q["G"], device=self.dev)
            self.key.copy_(k)
            del k
            self.key_of = (q["G"], q["dist"])
        return self.key

    def prepare(self, q: dict, rows: int | None = None) -> dict:
        """Registers the query's fact table (a prefix of `rows` rows) as
        table "q" and returns its plan."""
        r = q["rows"] if rows is None else rows
        if q["family"] == "filter":
            self.ctx.register_table("q", {c: t[:r] for c, t in self.filter.items()})
            plan = {"fact": "q", "filters": [["a", "lt", q["A"]], ["b", "between", q["B0"], q["B1"]]]}
            if q["kind"] == "aggregate":
                plan["aggs"] = [["sum", [["x", "price"]]], ["count"]]
            else:
                plan["project"] = ["a", "price"]
            return plan
        if q["family"] == "grouped":
            self.ctx.register_table("q", {"key": self._keys(q)[:r], "val": self.val[:r]})
            return {"fact": "q", "filters": [["val", "lt", q["T"]]], "group_by": ["key"],
                    "aggs": [["sum", [["x", "val"]]], ["count"]]}
        self.ctx.register_table("q", {c: t[:r] for c, t in self.fact.items()})
        plan = workloads.star_plan(q["th"])
        plan["fact"] = "q"
        return plan

    def stats(self, q: dict) -> dict:
        """Plan features and column statistics, from the plan and from
        pipelines run on the first SAMPLE_ROWS rows (sample selectivity, group
        count and hottest-group share) through libpv."""
        ctx = self.ctx
        n = min(SAMPLE_ROWS, q["rows"])
        st = {"rows": q["rows"], "family": q["family"], "n_preds": 0, "n_probes": 0, "dim_rows": 0,
              "n_aggs": 2, "project": 0, "groups": 1, "top_share": 1.0}
        if q["family"] == "filter":
            plan = self.prepare(q, n)
            cnt = int(ctx.query(dict(plan, project=[], aggs=[["sum", [["x", "price"]]], ["count"]]),
                                pv.variant())[1][0])
            st.update(sel=max(cnt, 0.5) / n, n_preds=2, bytes_in=16, project=int(q["kind"] == "project"),
                      bytes_out=12 if q["kind"] == "project" else 0)
        elif q["family"] == "grouped":
            plan = self.prepare(q, n)
            cols = ctx.query(plan, pv.variant(agg="global", ht="linear", items_per_thread=1))
            counts = cols[2]
            tot = int(counts.sum())
            self.prepare(q)
            lo, hi = ctx.column_stats("q", "key")
            st.update(sel=max(tot, 0.5) / n, n_preds=1, bytes_in=12, bytes_out=0,
                      groups=min(hi - lo + 1, q["rows"]), top_share=float(counts.max()) / max(tot, 1),
                      collision=_collision(counts))
        else:
            plan = self.prepare(q, n)
            cols = ctx.query(plan, pv.variant(items_per_thread=1, ht="linear"), pv.ht_variant("linear"))
            counts = cols[3]
            tot = int(counts.sum())
            # rows surviving the first probe alone (what compacted execution queues)
            b0 = plan["builds"][plan["probes"][0]["build"]]
            first = {"fact": plan["fact"], "builds": [b0], "probes": [{"build": 0, "fk": plan["probes"][0]["fk"]}],
                     "aggs": [["count"]]}
            c1 = int(ctx.query(first, pv.variant(items_per_thread=1), pv.ht_variant("perfect"))[0][0])
            st["sel_first"] = max(c1, 0.5) / n
            st.update(sel=max(tot, 0.5) / n, n_probes=4, bytes_in=24, bytes_out=0,
                      dim_rows=sum(r for _, r, _ in datagen.STAR_DIMS), groups=max(len(counts), 1),
                      top_share=float(counts.max()) / max(tot, 1) if tot else 0.0, collision=_collision(counts))
        return st


def _collision(counts) -> float:
    """Probability that two surviving rows drawn at random share a group
    (sum of squared group shares), from the sample's group counts."""
    c = np.asarray(counts, dtype=np.float64)
    t = c.sum()
    return float(((c / t) ** 2).sum()) if t > 0 else 1.0


def time_query(data: SuiteData, q: dict, reps: int = 3) -> dict:
    """Exhaustive timing of the query's grid; returns {variant key: ms}."""
    plan = data.prepare(q)
    grid = GRIDS[grid_key(q)]
    out = {}
    if q["family"] == "star":
        for bk in ("perfect", "linear", "cuckoo"):
            m = autotune.Measurer(data.ctx, plan, build_ht=bk, reps=reps)
            for v in grid:
                if v["build"] == bk:
                    vv = {k: x for k, x in v.items() if k != "build"}
                    out[autotune.variant_key(v)] = m(vv)
            m.close()
    else:
        m = autotune.Measurer(data.ctx, plan, reps=reps)
        for v in grid:
            out[autotune.variant_key(v)] = m(v)
        m.close()
    return out


def algorithm1_config(train: list, timings: dict, grid: list, q_sweeps: int = 3, counts: dict | None = None,
                      name: str = "") -> dict:
    """Per-workload configuration (Section 8.3): Algorithm 1 over the grid's
    dimensions with the workload time = the sum of the training queries'
    times (looked up from the exhaustive timings; a variant missing from the
    grid costs infinity)."""
    names = list(grid[0].keys())
    dims = []
    for n in names:
        vals = []
        for v in grid:
            if v[n] not in vals:
                vals.append(v[n])
        dims.append((n, vals))
    keys = {autotune.variant_key(v) for v in grid}
    evaluated = set()

    def cost(v):
        k = autotune.variant_key(v)
        evaluated.add(k)
        if k not in keys:
            return math.inf
        return sum(timings[q["id"]].get(k, math.inf) for q in train)

    v, c, n = autotune.feature_wise(cost, dims, q=q_sweeps)
    if counts is not None:
        counts[name] = sum(1 for k in evaluated if k in keys)
    return v


def explore(ctx: "pv.Context", n_queries: int = 500, max_rows: int = 300_000_000, min_rows: int = 1_000_000,
            seed: int = 1709, reps: int = 3, log=print, data: "SuiteData | None" = None) -> dict:
    """Statistics and exhaustive timings of every query of the suite."""
    t0 = time.time()
    queries = make_queries(n_queries, seed, min_rows, max_rows)
    data = data or SuiteData(ctx, max_rows)
    stats, timings = {}, {}
    for i, q in enumerate(queries):
        stats[q["id"]] = data.stats(q)
        timings[q["id"]] = time_query(data, q, reps)
        if log and (i % 25 == 0 or i == len(queries) - 1):
            log(f"  timed {i + 1}/{len(queries)} queries, {time.time() - t0:.0f}s")
    return {"queries": queries, "stats": stats, "timings": timings, "exploration_s": time.time() - t0,
            "seed": seed}


CANDIDATES = ((20000, 5, 1e-3), (30000, 8, 1e-3), (10000, 5, 2e-3))


def _rows(qs, stats, timings):
    X, y = [], []
    for q in qs:
        for v in GRIDS[grid_key(q)]:
            ms = timings[q["id"]].get(autotune.variant_key(v), math.inf)
            if math.isfinite(ms):
                X.append(costmodel.features(stats[q["id"]], v))
                y.append(math.log(ms))
    return np.array(X), np.array(y)


def _fit(ctx, X, y, epochs, ensemble, lr, seed):
    nets, hists = [], []
    for e in range(ensemble):
        net = costmodel.Net(ctx, costmodel.N_FEATURES, seed=seed + 17 * e)
        net.fit_standardisation(X)
        hists.append(net.train(X, y, epochs=epochs, lr=lr, report_every=max(1, epochs // 10)))
        nets.append(net)
    return costmodel.Ensemble(nets), hists[0]


def _evaluate(model, qs, stats, timings, configs=None, top_k=3):
    out = []
    for q in qs:
        tm = timings[q["id"]]
        finite = [v for v in GRIDS[grid_key(q)] if math.isfinite(tm.get(autotune.variant_key(v), math.inf))]
        best = min(tm[autotune.variant_key(v)] for v in finite)
        pick, pred = costmodel.pick(model, stats[q["id"]], finite)
        ranked = [finite[i] for i in np.argsort(pred)[:top_k]]
        r = {"id": q["id"], "family": grid_key(q), "rows": q["rows"], "best_ms": best,
             "pick_ms": tm[autotune.variant_key(pick)], "topk_ms": min(tm[autotune.variant_key(v)] for v in ranked),
             "pick": pick}
        if configs is not None:
            r["config_ms"] = tm.get(autotune.variant_key(configs[grid_key(q)]), math.inf)
        out.append(r)
    return out


def assess(ctx: "pv.Context", ex: dict, n_train: int | None = None, candidates=CANDIDATES, top_k: int = 3,
          n_val: int | None = None) -> dict:
    """Trains the cost model on the training queries' timings and judges its
    picks on the held-out queries against the exhaustive best, beside the
    per-family configuration of Algorithm 1.  The training settings (epochs,
    ensemble size, learning rate) are chosen among `candidates` on a
    validation split of the training queries; the held-out queries are used
    once, by the final model trained on all training queries."""
    queries, stats, timings = ex["queries"], ex["stats"], ex["timings"]
    seed = ex.get("seed", 1709)
    rng = np.random.default_rng(seed + 1)
    order = rng.permutation(len(queries))
    n_train = n_train if n_train is not None else int(round(0.8 * len(queries)))
    train = [queries[i] for i in order[:n_train]]
    test = [queries[i] for i in order[n_train:]]
    n_val = n_val if n_val is not None else len(train) // 5
    fit_part, val_part = train[:-n_val], train[-n_val:]
    t1 = time.time()
    validation = []
    if len(candidates) > 1 and n_val > 0:
        Xf, yf = _rows(fit_part, stats, timings)
        for epochs, ens, lr in candidates:
            model, _ = _fit(ctx, Xf, yf, epochs, ens, lr, seed)
            res = _evaluate(model, val_part, stats, timings)
            r = np.array([p["pick_ms"] / p["best_ms"] for p in res])
            validation.append({"epochs": epochs, "ensemble": ens, "lr": lr,
                               "within_10pct": float(np.mean(r <= 1.10)),
                               "geomean": float(np.exp(np.mean(np.log(r))))})
        best = max(validation, key=lambda c: (c["within_10pct"], -c["geomean"]))
        chosen = (best["epochs"], best["ensemble"], best["lr"])
    else:
        chosen = candidates[0]
    X, y = _rows(train, stats, timings)
    model, hist = _fit(ctx, X, y, *chosen, seed)
    t_train = time.time() - t1
    alg1_runs = {}
    configs = {g: algorithm1_config([q for q in train if grid_key(q) == g], timings, GRIDS[g], counts=alg1_runs, name=g)
               for g in GRIDS}
    per_query = _evaluate(model, test, stats, timings, configs, top_k)
    r_pick = np.array([p["pick_ms"] / p["best_ms"] for p in per_query])
    r_topk = np.array([p["topk_ms"] / p["best_ms"] for p in per_query])
    r_cfg = np.array([p["config_ms"] / p["best_ms"] for p in per_query])
    gm = lambda r: float(np.exp(np.mean(np.log(np.minimum(r, 1e6)))))  # noqa: E731
    return {
        "queries": len(queries), "train": len(train), "held_out": len(test),
        "grid_sizes": {g: len(v) for g, v in GRIDS.items()},
        "exploration_s": ex.get("exploration_s"), "train_s": t_train, "train_rows": len(X),
        "validation": validation, "chosen": {"epochs": chosen[0], "ensemble": chosen[1], "lr": chosen[2]},
        "loss_history": hist,
        "mlp_within_10pct": float(np.mean(r_pick <= 1.10)), "mlp_geomean_slowdown": gm(r_pick),
        "mlp_worst_slowdown": float(r_pick.max()),
        f"mlp_top{top_k}_within_10pct": float(np.mean(r_topk <= 1.10)),
        f"mlp_top{top_k}_geomean_slowdown": gm(r_topk),
        "alg1_within_10pct": float(np.mean(r_cfg <= 1.10)), "alg1_geomean_slowdown": gm(r_cfg),
        "alg1_worst_slowdown": float(r_cfg.max()), "alg1_configs": configs,
        "alg1_variants_run": alg1_runs, "per_query": per_query,
    }


def confirm(data: SuiteData, ex: dict, summary: dict, reps: int = 15, top: int = 3, log=print) -> dict:
    """Re-times, for every held-out query, the exploration's `top` fastest
    variants, the network's pick and the Algorithm 1 configuration with the
    median of `reps` cold-L2 runs each, and judges the pick and the
    configuration against the fastest of them.  The exploration's own best is
    the minimum of many 3-run medians (biased low by selection) and, for
    queries of tens of microseconds, of times quantised by the event timer;
    re-timing the candidates removes both effects from the assessment."""
    t0 = time.time()
    qmap = {q["id"]: q for q in ex["queries"]}
    rows = []
    for n, p in enumerate(summary["per_query"]):
        q = qmap[p["id"]]
        g = grid_key(q)
        tm = ex["timings"][q["id"]]
        finite = sorted((v for v in GRIDS[g] if math.isfinite(tm.get(autotune.variant_key(v), math.inf))),
                        key=lambda v: tm[autotune.variant_key(v)])
        cands = {}
        for v in finite[:top] + [p["pick"], summary["alg1_configs"][g]]:
            cands.setdefault(autotune.variant_key(v), v)
        plan = data.prepare(q)
        med = {}
        for bk in sorted({v.get("build", "") for v in cands.values()}):
            m = autotune.Measurer(data.ctx, plan, build_ht=bk or "perfect", reps=reps, cap_factor=math.inf)
            for k, v in cands.items():
                if v.get("build", "") == bk:
                    med[k] = m({kk: x for kk, x in v.items() if kk != "build"})
            m.close()
        best = min(med.values())
        rows.append({"id": q["id"], "family": g, "best_ms": best,
                     "pick_ratio": med[autotune.variant_key(p["pick"])] / best,
                     "config_ratio": med[autotune.variant_key(summary["alg1_configs"][g])] / best})
        if log and (n % 25 == 0 or n == len(summary["per_query"]) - 1):
            log(f"  confirmed {n + 1}/{len(summary['per_query'])} queries, {time.time() - t0:.0f}s")
    rp = np.array([r["pick_ratio"] for r in rows])
    rc = np.array([r["config_ratio"] for r in rows])
    gm = lambda r: float(np.exp(np.mean(np.log(np.minimum(r, 1e6)))))  # noqa: E731
    return {"reps": reps, "candidates": f"the exploration's {top} fastest, the pick, the Algorithm 1 configuration",
            "mlp_within_10pct": float(np.mean(rp <= 1.10)), "mlp_geomean_slowdown": gm(rp),
            "mlp_worst_slowdown": float(rp.max()), "alg1_within_10pct": float(np.mean(rc <= 1.10)),
            "alg1_geomean_slowdown": gm(rc), "alg1_worst_slowdown": float(rc.max()), "seconds": time.time() - t0,
            "per_query": rows}


def online_experiment(ctx: "pv.Context", ex: dict, n_seed: int = 100, tail: int = 100, seed_epochs: int = 10000,
                      ensemble: int = 3, lr: float = 2e-3, every: int = 16, steps: int = 400,
                      explore: float = 0.1, observe_top: int = 1, shadow_frac: float = 1.0,
                      update_lr: float = 5e-4) -> dict:
    """Run-time re-tuning: a network trained on the first n_seed queries (all
    their variants timed) then meets the other queries one at a time, in a
    seeded random order.  For each it picks a variant, observes that
    variant's time (from the exhaustive timings) and, with observe_top > 1,
    the times of its runner-ups (shadow runs), and learns from them
    (costmodel.OnlineTuner).  Over the last `tail` queries of the stream, the
    online picks are judged against the exhaustive best beside the picks of
    the seed network left as it was."""
    queries, stats, timings = ex["queries"], ex["stats"], ex["timings"]
    rng = np.random.default_rng(ex.get("seed", 1709) + 7)
    order = [queries[i] for i in rng.permutation(len(queries))]
    seed_qs, stream = order[:n_seed], order[n_seed:]
    X, y = _rows(seed_qs, stats, timings)
    static, _ = _fit(ctx, X, y, seed_epochs, ensemble, lr, 1709)
    online, _ = _fit(ctx, X, y, seed_epochs, ensemble, lr, 1709)
    tuner = costmodel.OnlineTuner(online, X, y, every=every, steps=steps, lr=update_lr, explore=explore,
                                  observe_top=observe_top, shadow_frac=shadow_frac)
    t0 = time.time()
    r_static, r_online = [], []
    for q in stream:
        tm = timings[q["id"]]
        finite = [v for v in GRIDS[grid_key(q)] if math.isfinite(tm.get(autotune.variant_key(v), math.inf))]
        best = min(tm[autotune.variant_key(v)] for v in finite)
        v = tuner.choose(stats[q["id"]], finite)
        ms = tm[autotune.variant_key(v)]
        shadows = [(s_, tm[autotune.variant_key(s_)]) for s_ in tuner.shadow_candidates(v)]
        tuner.observe(stats[q["id"]], v, ms, shadows)
        r_online.append(ms / best)
        p, _ = costmodel.pick(static, stats[q["id"]], finite)
        r_static.append(tm[autotune.variant_key(p)] / best)
    ro, rs = np.array(r_online[-tail:]), np.array(r_static[-tail:])
    gm = lambda r: float(np.exp(np.mean(np.log(r))))  # noqa: E731
    # what the stream taught: squared error in log time on the observations the tuner collected
    Xs, ys = np.stack(tuner.X[len(X):]), np.asarray(tuner.y[len(X):])
    fit = {"online_fit_mse": float(np.mean((online.predict(Xs) - ys) ** 2)),
           "static_fit_mse": float(np.mean((static.predict(Xs) - ys) ** 2)), "observations": int(len(ys))}
    return {"seed_queries": n_seed, "stream": len(stream), "tail": len(ro), "updates": tuner.updates,
            "explore": explore, "observe_top": observe_top, "shadow_frac": shadow_frac,
            "shadow_runs_per_query": tuner.shadow_runs / max(len(stream), 1), "seconds": time.time() - t0,
            "online_within_10pct": float(np.mean(ro <= 1.10)), "online_geomean": gm(ro),
            "static_within_10pct": float(np.mean(rs <= 1.10)), "static_geomean": gm(rs), **fit}


def run(ctx: "pv.Context", n_queries: int = 500, max_rows: int = 300_000_000, min_rows: int = 1_000_000,
        n_train: int | None = None, seed: int = 1709, reps: int = 3, candidates=CANDIDATES, log=print) -> dict:
    ex = explore(ctx, n_queries, max_rows, min_rows, seed, reps, log)
    return assess(ctx, ex, n_train, candidates)


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description="variant-selection suite on one GPU")
    ap.add_argument("--queries", type=int, default=500)
    ap.add_argument("--max-rows", type=int, default=300_000_000)
    ap.add_argument("--min-rows", type=int, default=1_000_000)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--epochs", type=int, default=0, help="fixed training setting instead of validation choice")
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--ensemble", type=int, default=5)
    ap.add_argument("--timings-in", default="", help="assess saved exploration results instead of timing again")
    ap.add_argument("--timings-out", default="")
    ap.add_argument("--out", default="")
    ap.add_argument("--graphs", action="store_true", help="run the CUDA-graph batch experiment only")
    ap.add_argument("--confirm-reps", type=int, default=15, help="re-timing runs per candidate (0 = skip)")
    ap.add_argument("--restat", action="store_true", help="with --timings-in: recompute the queries' statistics")
    ap.add_argument("--online", action="store_true", help="also run the run-time re-tuning experiment")
    ap.add_argument("--summary-out", default="", help="compact record of the figures (no per-query rows)")
    ap.add_argument("--l2-fetch-bytes", type=int, default=32, choices=[0, 32, 64, 128],
                    help="L2 fetch granularity of the CUDA context (pv_set_l2_fetch_bytes), as the benchmark sets it; 0 "
                         "leaves the context's initial setting")
    a = ap.parse_args(argv)
    ctx = pv.Context(0)
    if a.l2_fetch_bytes:
        ctx.set_l2_fetch_bytes(a.l2_fetch_bytes)
    if a.graphs:
        print(json.dumps(graph_experiment(ctx)))
        ctx.close()
        return
    data = None
    if a.timings_in:
        with open(a.timings_in) as f:
            ex = json.load(f)
        ex["stats"] = {int(k): v for k, v in ex["stats"].items()}
        ex["timings"] = {int(k): v for k, v in ex["timings"].items()}
        if a.restat:
            data = SuiteData(ctx, a.max_rows)
            ex["stats"] = {q["id"]: data.stats(q) for q in ex["queries"]}
    else:
        data = SuiteData(ctx, a.max_rows)
        ex = explore(ctx, a.queries, a.max_rows, a.min_rows, reps=a.reps, data=data)
        if a.timings_out:
            with open(a.timings_out, "w") as f:
                json.dump(ex, f)
    cands = ((a.epochs, a.ensemble, a.lr),) if a.epochs else CANDIDATES
    summary = assess(ctx, ex, candidates=cands)
    if a.confirm_reps > 0:
        data = data or SuiteData(ctx, a.max_rows)
        summary["confirmed"] = confirm(data, ex, summary, reps=a.confirm_reps)
    if a.online:
        # learning from the chosen variant's time alone, and from the top 3 of the ranking
        summary["online"] = {"chosen_only": online_experiment(ctx, ex),
                             "shadow_top3": online_experiment(ctx, ex, observe_top=3, explore=0.0, every=8,
                                                              steps=200, update_lr=1e-3)}
    print(json.dumps({k: (v if k != "confirmed" else {kk: vv for kk, vv in v.items() if kk != "per_query"})
                      for k, v in summary.items() if k != "per_query"}))
    if a.out:
        with open(a.out, "w") as f:
            json.dump(summary, f)
    if a.summary_out:
        with open(a.summary_out, "w") as f:
            json.dump(compact_record(summary, a, argv), f, indent=1)
    ctx.close()


def compact_record(summary: dict, args, argv=None) -> dict:
    """The suite's figures without per-query rows: how it was run (command,
    seed, sizes, grids, kernel sources), the network's and Algorithm 1's
    within-10% fractions and geometric-mean slowdowns on the held-out queries
    (against the exploration's timings and, when run, confirmed by re-timing),
    and the run-time re-tuning experiment when run."""
    import sys
    from . import build
    keep = ("queries", "train", "held_out", "grid_sizes", "exploration_s", "train_s", "train_rows", "chosen",
            "validation", "mlp_within_10pct", "mlp_geomean_slowdown", "mlp_worst_slowdown",
            "mlp_top3_within_10pct", "alg1_within_10pct", "alg1_geomean_slowdown", "alg1_worst_slowdown",
            "alg1_variants_run", "alg1_configs")
    rec = {"command": "python -m paper_1709_00700_gb300.suite " + " ".join(argv if argv is not None else sys.argv[1:]),
           "seed": 1709, "rows": [args.min_rows, args.max_rows], "reps": args.reps,
           "l2_fetch_bytes": getattr(args, "l2_fetch_bytes", None), "kernel_source_hash": build.source_hash(),
           "explored": {k: summary[k] for k in keep if k in summary}}
    if "confirmed" in summary:
        rec["confirmed"] = {k: v for k, v in summary["confirmed"].items() if k != "per_query"}
    if "online" in summary:
        rec["online"] = summary["online"]
    return rec



def graph_experiment(ctx: "pv.Context", n_queries: int = 64, rows: int = 1_000_000, reps: int = 20,
                     star_results: bool = False) -> dict:
    """CUDA graphs for many small pipelines: n_queries filter/aggregate queries
    (different constants, one shape) on a rows-row table replayed eagerly
    (one pv_rerun each) and as one captured graph; and a star join's four
    build pipelines plus its probe pipeline, eager and as one graph.  Every
    graph replay must leave the same results as the eager runs (asserted);
    with star_results the star join's result columns after the graph
    replays are returned too (key-sorted, int64), for a check against the
    oracle on datagen.star_schema(rows)."""
    import torch
    dev = f"cuda:{ctx.device}"
    u = datagen.uniform_int_torch
    seed = datagen.DEFAULT_SEED
    ctx.register_table("g", {"a": u(seed, 101, rows, 0, 100, torch.int32, device=dev),
                             "b": u(seed, 102, rows, 0, 100, torch.int32, device=dev),
                             "price": u(seed, 103, rows, 100, 10_000_000, torch.int64, device=dev)})
    rng = np.random.default_rng(7)
    var = pv.variant(pred="branch", access="grid", items_per_thread=4, block=512, grid_mult=2)
    results = []
    for _ in range(n_queries):
        lo = int(rng.integers(0, 60))
        plan = {"fact": "g", "filters": [["a", "lt", int(rng.integers(1, 100))], ["b", "between", lo, lo + 30]],
                "aggs": [["sum", [["x", "price"]]], ["count"]]}
        results.append(ctx.run(plan, var))
    ctx.sync()
    st = ctx.stream

    def timed(fn):
        ms = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            fn()
            b.record(st)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        return float(np.median(ms))

    eager = timed(lambda: [ctx.rerun(r) for r in results])
    want = [[int(c[0]) for c in ctx.fetch(r)] for r in results]
    gb = autotune.GraphBatch(ctx, results)
    graph = timed(gb.launch)
    got = [[int(c[0]) for c in ctx.fetch(r)] for r in results]
    assert got == want, "graph replay changed a result"
    gb.free()
    for r in results:
        ctx.free(r)
    # star join: builds + probe as one graph
    s = datagen.star_schema(rows)
    for t, cols in s.items():
        ctx.register_table(t, {c: torch.from_numpy(v).to(dev) for c, v in cols.items()})
    plan = workloads.star_plan()
    hts = ctx.build_all(plan, pv.ht_variant("perfect"))
    res = ctx.run(plan, pv.variant(agg="local", ht="perfect", items_per_thread=1, block=512), hts)
    ctx.sync()

    def star_eager():
        for h in hts:
            ctx.rebuild(h)
        ctx.rerun(res)

    def star_cols():
        cols = [c.astype(np.int64) for c in ctx.fetch(res)]
        order = np.lexsort((cols[1], cols[0]))
        return [c[order] for c in cols]

    star_e = timed(star_eager)
    ctx.sync()
    want_star = star_cols()
    ctx._check(ctx.lib.pv_graph_capture_begin(ctx.h))
    star_eager()
    g = ctypes_graph_end(ctx)
    star_g = timed(lambda: ctx._check(ctx.lib.pv_graph_launch(ctx.h, g)))
    ctx.sync()
    got_star = star_cols()
    assert all(np.array_equal(a, b) for a, b in zip(got_star, want_star)) and len(got_star) == len(want_star), \
        "graph replay of the star builds + probe changed its result"
    ctx.free(g)
    ctx.free(res)
    for h in hts:
        ctx.free(h)
    out = {"queries": n_queries, "rows": rows, "eager_ms": eager, "graph_ms": graph,
           "eager_us_per_query": 1000 * eager / n_queries, "graph_us_per_query": 1000 * graph / n_queries,
           "star_build_probe_rows": rows, "star_eager_ms": star_e, "star_graph_ms": star_g}
    if star_results:
        out["star_cols"] = got_star
    return out


def ctypes_graph_end(ctx) -> int:
    import ctypes
    g = ctypes.c_int32()
    ctx._check(ctx.lib.pv_graph_capture_end(ctx.h, ctypes.byref(g)))
    return g.value


if __name__ == "__main__":
    main()
