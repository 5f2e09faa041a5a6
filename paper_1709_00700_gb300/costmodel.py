"""Learned cost model for per-query variant selection.

The paper learns one variant configuration per processor and workload with
Algorithm 1 and applies it to every query (Section 8.3), and names a
run-time, per-query optimizer as future work (Section 9.4).  Here a small
network predicts the log run time of (query, variant) pairs from plan
features, column statistics and variant features; the pick for a query is
the variant with the smallest prediction.  Exhaustive search stays the
fallback and the yardstick.

Every forward pass, gradient and Adam step runs in libpv's kernels
(pv_mlp_forward / pv_mlp_backward / pv_mlp_adam); this module holds the
device buffers and does the bookkeeping.  Training is full batch.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import pv

H = 64

# ---------------------------------------------------------------------------
# Features
# ---------------------------------------------------------------------------
FAMILIES = ("filter", "grouped", "star")
PLAN_FEATURES = ("log_rows", "sel", "log_sel", "log_groups", "log_groups_per_row", "top_share", "n_preds",
                 "n_probes", "log_dim_rows", "bytes_in", "bytes_out", "n_aggs", "project", "log_bytes",
                 "log_out_rows", "fam_filter", "fam_grouped", "fam_star", "log_hot_rows", "log_groups_hit",
                 "log_rows_per_group", "log_collision", "warp_repeats", "sel_first", "log_sel_first",
                 "log_sel_after_first")
VARIANT_FEATURES = ("multi", "local", "ht_linear", "ht_cuckoo", "ht_perfect", "multshift", "predicated",
                    "chunked", "log_block", "grid_mult", "unroll", "private_tables", "prefetch", "build_linear",
                    "build_cuckoo", "build_perfect", "warp_agg", "compacted", "cluster", "compact_probes2",
                    "first_items2")
N_FEATURES = len(PLAN_FEATURES) + len(VARIANT_FEATURES)


def plan_vector(st: dict) -> list:
    """st: rows, sel (estimated fraction of rows surviving filters and
    probes), groups (estimated distinct groups), top_share (largest group's
    share of surviving rows), n_preds, n_probes, dim_rows (total build rows),
    bytes_in / bytes_out per row, n_aggs, project (0/1), family."""
    rows = max(1.0, float(st["rows"]))
    sel = min(1.0, max(float(st["sel"]), 1e-6))
    groups = max(1.0, float(st.get("groups", 1)))
    fam = st["family"]
    # without a measured collision probability: uniform over the groups, or one group when filtering
    coll = float(st["collision"]) if "collision" in st else (1.0 if fam == "filter" else 1.0 / groups)
    sel1 = min(1.0, max(float(st.get("sel_first", sel)), sel))
    return [math.log10(rows), sel, math.log10(sel), math.log10(groups), math.log10(groups / rows),
            float(st.get("top_share", 0.0)), float(st.get("n_preds", 0)), float(st.get("n_probes", 0)),
            math.log10(1.0 + float(st.get("dim_rows", 0))), float(st.get("bytes_in", 0)),
            float(st.get("bytes_out", 0)), float(st.get("n_aggs", 0)), float(st.get("project", 0)),
            math.log10(rows * max(1.0, float(st.get("bytes_in", 1)))), math.log10(1.0 + rows * sel),
            float(fam == "filter"), float(fam == "grouped"), float(fam == "star"),
            # contention proxies: rows of the hottest group, groups touched, rows per touched group
            math.log10(1.0 + rows * sel * float(st.get("top_share", 0.0))),
            math.log10(max(1.0, min(groups, rows * sel))),
            math.log10(max(1.0, rows * sel / max(1.0, min(groups, rows * sel)))),
            # key repeats: probability that two surviving rows share a group, and the expected
            # number of other rows of a 32-row warp step holding the same key
            math.log10(max(coll, 1e-9)), min(31.0, 31.0 * coll),
            # the first operation's own selectivity (what compacted execution queues) and the rest's
            sel1, math.log10(sel1), math.log10(min(1.0, sel / sel1))]


def variant_vector(v: dict) -> list:
    ht = v.get("ht", "linear")
    b = v.get("build", "")
    return [float(v.get("exec") == "multi"), float(v.get("agg", "local") == "local"), float(ht == "linear"),
            float(ht == "cuckoo"), float(ht == "perfect"), float(v.get("hash") == "multshift"),
            float(v.get("pred") == "predicated"), float(v.get("access") == "chunked"),
            math.log2(v.get("block", 256)), float(v.get("grid_mult", 0)), float(v.get("items_per_thread", 2)),
            float(v.get("threads_per_table", 0) == 1), float(v.get("prefetch", 0)), float(b == "linear"),
            float(b == "cuckoo"), float(b == "perfect"), float(v.get("warp_agg", 0)),
            float(v.get("pred") == "compacted"), float(v.get("agg") == "cluster"),
            float(v.get("compact_probes", 1) == 2), float(v.get("first_items", 1) == 2)]


def features(stats: dict, variant: dict) -> np.ndarray:
    return np.asarray(plan_vector(stats) + variant_vector(variant), dtype=np.float64)


# ---------------------------------------------------------------------------
# Network on the GPU
# ---------------------------------------------------------------------------
def n_params(F: int) -> int:
    return F * H + H + H * H + H + H + 1


class Net:
    """Parameters, Adam moments and standardisation on the device."""

    def __init__(self, ctx: "pv.Context", n_features: int, seed: int = 0):
        import torch
        self.torch = torch
        self.ctx = ctx
        self.F = n_features
        rng = np.random.default_rng(seed)
        F = n_features
        W1 = rng.uniform(-1, 1, (F, H)) * math.sqrt(6.0 / F)
        W2 = rng.uniform(-1, 1, (H, H)) * math.sqrt(6.0 / H)
        w3 = rng.uniform(-1, 1, H) * math.sqrt(6.0 / H)
        p = np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), w3, np.zeros(1)])
        dev = f"cuda:{ctx.device}"
        self.p = torch.tensor(p, dtype=torch.float32, device=dev)
        self.m = torch.zeros_like(self.p)
        self.v = torch.zeros_like(self.p)
        self.g = torch.zeros_like(self.p)
        self.mu = torch.zeros(F, dtype=torch.float32, device=dev)
        self.sigma = torch.ones(F, dtype=torch.float32, device=dev)
        self.step = 0

    @staticmethod
    def _p(t):
        return ctypes.c_void_p(t.data_ptr())

    def fit_standardisation(self, X: np.ndarray):
        X = np.asarray(X, np.float64)
        sd = X.std(axis=0)
        sd[sd < 1e-6] = 1.0
        self.mu.copy_(self.torch.tensor(X.mean(axis=0), dtype=self.torch.float32))
        self.sigma.copy_(self.torch.tensor(sd, dtype=self.torch.float32))

    def _dev(self, a):
        return self.torch.tensor(np.asarray(a, np.float32), device=self.p.device)

    def _forward(self, x, B, y, act):
        lib, ctx = self.ctx.lib, self.ctx
        ctx._check(lib.pv_mlp_forward(ctx.h, self._p(self.p), self._p(x), self._p(self.mu), self._p(self.sigma), B,
                                      self.F, self._p(y), self._p(act) if act is not None else None))

    def predict(self, X: np.ndarray) -> np.ndarray:
        X = np.asarray(X)
        B = len(X)
        if B == 0:
            return np.zeros(0)
        x = self._dev(X)
        y = self.torch.empty(B, dtype=self.torch.float32, device=self.p.device)
        self._forward(x, B, y, None)
        self.ctx.stream.synchronize()
        return y.cpu().numpy().astype(np.float64)

    def loss(self, X, t) -> float:
        y = self.predict(X)
        return float(np.mean((y - np.asarray(t)) ** 2))

    def train(self, X: np.ndarray, t: np.ndarray, epochs: int = 500, lr: float = 1e-3, batch: int | None = None,
              report_every: int = 50) -> list:
        """Full-batch Adam on the mean squared error; returns the loss every
        report_every epochs."""
        torch, lib, ctx = self.torch, self.ctx.lib, self.ctx
        B = len(X)
        x, tt = self._dev(X), self._dev(t)
        y = torch.empty(B, dtype=torch.float32, device=self.p.device)
        act = torch.empty(B * 2 * H, dtype=torch.float32, device=self.p.device)
        dz = torch.empty(B * (2 * H + 1), dtype=torch.float32, device=self.p.device)
        loss = torch.empty(1, dtype=torch.float32, device=self.p.device)
        hist = []
        n = self.p.numel()
        for e in range(epochs):
            self._forward(x, B, y, act)
            ctx._check(lib.pv_mlp_backward(ctx.h, self._p(self.p), self._p(x), self._p(self.mu), self._p(self.sigma),
                                           self._p(act), self._p(y), self._p(tt), B, self.F, self._p(dz),
                                           self._p(self.g), self._p(loss)))
            self.step += 1
            ctx._check(lib.pv_mlp_adam(ctx.h, self._p(self.p), self._p(self.g), self._p(self.m), self._p(self.v), n,
                                       lr, 0.9, 0.999, 1e-8, self.step))
            if e % report_every == 0 or e == epochs - 1:
                ctx.stream.synchronize()
                hist.append(float(loss.item()))
        return hist


class Ensemble:
    """Mean prediction of several independently initialised networks."""

    def __init__(self, nets: list):
        self.nets = nets

    def predict(self, X: np.ndarray) -> np.ndarray:
        return np.mean([n.predict(X) for n in self.nets], axis=0)


# ---------------------------------------------------------------------------
# Selection
# ---------------------------------------------------------------------------
def pick(net, stats: dict, grid: list) -> tuple:
    """Variant of grid with the smallest predicted log time."""
    X = np.stack([features(stats, v) for v in grid])
    pred = net.predict(X)
    i = int(np.argmin(pred))
    return grid[i], pred


# ---------------------------------------------------------------------------
# Run-time re-tuning
# ---------------------------------------------------------------------------
class OnlineTuner:
    """Per-query variant choice that keeps learning from the queries it runs
    (a run-time optimizer, the paper's future work).

    Every executed query contributes (its features, the measured log time of
    the variant that ran) to a replay buffer.  With observe_top = k > 1 the
    runner-ups of the network's ranking (its 2nd .. k-th choices) are timed as
    well, on a fraction shadow_frac of the queries: extra runs of the query
    that cost time but show the network where its ranking is wrong, which the
    chosen variant's time alone rarely does.  With probability `explore` the
    network's second choice runs instead of its first.  Every `every` queries
    each network of the ensemble continues training on the whole buffer for
    `steps` Adam steps (its weights, moments and step count carry over; the
    standardisation fitted on the seed data stays)."""

    def __init__(self, model: Ensemble, X: np.ndarray, y: np.ndarray, every: int = 16, steps: int = 400,
                 lr: float = 5e-4, explore: float = 0.1, cap: int = 50_000, seed: int = 0, observe_top: int = 1,
                 shadow_frac: float = 1.0):
        self.model = model
        self.X = [np.asarray(x, np.float64) for x in X]
        self.y = [float(v) for v in y]
        self.every, self.steps, self.lr, self.explore, self.cap = every, steps, lr, explore, cap
        self.observe_top, self.shadow_frac = observe_top, shadow_frac
        self.rng = np.random.default_rng(seed)
        self.pending = 0
        self.updates = 0
        self.shadow_runs = 0
        self._ranked = []

    def choose(self, stats: dict, grid: list) -> dict:
        X = np.stack([features(stats, v) for v in grid])
        order = np.argsort(self.model.predict(X))
        self._ranked = [grid[int(i)] for i in order]
        if len(order) > 1 and self.rng.random() < self.explore:
            return self._ranked[1]
        return self._ranked[0]

    def shadow_candidates(self, picked: dict) -> list:
        """The variants to time besides the one that ran, for the last choose():
        the top observe_top of the ranking other than `picked` (none on the
        queries outside the shadow fraction)."""
        if self.observe_top <= 1 or self.rng.random() >= self.shadow_frac:
            return []
        out = [v for v in self._ranked[:self.observe_top] if v is not picked][:self.observe_top - 1]
        self.shadow_runs += len(out)
        return out

    def _add(self, stats: dict, variant: dict, ms: float):
        if not (ms > 0 and math.isfinite(ms)):
            return
        self.X.append(features(stats, variant))
        self.y.append(math.log(ms))
        if len(self.X) > self.cap:
            del self.X[0], self.y[0]

    def observe(self, stats: dict, variant: dict, ms: float, shadows=()):
        """One executed query: the time of the variant that ran, and the times
        of its shadow runs [(variant, ms), ...]."""
        self._add(stats, variant, ms)
        for v, t in shadows:
            self._add(stats, v, t)
        self.pending += 1
        if self.pending >= self.every:
            X, y = np.stack(self.X), np.asarray(self.y)
            for net in self.model.nets:
                net.train(X, y, epochs=self.steps, lr=self.lr, report_every=self.steps)
            self.pending = 0
            self.updates += 1
