"""Autotuner for shares and search-kernel schedules.

The paper's optimizer picks shares from a cost model (Sec. 5.2-5.3); its own
share study (Sec. 6, "Partition") shows the best split depends on the data.
This tuner times real launches of the library on the query and data at
hand and keeps the fastest configuration, searching one knob at a time
(coordinate descent) from the paper's plan:

  shares        the plan of ``choose_shares`` at several cell counts P, plus
                all-on-the-first-variable and square splits of the same P;
  item_grain    loop-2 candidates per work item;
  merge         when the last loop uses the warp merge path (min length,
                length ratio) or never;
  slice_grain   loop-3 candidates per slice of a hub (queries of 4+ loops).

The loop order is chosen the same way (``Tuner.tune_order``): the paper's
plan decision (Sec. 5.3) ranks orders by its cost estimate; here the cost
model's best few orders are timed on the data at hand and the fastest kept,
because the estimate does not see list-length skew or the GPU's search paths.

Results are cached per (query shape, log2 size bucket, mode) in memory and,
if a path is given, in a JSON file.  Tuning launches run in count mode; for
a materializing run the merge knobs are then re-chosen with materializing
launches, since writing tuples from a merge walk costs more than counting
them and moves the best threshold.
"""
from __future__ import annotations

import itertools
import json
import math
import os
import time
from dataclasses import dataclass, field

import torch

from . import Query, choose_shares, plan_cost, run_join

MERGE_OFF = 0xFFFFFFFF


@dataclass
class Config:
    shares: list
    item_grain: int = 64
    merge_min: int = 32
    merge_ratio: int = 4
    slice_grain: int = 256
    ms: float = float("inf")

    def options(self) -> dict:
        return {"shares": list(self.shares), "item_grain": self.item_grain, "merge_min": self.merge_min,
                "merge_ratio": self.merge_ratio, "slice_grain": self.slice_grain}

    def key(self) -> tuple:
        return (tuple(self.shares), self.item_grain, self.merge_min, self.merge_ratio, self.slice_grain)


def shape_key(query: Query, indexes) -> str:
    rows = max(ix.n for ix in indexes)
    bucket = int(math.log2(max(rows, 1)))
    return f"{query.n_vars}|{sorted(query.atoms, key=str)}|{query.loop_order()}|{bucket}"


def _time(query, indexes, cfg: Config, reps: int, stream, **extra) -> float:
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run_join(query, indexes, stream=stream, **cfg.options(), **extra)
        e1.record(stream)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def share_candidates(query: Query, indexes, P_list=(64, 256, 1024), min_cells: int = 1) -> list:
    """Share vectors (per variable id) to try: the plan at each P, P on the
    first loop variable alone, and a square split of P over the first two."""
    nv = query.n_vars
    first, second = query.loop_order()[0], query.loop_order()[1]
    out = []
    for P in P_list:
        if P < min_cells:
            continue
        out.append(choose_shares(query, indexes, P))
        s = [1] * nv
        s[first] = P
        out.append(s)
        r = int(round(math.sqrt(P)))
        if r * r == P:
            s = [1] * nv
            s[first], s[second] = r, r
            out.append(s)
    if min_cells <= 1:
        out.append([1] * nv)
    uniq = []
    for s in out:
        if s not in uniq:
            uniq.append(s)
    return uniq


def ranked_orders(query: Query, indexes) -> list:
    """Every loop order of the query, cheapest first by the Sec. 5.2 estimate
    with all shares 1 (the sum over loops of Lemma "cost-ub"'s bound); ties
    keep the lexicographic order.  The estimate reads only the indexes' sizes,
    whatever their attribute order."""
    ranked = []
    for order in itertools.permutations(range(query.n_vars)):
        c = plan_cost(query.with_order(order), indexes, [1] * query.n_vars)
        ranked.append((sum(c["level_cost"]), order))
    ranked.sort(key=lambda t: t[0])
    return [o for _, o in ranked]


@dataclass
class Tuner:
    path: str | None = None
    reps: int = 2
    cache: dict = field(default_factory=dict)

    def __post_init__(self):
        if self.path and os.path.exists(self.path):
            with open(self.path) as f:
                self.cache = json.load(f)

    def save(self) -> None:
        if self.path:
            os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
            with open(self.path, "w") as f:
                json.dump(self.cache, f, indent=1)

    def tune_order(self, query: Query, index_for, top_k: int = 4, stream=None, **options) -> tuple:
        """Loop order by measurement: the cost model's top_k orders
        (ranked_orders), each run in count mode on the data (best of
        self.reps launches, search kernel time); returns (order, {order:
        ms}).  ``index_for(j, attr_order)`` gives atom j's index in that
        attribute order; ``options`` go to run_join (shares default 1)."""
        stream = stream or torch.cuda.current_stream()
        base = [index_for(j, query.with_order(tuple(range(query.n_vars))).attr_order(j))
                for j in range(len(query.atoms))]
        times = {}
        for order in ranked_orders(query, base)[:max(1, top_k)]:
            qo = query.with_order(order)
            idx = [index_for(j, qo.attr_order(j)) for j in range(len(query.atoms))]
            best = float("inf")
            for _ in range(self.reps):
                r = run_join(qo, idx, stream=stream, time_kernels=True, **options)
                best = min(best, r.ms_join_kernel)
            times[tuple(order)] = best
        order = min(times, key=times.get)
        return order, times

    def tune(self, query: Query, indexes, P_list=(64, 256, 1024), min_cells: int = 1, stream=None,
             log=None, mode: str = "count", out_capacity: int = 0) -> Config:
        """Fastest configuration for this query and data.  mode="materialize"
        (with the output pool size out_capacity, 0 = two-pass) re-chooses the
        merge knobs with materializing launches."""
        key = shape_key(query, indexes) + f"|P{tuple(P_list)}|min{min_cells}" + (
            "" if mode == "count" else f"|{mode}")
        if key in self.cache:
            c = self.cache[key]
            return Config(**c)
        stream = stream or torch.cuda.current_stream()
        t0 = time.perf_counter()
        plan = choose_shares(query, indexes, max(P_list))
        start = Config(shares=plan if math.prod(plan) >= min_cells else [1] * query.n_vars)
        tried = {}

        def measure(c: Config) -> float:
            k = c.key()
            if k not in tried:
                tried[k] = _time(query, indexes, c, self.reps, stream)
            return tried[k]

        best = start
        best.ms = measure(best)
        knobs = [
            ("shares", share_candidates(query, indexes, P_list, min_cells)),
            ("item_grain", [16, 64, 256]),
            ("merge", [(32, 4), (32, 8), (64, 4), (MERGE_OFF, 1)]),
        ]
        if query.n_vars >= 4:
            knobs.append(("slice_grain", [128, 256, 1024]))
        for name, values in knobs:
            for v in values:
                c = Config(**{k: getattr(best, k) for k in ("shares", "item_grain", "merge_min", "merge_ratio",
                                                             "slice_grain")})
                if name == "merge":
                    c.merge_min, c.merge_ratio = v
                else:
                    setattr(c, name, list(v) if name == "shares" else v)
                c.ms = measure(c)
                if c.ms < best.ms:
                    best = c
        if mode == "materialize":
            extra = {"mode": "materialize", "out_capacity": out_capacity}
            best.ms = _time(query, indexes, best, self.reps, stream, **extra)
            for mm, mr in [(32, 2), (32, 4), (32, 8), (64, 4), (MERGE_OFF, 1)]:
                c = Config(shares=list(best.shares), item_grain=best.item_grain, merge_min=mm, merge_ratio=mr,
                           slice_grain=best.slice_grain)
                if c.key() == best.key():
                    continue
                c.ms = _time(query, indexes, c, self.reps, stream, **extra)
                if c.ms < best.ms:
                    best = c
        if log:
            log(f"autotune {key}: {len(tried)} launches in {time.perf_counter() - t0:.1f}s -> {best}")
        self.cache[key] = {"shares": best.shares, "item_grain": best.item_grain, "merge_min": best.merge_min,
                           "merge_ratio": best.merge_ratio, "slice_grain": best.slice_grain, "ms": best.ms}
        self.save()
        return best
