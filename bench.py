#!/usr/bin/env python
"""Benchmark of the HoneyComb hot path on a GB300.

Workload (one "step" = the whole hot path on one batch of input already in
HBM): the triangle query Q(x,y,z) = E(x,y), E(y,z), E(x,z) with x < y < z
(the selection pushed into the relation: E+ = {(u,v) in E : u < v}) over an
R-MAT graph of scale 22, edge factor 16, (a,b,c,d) = (.57,.19,.19,.05),
scrambled ids, symmetrised, de-duplicated, self loops removed.  A step:
  build_index(E+)        LSD radix sort + run-boundary scan (CoCo)
  run_join(materialize)  HyperCube routing of every atom whose shares are
                         not all 1, loop-1 intersection per cell, the
                         persistent search kernel counting then emitting
                         every output tuple.
Metric: output tuples per second (|Q| / step time), whole job.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  The reference arm times the CPU oracle (the
plain Generic Join used by the tests) on the host cores on a bounded sample
of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "join output tuples/s (R-MAT triangle)"
UNIT = "tuples/s"
PROFILE_NOTE = os.path.join(ROOT, "profiles", "gj_search_kernel_rmat22.md")
BUILD_PROFILE_NOTE = os.path.join(ROOT, "profiles", "radix_pass_rmat22_build.md")
KJOIN_PROFILE_NOTE = os.path.join(ROOT, "profiles", "kjoin_kernel_lw.md")  # LW over [512]^3, one cell


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--scale", type=int, default=None, help="R-MAT scale (default per workload)")
    ap.add_argument("--edge-factor", type=int, default=16)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--mode", choices=["materialize", "count"], default="materialize")
    ap.add_argument("--workload", choices=["triangle", "clique4", "cycle4", "batched", "serve", "build", "order",
                                           "lw", "ct", "skew"],
                    default="triangle",
                    help="triangle: R-MAT triangle (default line); clique4 / cycle4: R-MAT 4-clique / 4-cycle "
                         "counts; batched: 512 triangle/4-clique queries on induced subgraphs in one launch; "
                         "serve: continuous-batching server; build: CoCo index build of R-MAT E+; "
                         "order: 4-clique under every loop order beside the cost model's choice; "
                         "lw / ct: Loomis-Whitney / Clover-Triangle counts over ST-Dense's or ST-Sparse's "
                         "ternary relations; skew: per-cell work and time of the R-MAT triangle under the "
                         "paper's share vectors (Sec. 1, Examples 1-3)")
    ap.add_argument("--lw-n", type=int, default=512, help="lw: cube side n of ST-Dense's [n]^3 relations")
    ap.add_argument("--kshares", default="",
                    help="lw / ct: HyperCube shares of the four variables, e.g. 2,2,1,2 (Sec. 4, Example "
                         "'partition'); the relations are partitioned when their indexes are built")
    ap.add_argument("--tensor", choices=["dense", "sparse"], default="dense",
                    help="lw / ct: ST-Dense or ST-Sparse relations")
    ap.add_argument("--ct-m", type=int, default=4096, help="ct: m of the F x [m] x [m] relations")
    ap.add_argument("--ct-first", choices=["paper", "common"], default="paper",
                    help="ct: first-attribute sets {0,1},{0,2},{1,2} as written (empty result) or {0,1} in all three")
    ap.add_argument("--shares", default="autotune",
                    help="'autotune' (timed search from the paper's plan over HyperCube share vectors of "
                         ">= --min-cells cells and kernel schedules), 'plan' (Sec. 5.3 decision at --P cells), "
                         "or explicit, e.g. 32,32,1")
    ap.add_argument("--min-cells", type=int, default=64,
                    help="autotune: smallest number of cells (so the routing steps always run)")
    ap.add_argument("--P", type=int, default=1024)
    ap.add_argument("--grain", type=int, default=0)
    ap.add_argument("--merge", default="auto",
                    help="last-loop merge path: 'auto' (the autotuner's choice, else the library default), "
                         "'off', or MIN,RATIO")
    ap.add_argument("--dir-min", type=int, default=0,
                    help="searches of runs at least this long use the bucket directory (0: library default 16; "
                         "-1: plain binary search)")
    ap.add_argument("--pair-min", type=int, default=0,
                    help="last-loop bindings with a shorter list this long are searched by the whole warp "
                         "(0: library default 32; -1: never)")
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--capacity", default="plan",
                    help="materialize output pool: 'plan' = 1.25 x the planning run's count (one pass), "
                         "'0' = counting pass + emitting pass")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=10_000, help="serve: number of requests")
    ap.add_argument("--serve-select", choices=["all", "rmat"], default="all",
                    help="serve: restrict every request to a vertex sample (all), or only those with an R-MAT "
                         "atom (rmat; the others join the uniform relations unrestricted)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--batch-edges", default="1e4,8e6",
                    help="batched: range of the log-uniform subgraph edge counts")
    ap.add_argument("--cpu-frac", type=float, default=1.0 / 32,
                    help="fraction of x values in the oracle's bounded sample")
    return ap.parse_args()


def workload_name(a) -> str:
    return (f"triangle x<y<z, R-MAT scale {a.scale} ef {a.edge_factor} (a,b,c,d)=(.57,.19,.19,.05), "
            f"scrambled, symmetrised, deduplicated; {a.mode}")


def make_graph(a, rank: int, device: str | None):
    import datagen

    t = time.perf_counter()
    sym = datagen.rmat_graph(a.scale, a.edge_factor, a.seed + rank, device=device)
    ep = datagen.orient_lt(sym)
    del sym
    ep = datagen.scatter_order(ep, a.seed + rank)
    return ep, time.perf_counter() - t


def oracle_sample(ep, frac: float, seed: int):
    """Rows of R, S, T a restricted triangle query can touch: x in a seeded
    vertex subset F (R, T), and y in R[F] (S).  Exact: the count over these
    rows is |{(x,y,z) in Q : x in F}|."""
    import numpy as np

    import datagen

    nv = int(ep.max()) + 1
    mask = datagen.vertex_sample_mask(nv, seed, frac)
    rt = ep[mask[ep[:, 0]]]
    ys = np.zeros(nv, dtype=bool)
    ys[rt[:, 1]] = True
    s = ep[ys[ep[:, 0]]]
    return np.ascontiguousarray(rt), np.ascontiguousarray(s), np.nonzero(mask)[0].astype(np.uint32)


def run_oracle_sample(ep, frac, seed):
    import oracle

    rt, s, f = oracle_sample(ep, frac, seed)
    cores = os.cpu_count() or 1
    t = time.perf_counter()
    cnt, _, _ = oracle.gj_count(3, [(0, 1), (1, 2), (0, 2)], [rt, s, rt], filt=f, nthreads=cores)
    dt = time.perf_counter() - t
    desc = (f"triangles with x in a seeded {frac:.5f} vertex sample ({f.shape[0]} x values); oracle over the "
            f"{rt.shape[0]} R/T rows and {s.shape[0]} S rows that sample touches (trie builds included), "
            f"{cnt} tuples in {dt:.2f} s")
    return cnt, dt, cores, desc


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(gpu_index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        # nvidia-smi's start-up stalls the GPU for up to a second or so:
        # start timing only once it has produced its first sample
        self.first = []
        if self.proc is not None:
            import select

            ready, _, _ = select.select([self.proc.stdout], [], [], 15.0)
            if ready:
                self.first.append(self.proc.stdout.readline())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        lines = (self.first + out.strip().splitlines())[1:]  # samples taken while timing
        before = False
        if not lines and self.first:  # a timed region shorter than the sampling period
            lines, before = self.first, True
        for line in lines:
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for name, val in zip(self.NAMES, p[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        r = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
             "reasons": sorted(reasons), "samples": len(sm)}
        if before:
            r["note"] = "timed region shorter than the 200 ms sampling period: sample taken just before it"
        return r


def combine_ranks(ms_total: float, tuples: float, dist, device) -> tuple:
    """Whole-job figures over ranks: the slowest rank's time (max) and the
    tuples of all ranks (sum)."""
    import torch

    t = torch.tensor([ms_total], dtype=torch.float64, device=device)
    c = torch.tensor([tuples], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), float(c.item())


def measured_hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def source_hash(sources) -> str:
    """sha256 over the concatenated bytes of the given csrc files."""
    h = hashlib.sha256()
    for name in sources:
        h.update(open(os.path.join(ROOT, "paper_2502_06715_gb300", "csrc", name), "rb").read())
    return h.hexdigest()


def profiled_traffic(note: str = None, sources=("hc_join.cu", "hc_internal.cuh")):
    """Per-launch DRAM bytes of a kernel from a committed ncu summary, if it
    was taken on the current source of the files that hold the kernel."""
    try:
        text = open(note or PROFILE_NOTE).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*(\d+)", text)
    h = re.search(r"source_sha256:\s*([0-9a-f]{64})", text)
    if not m or not h:
        return None
    if source_hash(sources) != h.group(1):
        return None
    return int(m.group(1))


def main():
    a = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.scale is None:
        a.scale = {"triangle": 22, "clique4": 20, "cycle4": 20, "batched": 21, "serve": 23, "build": 22,
                   "order": 18, "lw": 0, "ct": 0, "skew": 22}[a.workload]
    if a.impl == "reference":
        return reference_arm(a, world, rank)
    if a.workload == "serve":
        return serve_workload(a, world, rank, local)
    if a.workload == "build":
        return build_workload(a, world, rank, local)
    if a.workload in ("lw", "ct"):
        return kary_workload(a, world, rank, local)
    if a.workload == "order":
        return order_workload(a, world, rank, local)
    if a.workload == "skew":
        return skew_workload(a, world, rank, local)
    if a.workload != "triangle":
        return other_workload(a, world, rank, local)

    import numpy as np
    import torch

    import __graft_entry__

    __graft_entry__.build()
    import paper_2502_06715_gb300 as hc

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)

    # independent problem per rank (weak scaling): seed + rank
    ep, gen_s = make_graph(a, rank, device=f"cuda:{local}")
    n = ep.shape[0]
    d_pairs = torch.from_numpy(ep.view(np.int32)).to(dev)
    stream = torch.cuda.current_stream(dev)
    q = hc.TRIANGLE

    # plan (host, untimed): shares per the paper's decision rule at P cells,
    # the autotuner's timed choice, or given; kernel schedules likewise
    ix0 = hc.build_index(d_pairs, 0)
    plan_shares = hc.choose_shares(q, [ix0] * 3, a.P)
    tuned = None
    if a.shares == "plan":
        shares = plan_shares
    elif a.shares == "autotune":
        from paper_2502_06715_gb300.autotune import Tuner

        # the output pool of a materializing run is sized from a count run
        cap = 0
        if a.mode == "materialize" and a.capacity == "plan":
            cap = int(1.25 * hc.run_join(q, [ix0] * 3, shares=plan_shares).count) + 1
        elif a.mode == "materialize":
            cap = int(a.capacity)
        tuned = Tuner().tune(q, [ix0] * 3, P_list=(64, 256, 1024), min_cells=a.min_cells, mode=a.mode,
                             out_capacity=cap)
        shares = tuned.shares
        if not a.grain:
            a.grain = tuned.item_grain
    else:
        shares = [int(x) for x in a.shares.split(",")]
    knobs = {"merge_min": tuned.merge_min, "merge_ratio": tuned.merge_ratio} if tuned else {}
    if a.merge == "off":
        knobs = {"merge_min": 0xFFFFFFFF, "merge_ratio": 1}
    elif a.merge != "auto":
        mm, mr = (int(x) for x in a.merge.split(","))
        knobs = {"merge_min": mm, "merge_ratio": mr}
    knobs["dir_min"] = a.dir_min & 0xFFFFFFFF
    knobs["pair_min"] = a.pair_min & 0xFFFFFFFF
    stats = hc.run_join(q, [ix0] * 3, shares=shares, stats=True, item_grain=a.grain, block_threads=a.threads,
                        **knobs)
    work, expect = stats.work, stats.count
    l1 = ix0.l1
    ix0.free()
    del stats

    capacity = int(1.25 * expect) + 1 if a.capacity == "plan" else int(a.capacity)

    def step():
        ix = hc.build_index(d_pairs, 0, stream=stream)
        r = hc.run_join(q, [ix, ix, ix], shares=shares, mode=a.mode, keep_device=True, time_kernels=True,
                        item_grain=a.grain, block_threads=a.threads, stream=stream, out_capacity=capacity, **knobs)
        ix.free()
        return r

    for _ in range(a.warmup):
        r = step()
        if r.count != expect:
            raise SystemExit(f"count mismatch in warm-up: {r.count} != {expect}")
        del r
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    launches0 = hc.kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kern_ms, kern_launches = 0.0, 0
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(a.steps):
        r = step()
        kern_ms += r.ms_join_kernel
        kern_launches += r.n_join_launches
        count = r.count
        del r
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = hc.kernel_launches() - launches0
    clk = clocks.stop()
    ms_total = ev0.elapsed_time(ev1)
    if dist:
        ms_total, total_tuples = combine_ranks(ms_total, float(count) * a.steps, dist, dev)
    else:
        total_tuples = float(count) * a.steps
    ms_step = ms_total / a.steps
    value = total_tuples / (ms_total / 1e3)

    # roofline of the search kernel: algorithmic bytes per launch = 4 B per
    # unit of the work counter (each element of the shortest list read once
    # per list it is searched in), plus, for the emitting launch, the output
    # tuples written (3 x 4 B each)
    n_launch_per_step = kern_launches / a.steps
    out_bytes = 12.0 * count if a.mode == "materialize" else 0.0
    alg_bytes = 4.0 * work + out_bytes / n_launch_per_step
    avg_launch_s = (kern_ms / max(1, kern_launches)) / 1e3
    peak, peak_kind = measured_hbm_peak()
    achieved = alg_bytes / avg_launch_s / 1e9 if avg_launch_s > 0 else 0.0
    roofline = {"bound": "hbm", "kernel": "gj_kernel (persistent search)", "achieved": round(achieved, 1),
                "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": profiled_traffic(), "alg_bytes_per_launch": alg_bytes,
                "avg_launch_ms": round(avg_launch_s * 1e3, 3)}

    e2e = None
    if not a.no_e2e:
        e2e = end_to_end(a, hc, ep, shares, q, dev, stream, expect, capacity, knobs)

    cpu = None
    if not a.no_cpu_baseline and rank == 0 and world == 1:
        cnt, dt, cores, desc = run_oracle_sample(ep, a.cpu_frac, 12345)
        cpu = {"value": cnt / dt, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic (seeded R-MAT)",
            "config": {"workload": workload_name(a), "scale": a.scale, "edge_factor": a.edge_factor,
                       "rows_E+": n, "distinct_x": l1, "tuples": count, "shares": shares,
                       "shares_from": a.shares if a.shares not in ("plan", "autotune") else
                       (f"choose_shares(P={a.P})" if a.shares == "plan" else
                        f"autotune (>= {a.min_cells} cells; candidates include choose_shares(P=64..1024))"),
                       "plan_shares_P1024": plan_shares, "item_grain": a.grain or 64,
                       "merge": [knobs.get("merge_min", 32), knobs.get("merge_ratio", 4)],
                       "dir_min": knobs["dir_min"] or 16, "pair_min": knobs["pair_min"] or 32,
                       "out_capacity": capacity if a.mode == "materialize" else None,
                       "search_launches_per_step": n_launch_per_step,
                       "work_counter": work, "l2": "inputs larger than L2 (E+ is %.0f MB)" % (n * 8 / 1e6),
                       "parallelism": f"replicas x{world}", "generate_s": round(gen_s, 1)},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def end_to_end(a, hc, ep, shares, q, dev, stream, expect, capacity, knobs):
    """Same metric through the public API from pinned HOST memory: the H2D
    copy of E+, the build, the join and the transfer of the result to pinned
    host memory (all tuples in materialize mode, through hc_run_join_to_host,
    which copies each search segment's output while the next one runs; the
    count otherwise) are inside the timed region."""
    import numpy as np
    import torch

    host_in = torch.from_numpy(ep.view(np.int32)).pin_memory()
    nvars = 3
    host_out = None
    if a.mode == "materialize":
        host_out = torch.empty((expect, nvars), dtype=torch.int32, pin_memory=True)
    opts = {k: v for k, v in knobs.items()}

    def e2e_step():
        d = host_in.to(dev, non_blocking=True)
        ix = hc.build_index(d, 0, stream=stream)
        if host_out is not None:
            c = hc.run_join_to_host(q, [ix, ix, ix], host_out, shares=shares, item_grain=a.grain,
                                    block_threads=a.threads, stream=stream, **opts)
        else:
            c = hc.run_join(q, [ix, ix, ix], shares=shares, mode=a.mode, item_grain=a.grain,
                            block_threads=a.threads, stream=stream, **knobs).count
        torch.cuda.current_stream(dev).synchronize()
        ix.free()
        del d
        return c

    for _ in range(max(1, min(2, a.warmup))):
        e2e_step()
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(a.steps):
        c = e2e_step()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t
    if c != expect:
        raise SystemExit("end-to-end count mismatch")
    return {"value": c * a.steps / dt, "unit": UNIT, "h2d_bytes_per_step": int(host_in.numel() * 4),
            "d2h_bytes_per_step": int(host_out.numel() * 4) if host_out is not None else 8,
            "ms_per_step": dt / a.steps * 1e3}


def other_workload(a, world, rank, local):
    """Lines for the other configurations (not the default bench line)."""
    import numpy as np
    import torch

    import __graft_entry__
    import datagen

    __graft_entry__.build()
    import paper_2502_06715_gb300 as hc
    from paper_2502_06715_gb300.autotune import Tuner

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    t = time.perf_counter()
    sym = datagen.rmat_graph(a.scale, a.edge_factor, a.seed + rank, device=f"cuda:{local}")
    gen_s = time.perf_counter() - t
    clocks = None
    if a.workload in ("clique4", "cycle4"):
        rel = datagen.orient_lt(sym) if a.workload == "clique4" else sym
        rel = datagen.scatter_order(rel, a.seed)
        d = torch.from_numpy(rel.view(np.int32)).to(dev)
        q = hc.FOUR_CLIQUE if a.workload == "clique4" else hc.FOUR_CYCLE
        ix0 = hc.build_index(d, 0)
        if a.shares == "autotune":
            cfg = Tuner(reps=1).tune(q, [ix0] * len(q.atoms), P_list=(64, 256), min_cells=a.min_cells)
            opts = cfg.options()
        elif a.shares == "plan":
            opts = {"shares": hc.choose_shares(q, [ix0] * len(q.atoms), a.P)}
        else:
            opts = {"shares": [int(x) for x in a.shares.split(",")]}
        stats = hc.run_join(q, [ix0] * len(q.atoms), stats=True, **opts)
        ix0.free()

        def step():
            ix = hc.build_index(d, 0, stream=stream)
            r = hc.run_join(q, [ix] * len(q.atoms), stream=stream, time_kernels=True, **opts)
            ix.free()
            return r

        for _ in range(a.warmup):
            step()
        torch.cuda.synchronize()
        sampler = ClockSampler(local)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        kern = 0.0
        for _ in range(a.steps):
            r = step()
            kern += r.ms_join_kernel
        e1.record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        ms = e0.elapsed_time(e1) / a.steps
        # roofline: the work counter measures the unrewritten loops, so it is
        # set against the kernel that runs them (a stats run does not rewrite,
        # Sec. 5.1); the timed steps of the 4-clique run rewritten
        roof_ms = kern / a.steps
        if a.workload == "clique4":
            ix = hc.build_index(d, 0, stream=stream)
            ru = hc.run_join(q, [ix] * len(q.atoms), stream=stream, stats=True, time_kernels=True, **opts)
            ix.free()
            roof_ms = ru.ms_join_kernel
        line = {"metric": "join output tuples/s (R-MAT %s)" % ("4-clique" if a.workload == "clique4" else "4-cycle"),
                "value": r.count / (ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
                "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
                "data": "synthetic (seeded R-MAT)",
                "config": {"workload": f"{a.workload} on R-MAT scale {a.scale} ef {a.edge_factor}, "
                                       f"{'E+ (x<y)' if a.workload == 'clique4' else 'symmetric'}; count",
                           "rows": int(rel.shape[0]), "tuples": r.count, "work_counter": stats.work,
                           "options": opts, "search_kernel_ms": kern / a.steps, "generate_s": round(gen_s, 1)},
                "roofline": {"bound": "hbm", "kernel": "gj_kernel (persistent search)",
                             "achieved": 4.0 * stats.work / (roof_ms / 1e3) / 1e9,
                             "peak": measured_hbm_peak()[0], "unit": "GB/s",
                             "frac": 4.0 * stats.work / (roof_ms / 1e3) / 1e9 / measured_hbm_peak()[0],
                             "traffic": None, "avg_launch_ms": roof_ms,
                             "note": ("the unrewritten search (a stats run), whose loops the work counter measures; "
                                      "the timed steps run with Sec. 5.1's rewriting (search_kernel_ms)")
                             if a.workload == "clique4" else None},
                "clocks": clocks}
        print(json.dumps(line), flush=True)
        return
    # batched: 512 triangle / 4-clique queries on induced subgraphs of E+
    ep = datagen.orient_lt(sym)
    d = torch.from_numpy(ep.view(np.int32)).to(dev)
    nv = int(sym.max()) + 1
    rng = np.random.default_rng(4)
    n = 512
    kinds = rng.random(n) < 0.5
    lo_e, hi_e = (float(x) for x in a.batch_edges.split(","))
    targets = np.exp(rng.uniform(np.log(lo_e), np.log(hi_e), size=n)).astype(np.int64)
    qs, idx = [], []
    t = time.perf_counter()
    for i in range(n):
        sub = datagen.induced_by_key(d, nv, 4_000_000 + i, int(targets[i]))
        ix = hc.build_index(sub, 0)
        q = hc.TRIANGLE if kinds[i] else hc.FOUR_CLIQUE
        qs.append(q)
        idx.append([ix] * len(q.atoms))
    prep_s = time.perf_counter() - t
    # autotune per (kind, size bucket) on the group's first query
    tuner = Tuner(reps=1)
    opts = []
    t = time.perf_counter()
    for q, l in zip(qs, idx):
        cfg = tuner.tune(q, l, P_list=(8, 64), min_cells=1)
        o = cfg.options()
        opts.append(o)
    tune_s = time.perf_counter() - t
    sep_counts = [hc.run_join(q, l, **o).count for q, l, o in zip(qs, idx, opts)]
    side = torch.cuda.Stream(dev)
    b = hc.Batch(qs, idx, opts, stream=side)
    l0 = hc.kernel_launches()
    b.capture(side)
    per_replay = hc.kernel_launches() - l0  # kernels recorded in the graph
    b.launch(side)
    if b.counts() != sep_counts:
        raise SystemExit("batched counts differ from separate launches")
    for _ in range(a.warmup):
        b.launch(side)
        b.counts()
        pend = [hc.run_join_async(q, l, stream=side, **o) for q, l, o in zip(qs, idx, opts)]
        [p.count() for p in pend]
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    launches0 = hc.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(side)
    for _ in range(a.steps):
        b.launch(side)
    e1.record(side)
    torch.cuda.synchronize()
    batched_ms = e0.elapsed_time(e1) / a.steps
    launches = hc.kernel_launches() - launches0 + per_replay * a.steps
    t = time.perf_counter()
    for _ in range(a.steps):
        pend = [hc.run_join_async(q, l, stream=side, **o) for q, l, o in zip(qs, idx, opts)]
        counts = [p.count() for p in pend]
    torch.cuda.synchronize()
    sep_ms = (time.perf_counter() - t) * 1e3 / a.steps
    clocks = sampler.stop()
    total = sum(sep_counts)
    line = {"metric": "join output tuples/s (batched triangle/4-clique on induced R-MAT subgraphs)",
            "value": total / (batched_ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": batched_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic (seeded R-MAT)",
            "config": {"workload": f"512 queries (triangle/4-clique 50/50) on induced subgraphs of R-MAT scale "
                                   f"{a.scale} ef {a.edge_factor} E+, edges log-uniform {lo_e:g}..{hi_e:g}",
                       "tuples": total, "edges_min": int(min(ix[0].n for ix in idx)),
                       "edges_max": int(max(ix[0].n for ix in idx)),
                       "separate_launches_ms_per_step": sep_ms,
                       "speedup_vs_separate": sep_ms / batched_ms, "graph_replay": True,
                       "tuning_groups": len(tuner.cache), "tune_s": round(tune_s, 1),
                       "prep_s": round(prep_s, 1), "counts_equal_separate": True},
            "gpu_launches": launches, "clocks": clocks}
    print(json.dumps(line), flush=True)


def order_workload(a, world, rank, local):
    """Loop-order sweep (Sec. 5.3, the paper's order study): the 4-clique on
    R-MAT E+ counted under every loop order (shares 1, each order's indexes in
    the attribute orders it needs), beside the order hc_choose_plan picks from
    the cost model.  The metric is the chosen plan's throughput."""
    import itertools

    import numpy as np
    import torch

    import __graft_entry__
    import datagen

    __graft_entry__.build()
    import paper_2502_06715_gb300 as hc

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    t = time.perf_counter()
    sym = datagen.rmat_graph(a.scale, a.edge_factor, a.seed + rank, device=f"cuda:{local}")
    ep = datagen.scatter_order(datagen.orient_lt(sym), a.seed)
    gen_s = time.perf_counter() - t
    d = torch.from_numpy(ep.view(np.int32)).to(dev)
    q = hc.FOUR_CLIQUE
    ix = {ao: hc.build_index(d, ao) for ao in (0, 1)}
    chosen, chosen_shares = hc.choose_plan(q, [ix[0]] * len(q.atoms), 1)

    def timed(order, steps):
        qo = q.with_order(order)
        idx = [ix[qo.attr_order(j)] for j in range(len(q.atoms))]
        best, cnt = float("inf"), 0
        for _ in range(steps):
            r = hc.run_join(qo, idx, time_kernels=True)
            best, cnt = min(best, r.ms_join_kernel), r.count
        return best, cnt

    for _ in range(a.warmup):
        timed(chosen, 1)
    sampler = ClockSampler(local)
    times, counts = {}, set()
    for order in itertools.permutations(range(q.n_vars)):
        ms, cnt = timed(order, a.steps)
        times["".join("XYZU"[v] for v in order)] = round(ms, 2)
        counts.add(cnt)
    clocks = sampler.stop()
    if len(counts) != 1:
        raise SystemExit(f"orders disagree on the count: {sorted(counts)}")
    cnt = counts.pop()
    key = "".join("XYZU"[v] for v in chosen)
    ranked = sorted(times, key=times.get)
    # the order chosen by measurement among the cost model's best four
    from paper_2502_06715_gb300.autotune import Tuner, ranked_orders

    tuned, tuned_ms = Tuner(reps=a.steps).tune_order(q, lambda j, ao: ix[ao], top_k=4)
    tkey = "".join("XYZU"[v] for v in tuned)
    model_rank = ["".join("XYZU"[v] for v in o) for o in ranked_orders(q, [ix[0]] * len(q.atoms))]
    if rank == 0:
        line = {"metric": "join output tuples/s (R-MAT 4-clique, order chosen by the cost model)",
                "value": cnt / (times[key] / 1e3), "unit": UNIT, "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": times[key], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u32", "data": "synthetic (seeded R-MAT)",
                "config": {"workload": f"4-clique on E+ of R-MAT scale {a.scale} ef {a.edge_factor}, count, shares 1, "
                                       f"every loop order (search kernel time, best of {a.steps})",
                           "tuples": cnt, "chosen_order": key, "chosen_rank": ranked.index(key) + 1,
                           "measured_choice": {"order": tkey, "rank": ranked.index(tkey) + 1,
                                               "ms": times[tkey],
                                               "tried": {"".join("XYZU"[v] for v in o): round(m, 2)
                                                         for o, m in tuned_ms.items()}},
                           "cost_model_ranking": model_rank,
                           "orders": len(times), "best_order": ranked[0], "best_ms": times[ranked[0]],
                           "worst_order": ranked[-1], "worst_ms": times[ranked[-1]], "ms_by_order": times,
                           "generate_s": round(gen_s, 1)},
                "clocks": clocks}
        print(json.dumps(line), flush=True)


def skew_workload(a, world, rank, local):
    """The paper's share study (Sec. 1, Examples 1-3: the triangle at 4096x1x1,
    16x16x16 and 64x64x1 cells, each cell a thread of work) on this GPU: for
    each share vector, the search kernel's time (count mode) and, per cell,
    its work units and the SM cycles its warps spent on it.  Skew is the
    largest cell over the mean cell (of cycles, and of work).  One JSON line
    per share vector."""
    import numpy as np
    import torch

    import __graft_entry__

    __graft_entry__.build()
    import paper_2502_06715_gb300 as hc

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ep, gen_s = make_graph(a, rank, device=f"cuda:{local}")
    d = torch.from_numpy(ep.view(np.int32)).to(dev)
    ix = hc.build_index(d, 0)
    q = hc.TRIANGLE
    knobs = {"item_grain": a.grain or 64, "merge_min": 0xFFFFFFFF, "merge_ratio": 1}
    for sh in ([1, 1, 1], [64, 1, 1], [4096, 1, 1], [16, 16, 16], [64, 64, 1]):
        for _ in range(max(1, a.warmup)):
            hc.run_join(q, [ix] * 3, shares=sh, **knobs)
        ms = []
        for _ in range(max(1, a.steps)):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            r = hc.run_join(q, [ix] * 3, shares=sh, time_kernels=True, **knobs)
            e1.record()
            torch.cuda.synchronize()
            ms.append((e0.elapsed_time(e1), r.ms_join_kernel))
        prof = hc.run_join(q, [ix] * 3, shares=sh, cell_profile=True, **knobs).cell_profile.cpu().numpy()
        work, cyc = prof[:, 0].astype(np.float64), prof[:, 1].astype(np.float64)
        line = {"metric": "per-cell skew (triangle)", "workload": workload_name(a).replace("; materialize", ""),
                "shares": sh, "cells": int(prof.shape[0]), "count": r.count,
                "join_ms": round(statistics.median(m[0] for m in ms), 3),
                "search_ms": round(statistics.median(m[1] for m in ms), 3),
                "cycles_sum": float(cyc.sum()), "cycles_max_cell": float(cyc.max()),
                "cycle_skew_max_over_mean": round(float(cyc.max() / max(cyc.mean(), 1.0)), 2),
                "work_sum": float(work.sum()), "work_max_cell": float(work.max()),
                "work_skew_max_over_mean": round(float(work.max() / max(work.mean(), 1.0)), 2),
                "note": "cycles: SM clock cycles of the warps' work items of each cell, summed (the analogue of "
                        "a thread's time); the join itself runs every cell's items on all SMs at once"}
        if rank == 0:
            print(json.dumps(line), flush=True)


def build_workload(a, world, rank, local):
    """CoCo construction of the R-MAT E+ relation (LSD radix sort + run-boundary
    scan) as the step.  Metric: effective index-build GB/s, the algorithmic
    bytes 8N (pairs read) + 4N (V2) + 8 l1 + 4 (V1, O1) over the step time."""
    import numpy as np
    import torch

    import __graft_entry__

    __graft_entry__.build()
    import paper_2502_06715_gb300 as hc

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ep, gen_s = make_graph(a, rank, device=f"cuda:{local}")
    n = int(ep.shape[0])
    d = torch.from_numpy(ep.view(np.int32)).to(dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        ix = hc.build_index(d, 0, stream=stream, time_kernels=True)
        r = (ix.l1, ix.ms_radix_passes, ix.n_radix_passes, ix.ms_boundary)
        ix.free()
        return r

    for _ in range(a.warmup):
        l1 = step()[0]
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    launches0 = hc.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    radix_ms, radix_n, bnd_ms = 0.0, 0, 0.0
    e0.record(stream)
    for _ in range(a.steps):
        l1, rm, rn, bm = step()
        radix_ms += rm
        radix_n += rn
        bnd_ms += bm
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    launches = hc.kernel_launches() - launches0
    ms = e0.elapsed_time(e1) / a.steps
    b_build = 8 * n + 4 * n + 8 * l1 + 4
    value = b_build / (ms / 1e3) / 1e9
    peak, peak_kind = measured_hbm_peak()
    pass_ms = radix_ms / max(1, radix_n)
    achieved = 16.0 * n / (pass_ms / 1e3) / 1e9
    bnd_alg = 8 * n + 4 * n + 8 * l1 + 4  # keys read; V2, V1, O1 written
    roofline = {"bound": "hbm", "kernel": "onesweep_kernel (radix pass)", "achieved": round(achieved, 1),
                "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": profiled_traffic(BUILD_PROFILE_NOTE, ("hc_sort.cu", "hc_internal.cuh")),
                "alg_bytes_per_launch": 16 * n, "avg_launch_ms": round(pass_ms, 4),
                "passes_per_step": radix_n / a.steps,
                "boundary_kernel": {"achieved": round(bnd_alg / (bnd_ms / a.steps / 1e3) / 1e9, 1),
                                    "avg_launch_ms": round(bnd_ms / a.steps, 4)}}

    e2e = None
    if not a.no_e2e:
        host = torch.from_numpy(ep.view(np.int32)).pin_memory()
        dbuf = torch.empty_like(d)

        def e2e_step():
            dbuf.copy_(host, non_blocking=True)
            ix = hc.build_index(dbuf, 0, stream=stream)
            got = ix.l1  # read back by the library (its control block)
            ix.free()
            return got

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(a.steps):
            e2e_step()
        torch.cuda.synchronize()
        e2e_ms = (time.perf_counter() - t0) * 1e3 / a.steps
        e2e = {"value": b_build / (e2e_ms / 1e3) / 1e9, "unit": "GB/s", "h2d_bytes_per_step": 8 * n,
               "d2h_bytes_per_step": 128, "ms_per_step": e2e_ms}

    cpu = None
    if not a.no_cpu_baseline and rank == 0 and world == 1:
        import oracle

        rng = np.random.default_rng(12345)
        m = min(n, 24_000_000)
        sample = np.ascontiguousarray(ep[np.sort(rng.choice(n, size=m, replace=False))])
        t0 = time.perf_counter()
        v1, o1, v2 = oracle.coco_build(sample, 0)
        dt = time.perf_counter() - t0
        cpu = {"value": (12 * m + 8 * v1.shape[0] + 4) / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"CoCo build of a seeded random sample of {m} of the {n} rows ({dt:.2f} s, one thread)"}

    if rank == 0:
        line = {"metric": "index-build GB/s (CoCo of R-MAT E+)", "value": value, "unit": "GB/s", "n_gpus": world,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic (seeded R-MAT)",
                "config": {"workload": f"build_index of E+ (x<y) of R-MAT scale {a.scale} ef {a.edge_factor}, "
                                       f"scrambled, symmetrised, deduplicated, rows in random order",
                           "rows": n, "l1": int(l1), "alg_bytes_per_step": b_build,
                           "l2": "inputs larger than L2 (%.0f MB of pairs)" % (8 * n / 1e6),
                           "generate_s": round(gen_s, 1)},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": launches}
        print(json.dumps(line), flush=True)


def tensor_relations(a, rank: int, device):
    """Host relations of the k-ary workloads (Sec. 6 tensor data), the query's
    atoms, a description and the closed-form count (or None).  lw: the first
    four relations of ST-Dense ([n]^3 cubes, n^4 results) or ST-Sparse (n^3
    distinct uniform tuples of [10 n]^3).  ct: the last three, F x [m] x [m];
    with --ct-first paper the first-attribute sets are ST-Dense's {0,1},
    {0,2}, {1,2} (no common value: 0 results, C22), with common all three
    take {0,1} (2 m^3 results on ST-Dense)."""
    import numpy as np

    import datagen

    if a.workload == "lw":
        n = a.lw_n
        atoms = [(0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)]
        if a.tensor == "dense":
            cube = datagen.full_cube(n)
            return atoms, [cube] * 4, f"Loomis-Whitney over ST-Dense's four [{n}]^3 relations (Sec. 6), count", n ** 4
        rels = datagen.st_sparse(n=n, domain=10 * n, m=1, m_domain=1, seed=a.seed + rank, device=device)[:4]
        return atoms, rels, (f"Loomis-Whitney over ST-Sparse's first four relations ({n ** 3} distinct uniform "
                             f"tuples of [{10 * n}]^3 each, Sec. 6), count"), None
    m = a.ct_m
    atoms = [(0, 1, 2), (0, 1, 3), (0, 2, 3)]
    sets = [(0, 1), (0, 2), (1, 2)] if a.ct_first == "paper" else [(0, 1)] * 3
    if a.tensor == "dense":
        rels = [datagen.prefixed_square(np.array(f, dtype=np.uint32), m) for f in sets]
        expect = 0 if a.ct_first == "paper" else 2 * m ** 3
        return atoms, rels, (f"Clover-Triangle over ST-Dense's F x [{m}] x [{m}] relations, F = {sets} "
                             f"(Sec. 6), count"), expect
    rels = datagen.st_sparse(n=1, domain=1, m=m, m_domain=10 * m, seed=a.seed + rank, device=device)[4:]
    if a.ct_first != "paper":  # the same first values {0, 1} in all three
        rels = [_common_first(r) for r in rels]
    return atoms, rels, (f"Clover-Triangle over ST-Sparse's last three relations ({m}^2 distinct uniform pairs of "
                         f"[{10 * m}]^2 per first value, first values {sets}, Sec. 6), count"), None


def _common_first(r):
    """Relabel a relation's two first-attribute values to 0 and 1 (rows stay distinct)."""
    import numpy as np

    lo = r[:, 0].min()
    out = r.copy()
    out[:, 0] = (r[:, 0] != lo).astype(np.uint32)
    return out[np.lexsort(out.T[::-1])]


def tensor_sample(a, atoms, host_rels, device):
    """Bounded sample of the k-ary workload: the query restricted to
    X < fx and Y < fy (X = variable 0 of LW, variable 1 of CT; Y the next).
    For LW, R4(Y,Z,U) keeps only rows whose (y, z) occurs in the sampled R1
    (an exact semi-join reduction, found with torch.isin; no join
    arithmetic).  Returns the sampled relations, a description and the
    restriction ((variable, bound), (variable, bound))."""
    import numpy as np
    import torch

    if a.workload == "lw":
        n = a.lw_n
        fx, fy = (min(n, 32), min(n, 16)) if a.tensor == "dense" else (max(1, n // 4), 10 * n)
        R1, R2, R3, R4 = host_rels
        r1 = R1[(R1[:, 0] < fx) & (R1[:, 1] < fy)]
        r2 = R2[(R2[:, 0] < fx) & (R2[:, 1] < fy)]
        r3 = R3[R3[:, 0] < fx]
        k1 = torch.from_numpy((r1[:, 1].astype(np.int64) << 32) | r1[:, 2].astype(np.int64)).to(device)
        k4 = torch.from_numpy((R4[:, 0].astype(np.int64) << 32) | R4[:, 1].astype(np.int64)).to(device)
        keep = torch.isin(k4, torch.unique(k1)).cpu().numpy()
        del k1, k4
        sample = [r1, r2, r3, R4[keep]]
        desc = f"LW with x < {fx} and y < {fy}"
        restriction = ((0, fx), (1, fy))
    else:
        m = a.ct_m
        fx, fy = min(m, 16), min(m, 256)
        R5, R6, R7 = host_rels  # R5(U,X,Y), R6(U,X,Z), R7(U,Y,Z)
        sample = [R5[(R5[:, 1] < fx) & (R5[:, 2] < fy)], R6[R6[:, 1] < fx], R7[R7[:, 1] < fy]]
        desc = f"CT with x < {fx} and y < {fy}"
        restriction = ((1, fx), (2, fy))
    sample = [np.ascontiguousarray(r) for r in sample]
    return sample, f"{desc}, rows {[int(r.shape[0]) for r in sample]}", restriction


def kary_workload(a, world, rank, local):
    """LW or CT (Table "Queries") over Sec. 6's tensor relations
    (tensor_relations), count mode, in the loop order hc_choose_korder picks;
    the step is one k-ary join over resident 3-level CoCo indexes (built
    once, timed separately).  Metric: results per second.  Roofline of the
    search kernel: 4 bytes per unit of the work measure (sum over loops and
    bindings of lists x shortest list) per launch.  A bounded sample
    (tensor_sample) is counted by the oracle and by the GPU on the same
    rows."""
    import numpy as np
    import torch

    import __graft_entry__

    __graft_entry__.build()
    import paper_2502_06715_gb300 as hc

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    dist = None
    if world > 1:  # independent replicas (seed + rank), no data-path collective
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    t0 = time.perf_counter()
    atoms, host_rels, desc, closed = tensor_relations(a, rank, f"cuda:{local}")
    gen_s = time.perf_counter() - t0
    na = len(atoms)
    rows = [torch.from_numpy(r.view(np.int32)).to(dev) for r in host_rels]
    q = hc.KQuery(4, tuple(atoms))
    ixs = [hc.build_kindex(rows[j], None, stream=stream) for j in range(na)]
    q = q.with_order(hc.choose_korder(q, ixs))  # Sec. 5.2-5.3 from the built indexes' statistics
    kshares = tuple(int(x) for x in a.kshares.split(",")) if a.kshares else (1, 1, 1, 1)
    per_atom = hc.atom_shares(q, kshares)

    def kbuild(j, r, **kw):
        if kshares == (1, 1, 1, 1):
            return hc.build_kindex(r, q.level_cols(j), stream=stream, **kw)
        return hc.build_kindex(r, q.level_cols(j), stream=stream, seeds=per_atom[j][0], shares=per_atom[j][1], **kw)

    ixs = [ix if ix.level_cols == q.level_cols(j) and kshares == (1, 1, 1, 1) else kbuild(j, rows[j])
           for j, ix in enumerate(ixs)]
    tb = [kbuild(j, rows[j], time_kernels=True) for j in range(na)]
    build_ms = [ix.ms_sort + ix.ms_levels for ix in tb]
    del tb
    stats = hc.run_kjoin(q, ixs, stats=True, stream=stream)
    expect = stats.count
    if closed is not None and expect != closed:
        raise RuntimeError(f"count {expect} != closed form {closed}")
    work = stats.work

    def step():
        return hc.run_kjoin(q, ixs, stream=stream, time_kernels=True, item_grain=a.grain,
                            block_threads=a.threads)

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
        torch.cuda.synchronize()
    sampler = ClockSampler(local)
    launches0 = hc.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kern_ms = 0.0
    e0.record(stream)
    for _ in range(a.steps):
        r = step()
        if r.count != expect:
            raise RuntimeError("the count changed between steps")
        kern_ms += r.ms_join_kernel
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    launches = hc.kernel_launches() - launches0
    ms_total, results = e0.elapsed_time(e1), float(expect) * a.steps
    if dist:  # the slowest rank's time, the results of all ranks
        ms_total, results = combine_ranks(ms_total, results, dist, dev)
    ms = ms_total / a.steps
    value = results / (ms_total / 1e3)
    peak, peak_kind = measured_hbm_peak()
    kms = kern_ms / a.steps
    metric = "LW results/s (count)" if a.workload == "lw" else "CT results/s (count)"
    achieved = 4.0 * work / (kms / 1e3) / 1e9
    # the committed capture covers LW over ST-Dense's [512]^3 cubes in one cell
    profiled = (a.workload == "lw" and a.lw_n == 512 and a.tensor == "dense" and kshares == (1, 1, 1, 1))
    roofline = {"bound": "hbm", "kernel": "kjoin_kernel<4> (k-ary search)", "achieved": round(achieved, 1),
                "launches_per_step": 1,
                "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": profiled_traffic(KJOIN_PROFILE_NOTE, ("hc_kary.cu", "hc_internal.cuh")) if profiled else None,
                "alg_bytes_per_launch": 4 * work, "avg_launch_ms": round(kms, 3),
                "note": "work measure x 4 B; short lists are L1/L2-resident, so this can exceed what DRAM moves"}

    e2e = None
    if not a.no_e2e:
        hosts = [torch.from_numpy(r.view(np.int32)).pin_memory() for r in host_rels]
        bufs = [torch.empty_like(r) for r in rows]

        def e2e_step():
            for b, h in zip(bufs, hosts):
                b.copy_(h, non_blocking=True)
            xs = [kbuild(j, bufs[j]) for j in range(na)]
            c = hc.run_kjoin(q, xs, stream=stream).count
            for x in xs:
                x.free()
            return c

        e2e_step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(a.steps):
            e2e_step()
        torch.cuda.synchronize()
        e2e_total, e2e_results = (time.perf_counter() - t0) * 1e3, float(expect) * a.steps
        if dist:
            e2e_total, e2e_results = combine_ranks(e2e_total, e2e_results, dist, dev)
        e2e_ms = e2e_total / a.steps
        e2e = {"value": e2e_results / (e2e_total / 1e3), "unit": "tuples/s",
               "h2d_bytes_per_step": sum(12 * r.shape[0] for r in host_rels), "d2h_bytes_per_step": 8,
               "ms_per_step": e2e_ms,
               "includes": "H2D of the relations, their 3-level CoCo builds, the join, the count read back"}

    cpu = None
    if not a.no_cpu_baseline and rank == 0 and world == 1:
        import oracle

        sample, sdesc, _ = tensor_sample(a, atoms, host_rels, dev)
        threads = min(64, os.cpu_count() or 1)
        t0 = time.perf_counter()
        c = oracle.kgj(4, atoms, sample, order=list(q.loop_order()), nthreads=threads)
        dt = time.perf_counter() - t0
        sx = [kbuild(j, torch.from_numpy(r.view(np.int32)).to(dev)) for j, r in enumerate(sample)]
        got = hc.run_kjoin(q, sx).count
        if got != c:
            raise RuntimeError(f"sampled parity: GPU {got} != oracle {c}")
        cpu = {"value": c / dt, "unit": "tuples/s", "cores": threads, "kind": "oracle",
               "sample": f"{sdesc} ({c} results, {dt:.1f} s incl. the trie sorts, {threads} threads over the "
                         f"first loop's values; the GPU counts the same sample equal)"}

    if rank == 0:
        v2_bytes = sum(4 * r.shape[0] for r in host_rels)
        tname = "Dense" if a.tensor == "dense" else "Sparse"
        line = {"metric": metric, "value": value, "unit": "tuples/s", "n_gpus": world,
                "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32",
                "data": f"synthetic (ST-{tname} shape, seeded)",
                "config": {"workload": desc, "rows_per_relation": [int(r.shape[0]) for r in host_rels],
                           "order": list(q.loop_order()), "shares": list(kshares), "n_cells": int(stats.n_cells),
                           "count": int(expect), "work": int(work),
                           "index_build_ms": [round(b, 3) for b in build_ms],
                           "l2": ("inputs larger than L2: %.0f MB of V_2 over the indexes" if v2_bytes > 129e6
                                  else "inputs within L2: %.0f MB of V_2 over the indexes") % (v2_bytes / 1e6),
                           "generate_s": round(gen_s, 1)},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": launches}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def serve_workload(a, world, rank, local):
    """Serving: 10,000 Poisson-arriving requests (60% triangle, 30% 4-cycle,
    10% 4-clique) over four resident relations, against serial execution."""
    import numpy as np
    import torch

    import __graft_entry__
    import datagen

    __graft_entry__.build()
    import paper_2502_06715_gb300 as hc
    from paper_2502_06715_gb300.serve import Request, Server, fifo_latencies, serve_serial

    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    t = time.perf_counter()
    nv = 1 << 24
    rels = {"rmat23": datagen.rmat_graph(a.scale, a.edge_factor, 5, device=dev),
            "u50M": datagen.uniform_relation(50_000_000, nv, 51, device=dev),
            "u10M": datagen.uniform_relation(10_000_000, nv, 52, device=dev),
            "u1M": datagen.uniform_relation(1_000_000, nv, 53, device=dev)}
    idx = {k: hc.build_index(torch.from_numpy(v.view(np.int32)).to(dev), 0) for k, v in rels.items()}
    gen_s = time.perf_counter() - t
    deg = np.bincount(rels["rmat23"][:, 0], minlength=nv)
    pool = np.nonzero(deg <= 64)[0].astype(np.uint32)
    rng = np.random.default_rng(5)
    names = sorted(rels)
    n = a.serve_requests
    reqs = []
    for i in range(n):
        u = rng.random()
        base = hc.TRIANGLE if u < 0.6 else (hc.FOUR_CYCLE if u < 0.9 else hc.FOUR_CLIQUE)
        rel_names = tuple(names[k] for k in rng.integers(0, len(names), size=len(base.atoms)))
        size = int(np.exp(rng.uniform(np.log(4096), np.log(131072))))
        f = np.unique(pool[rng.integers(0, pool.shape[0], size=size)])
        if a.serve_select == "rmat" and "rmat23" not in rel_names:
            reqs.append(Request(i, base, rel_names, None))  # the uniform relations as they are
            continue
        q = base.with_atoms([(v, None) for v in range(base.n_vars)])
        reqs.append(Request(i, q, rel_names, f))
    srv = Server(idx, budget_bytes=120 << 30, max_inflight=8, device=dev)
    serve_serial(srv, reqs[:200])  # warm-up
    t = time.perf_counter()
    serial = serve_serial(srv, reqs)
    serial_s = time.perf_counter() - t
    service = [o.done - o.admitted for o in sorted(serial, key=lambda o: o.rid)]
    alone = {o.rid: o.count for o in serial}
    mu = n / serial_s
    rates = {}
    sampler = ClockSampler(local)
    for rho in (0.5, 0.8, 0.95):
        lam = rho * mu
        arr = np.cumsum(np.random.default_rng(int(rho * 100)).exponential(1.0 / lam, size=n))
        for r, at in zip(reqs, arr):
            r.arrival = float(at)
        t = time.perf_counter()
        out = srv.run(reqs)
        span = time.perf_counter() - t
        lat = np.array([o.latency for o in out])
        if {o.rid: o.count for o in out} != alone:
            raise SystemExit("served counts differ from the same requests run alone")
        slat = np.array(fifo_latencies(service, list(arr)))
        rates[str(rho)] = {"arrival_rate_per_s": lam, "p50_ms": float(np.percentile(lat, 50) * 1e3),
                           "p99_ms": float(np.percentile(lat, 99) * 1e3), "throughput_per_s": n / span,
                           "serial_p50_ms": float(np.percentile(slat, 50) * 1e3),
                           "serial_p99_ms": float(np.percentile(slat, 99) * 1e3)}
    clocks = sampler.stop()
    top = rates["0.95"]
    line = {"metric": "serving p50/p99 latency vs serial (join requests)", "value": top["p99_ms"],
            "unit": "ms (p99 at 0.95 of serial throughput)", "n_gpus": world, "steps": n, "warmup": 200,
            "ms_per_step": 1e3 * serial_s / n, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic (seeded R-MAT + uniform relations)",
            "config": {"workload": f"{n:,} Poisson requests, 60% Q1 / 30% Q2 / 10% Q6 over R-MAT scale 23 ef 16 "
                                   "(symmetric) + uniform 50M/10M/1M pairs on 2^24 vertices; " + (
                                       "every variable restricted to a request vertex sample (4096..131072 "
                                       "vertices of R-MAT degree <= 64)" if a.serve_select == "all" else
                                       "requests with an R-MAT atom restricted to a request vertex sample "
                                       "(4096..131072 vertices of R-MAT degree <= 64), the others over the "
                                       "uniform relations as they are"),
                       "unrestricted_requests": sum(1 for r in reqs if r.restrict is None),
                       "rows": {k: int(v.shape[0]) for k, v in rels.items()}, "max_inflight": 8,
                       "hbm_budget_gb": 120, "serial_throughput_per_s": mu, "rates": rates,
                       "counts_equal_alone": True, "generate_s": round(gen_s, 1)},
            "clocks": clocks}
    print(json.dumps(line), flush=True)


def reference_arm(a, world, rank):
    """The oracle as it stands, on the host cores, over a bounded sample of
    the same workload each step."""
    if rank != 0:
        return
    if a.workload in ("lw", "ct"):
        return reference_tensor(a, world)
    if a.workload != "triangle":
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm covers the triangle (default), lw "
                                                              "and ct workloads"}), flush=True)
        return
    ep, gen_s = make_graph(a, 0, device=None if os.environ.get("HC_GEN_CPU") else _maybe_cuda())
    times, counts = [], []
    desc, cores = "", 1
    for i in range(a.warmup + a.steps):
        cnt, dt, cores, desc = run_oracle_sample(ep, a.cpu_frac, 12345)
        if i >= a.warmup:
            times.append(dt)
            counts.append(cnt)
    total = sum(counts) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": total, "unit": UNIT, "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic (seeded R-MAT)",
            "config": {"workload": workload_name(a), "scale": a.scale, "edge_factor": a.edge_factor,
                       "sample_frac": a.cpu_frac},
            "cpu_baseline": {"kind": "oracle", "cores": cores, "sample": desc, "value": total, "unit": UNIT},
            "e2e": {"value": total, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def reference_tensor(a, world):
    """The k-ary oracle on the k-ary workload's bounded sample, each step."""
    import oracle

    dev = _maybe_cuda() or "cpu"
    atoms, host_rels, desc, _ = tensor_relations(a, 0, None if dev == "cpu" else dev)
    sample, sdesc, _ = tensor_sample(a, atoms, host_rels, dev)
    threads = min(64, os.cpu_count() or 1)
    times, counts = [], []
    for i in range(a.warmup + a.steps):
        t0 = time.perf_counter()
        c = oracle.kgj(4, atoms, sample, nthreads=threads)
        dt = time.perf_counter() - t0
        if i >= a.warmup:
            times.append(dt)
            counts.append(c)
    total = sum(counts) / sum(times)
    unit = "tuples/s"
    metric = "LW results/s (count)" if a.workload == "lw" else "CT results/s (count)"
    line = {"impl": "reference", "metric": metric, "value": total, "unit": unit,
            "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": f"synthetic (ST-{'Dense' if a.tensor == 'dense' else 'Sparse'} shape, seeded)",
            "config": {"workload": desc},
            "cpu_baseline": {"kind": "oracle", "cores": threads, "value": total, "unit": unit,
                             "sample": f"{sdesc} ({counts[0]} results, trie sorts included, {threads} threads)"},
            "e2e": {"value": total, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _maybe_cuda():
    try:
        import torch

        return "cuda:0" if torch.cuda.is_available() else None
    except Exception:
        return None


if __name__ == "__main__":
    main()
