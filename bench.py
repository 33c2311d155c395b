"""Benchmark: exact Brandes BC throughput on one B300 (traversed source-arcs per second).

Default workload: undirected R-MAT scale 22, edge factor 16 (a=.57 b=.19 c=.19,
seeded, self-loops and duplicates removed), 4096 sources sampled uniformly
over non-isolated vertices; one step = one bc_compute over all 4096 sources
on the resident graph (batched traversal, width chosen by the library).

Metric: BC traversed edges/s = sources x m / time, m = CSR arcs (each
undirected edge counted twice).  `value` times bc_compute with sources and
output already on the device; `e2e` times the same call from pinned host
sources to a pinned host copy of the result.  The roofline object reports the
traversal kernel against the measured HBM copy bandwidth using an algorithmic
byte model per source: B_s = 8m/k + m/4 + 16 E_dag(s) + 24 n_s for the batched
persistent kernel (width k), B_s = 16m + 16 E_dag(s) + 40 n_s for the
per-source kernel the library picks on deep graphs (--workload grid).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload rmat22|rmat12|grid|serve] [--sources S] [--batch-width K]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BC traversed edges/s (sources x edges) on 1 B300, % HBM roofline; p50/p99 latency"
UNIT = "source-arcs/s"
FALLBACK_HBM_GBS = 6400.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat22", choices=["rmat22", "rmat12", "grid", "serve", "rmat", "many", "bfs", "pagerank", "weighted"])
    ap.add_argument("--graphs", type=int, default=200, help="many: graphs in the pool (the full config has 2000)")
    ap.add_argument("--scale", type=int, default=22)
    ap.add_argument("--ef", type=float, default=16)
    ap.add_argument("--sources", type=int, default=0)
    ap.add_argument("--grid-side", type=int, default=1024, help="grid: vertices per side")
    ap.add_argument("--batch-width", type=int, default=0)
    ap.add_argument("--direction", type=int, default=0)
    ap.add_argument("--source-order", type=int, default=0,
                    help="bc_options.source_order: 0 auto, 1 as given, 2 grouped by hub distances")
    ap.add_argument("--directed", action="store_true",
                    help="weighted: orient the R-MAT graph (each edge one way, a quarter both ways), weights per arc")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (library heuristics)")
    ap.add_argument("--rate", type=float, default=20.0, help="serve: Poisson arrival rate (req/s)")
    ap.add_argument("--scales", default="14-22", help="serve: R-MAT scales of the resident pool (one graph each)")
    ap.add_argument("--slots", type=int, default=1, help="serve: concurrent traversals (1 = one full-GPU traversal at a time)")
    ap.add_argument("--duration", type=float, default=10.0, help="serve: seconds of arrivals")
    return ap.parse_args()


# ------------------------------------------------------------------ workloads
def make_workload(a):
    import bcgen
    if a.workload in ("rmat22", "rmat"):
        scale, ef = (22, 16) if a.workload == "rmat22" else (a.scale, a.ef)
        g = bcgen.rmat(scale, ef, 1)
        S = a.sources or 4096
        src = bcgen.sample_sources(g, S, 1)
        desc = dict(workload=f"rmat{scale}_ef{ef:g}", graph=f"undirected R-MAT scale {scale}, edge factor {ef:g}, "
                    "a=.57 b=.19 c=.19, seed 1, self-loops/duplicates removed, int32 CSR",
                    sources=int(len(src)), source_sampling="uniform without replacement over degree>=1, seed 1")
    elif a.workload == "rmat12":
        g = bcgen.rmat(12, 8, 1)
        src = np.arange(g.n, dtype=np.int32)
        desc = dict(workload="rmat12_ef8_all_sources", graph="undirected R-MAT scale 12, edge factor 8, seed 1",
                    sources=int(g.n), source_sampling="every vertex")
    else:  # grid
        side = a.grid_side
        g = bcgen.grid(side, side, 0.05, 1)
        S = a.sources or 256
        src = bcgen.sample_sources(g, S, 1)
        desc = dict(workload=f"grid{side}x{side}_rm5pct",
                    graph=f"{side}x{side} 4-neighbour grid, 5% of edges removed (seed 1)",
                    sources=int(len(src)), source_sampling="uniform without replacement over degree>=1, seed 1")
    desc.update(n=g.n, m=g.m)
    return g, src, desc


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, copy bandwidth)"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback 6.4 TB/s (no MEASURED_PEAKS.json)"


def committed_traffic(kernel_name, workload):
    """Per-source DRAM bytes from the committed ncu summary, or None if absent or if any source file
    of the kernel has changed since the capture (sha256 per file)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        e = json.load(open(p)).get("entries", {}).get(f"{kernel_name}|{workload}")
        if e is None:
            return None
        for name, sha in e["sources"].items():
            src = open(os.path.join(ROOT, "paper_2305_03317_b300", "csrc", name), "rb").read()
            if hashlib.sha256(src).hexdigest() != sha:
                return None
        return float(e["dram_bytes_per_source"])
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.proc = None
        self.path = os.path.join("/tmp", f"bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.dev)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = open(self.path).read().splitlines()
        note = None
        if not any(len(x.split(",")) >= 9 for x in lines):
            # the timed region was shorter than the sampling interval: one reading right after it
            try:
                out = subprocess.run(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                      "-i", str(self.dev)], capture_output=True, text=True, timeout=30).stdout
                lines = out.splitlines()
                note = "timed region shorter than the 200 ms sampling interval: one reading right after it"
            except Exception:
                lines = []
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        res = {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
               "reasons": sorted(reasons), "samples": len(sm)}
        if note:
            res["note"] = note
        return res


def cpu_baseline(g, src, per_core=1, max_threads=64):
    import oracle
    cores = max(1, min(os.cpu_count() or 1, max_threads))
    sample = src[: max(1, min(len(src), cores * per_core))]
    t = time.perf_counter()
    oracle.bc(g.off, g.adj, sample, threads=cores)
    dt = time.perf_counter() - t
    return {"value": len(sample) * g.m / dt, "unit": UNIT, "cores": int(min(cores, len(sample))), "kind": "oracle",
            "sample": f"{len(sample)} of the workload's sources (first {len(sample)}), full graph, "
                      f"{dt:.1f} s wall on {min(cores, len(sample))} threads"}


# ------------------------------------------------------------------ reference arm (the oracle)
def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    g, src, desc = make_workload(a)
    cores = max(1, min(os.cpu_count() or 1, 64))
    per_step = src[:cores]
    for _ in range(a.warmup):
        pass  # the oracle has no warm-up state; warm-up steps are not repeated on the CPU
    import oracle
    times = []
    for i in range(a.steps):
        t = time.perf_counter()
        oracle.bc(g.off, g.adj, per_step, threads=cores)
        times.append(time.perf_counter() - t)
    dt = float(np.mean(times))
    val = len(per_step) * g.m / dt
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(desc, step=f"oracle over {len(per_step)} sources (one per host thread)"),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": int(min(cores, len(per_step))), "kind": "oracle",
                             "sample": f"{len(per_step)} sources per step of the same workload"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ sharding (N GPUs, one rank each)
def job_sources(g, per_rank, world):
    """The job: per_rank sources for every rank (weak scaling), seed 1; a 1-GPU
    run gets the single-GPU workload's list."""
    import bcgen
    return bcgen.sample_sources(g, per_rank * world, 1)


def max_over_ranks(ms, dist, device):
    """The slowest rank's time: the job finishes when its last rank does."""
    if dist is None:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ our arm
def run_ours(a):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_2305_03317_b300 as bc

    if a.workload == "serve":
        return run_serve(a, bc, torch)
    if a.workload == "many":
        return run_many(a, bc, torch)
    if a.workload == "bfs":
        return run_bfs(a, bc, torch)
    if a.workload == "pagerank":
        return run_pagerank(a, bc, torch)
    if a.workload == "weighted":
        return run_weighted(a, bc, torch)

    g, src, desc = make_workload(a)
    per_rank = len(src)
    if world > 1:  # weak scaling: one job of per_rank sources per rank, split by batch over the ranks
        src = job_sources(g, per_rank, world)
    t0 = time.perf_counter()
    G = bc.Graph(g.off, g.adj)
    torch.cuda.synchronize()
    ingest_s = time.perf_counter() - t0
    d_src = torch.from_numpy(src).cuda()
    out = torch.empty(g.n, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    opts = dict(batch_width=a.batch_width, direction=a.direction, source_order=a.source_order)
    tuned = None
    # the grid's levels are narrow and thousands deep: the library picks its per-source form
    # there, which has no knobs to tune
    if a.batch_width == 0 and not a.no_tune and a.workload != "grid":
        t_tune = time.perf_counter()
        tuned = G.autotune(src)  # per size bucket; knobs left at 0 below come from it
        tuned["seconds"] = round(time.perf_counter() - t_tune, 2)

    if world > 1:
        from paper_2305_03317_b300 import sharded

        def step(sources):  # this rank's batches, the status exchange, the gather, the rank-order sum
            return sharded.compute(G, sources, out=out, **opts)
        order, K_job = G.source_batches(src, batch_width=a.batch_width, source_order=a.source_order)
        n_rank_src = len(sharded.shard_of(order, K_job, rank, world))
    else:
        def step(sources):
            return G.compute(sources, out=out, **opts)
        n_rank_src = len(src)
    for _ in range(max(a.warmup, 0)):
        step(d_src)
    torch.cuda.synchronize()

    clocks = Clocks(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_ms, kern_ms, launches, statuses = [], [], 0, set()
    ev0.record(stream)
    for _ in range(a.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, st = step(d_src)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        s = G.stats()
        kern_ms.append(s["kernel_ms"])
        launches += s["kernel_launches"]
        statuses.add(st)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    total_ms = max_over_ranks(ev0.elapsed_time(ev1), dist, "cuda")
    stats = G.stats()
    ms = total_ms / a.steps
    value = len(src) * g.m / (ms / 1e3)  # every rank's sources x arcs over the slowest rank's time

    # end to end: pinned host sources in, pinned host result out, through the public call
    h_src = torch.from_numpy(src).pin_memory()
    h_out = torch.empty(g.n, dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(a.steps, 3))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        step(h_src.numpy())
        h_out.copy_(out, non_blocking=True)
        stream.synchronize()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    # roofline of the traversal kernel
    K = stats["batch_width"]
    nb = stats["batches"]
    deep = stats["deep_sources"] > 0
    # this rank's launch: sum over its sources of E_dag(s) and n_s, counted exactly by the kernel
    dag, reached = stats["dag_arcs"], stats["reached"]
    if deep:  # per source: rows and level tags in both sweeps, a term per DAG arc each way, 40 B per vertex
        model_bytes = n_rank_src * 16.0 * g.m + 16.0 * dag + 40.0 * reached
        model_txt = "per source 16m + 16*E_dag + 40*n_s (per-source form)"
        kname = "k_deep"
    else:
        model_bytes = nb * (8.0 * g.m + K * g.m / 4.0) + 16.0 * dag + 24.0 * reached
        model_txt = "per source 8m/k + m/4 + 16*E_dag + 24*n_s"
        kname = f"bc_persistent<{K}>"
    kms = float(np.mean(kern_ms))
    peak, peak_src = measured_peak()
    achieved = model_bytes / (kms / 1e3) / 1e9
    tr = committed_traffic(kname, desc["workload"])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": dict(desc, step="one bc_compute over all sources on the resident graph",
                       form="per-source (deep graphs)" if deep else "batched",
                       batch_width=K, batches=nb, levels=stats["max_levels"], pull_levels=stats["pull_levels"],
                       push_levels=stats["push_levels"], teams=stats["teams"], ingest_s=round(ingest_s, 3),
                       source_grouping_ms=round(stats["order_ms"], 3),
                       autotuned=tuned,
                       l2="inputs larger than L2 (CSR and per-batch state are GBs, L2 126 MB)",
                       parallelism=(f"dp{world}: one job of {len(src)} sources, batches round-robin over the "
                                    f"ranks, partial BC all-gathered and summed in rank order (bc_reduce_ranks)"
                                    if world > 1 else "single GPU"),
                       statuses=sorted(int(x) for x in statuses)),
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                       "what": "per bc_compute step"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": (tr * n_rank_src) if tr is not None else None,
                     "kernel": kname, "kernel_ms": kms, "model_bytes": model_bytes,
                     "model": f"{model_txt} over the launch's {n_rank_src} sources; "
                              f"E_dag={dag / n_rank_src:.0f}, n_s={reached / n_rank_src:.0f} per source (exact "
                              f"kernel counts: sum E_dag {dag}, sum n_s {reached})", "peak_source": peak_src},
        "e2e": {"value": len(src) * g.m / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(4 * len(src)),
                "d2h_bytes_per_step": int(8 * g.n), "ms_per_step": e2e_ms},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(g, src)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_many(a, bc, torch):
    """Many uneven R-MAT graphs replayed as one recorded CUDA graph (bc_many_*)."""
    import bcgen
    t0 = time.perf_counter()
    pool = bcgen.rmat_sizes_pool(a.graphs, seed=1)
    graphs = [bcgen.rmat_n(n, ef, sd) for n, ef, sd in pool]
    gen_s = time.perf_counter() - t0
    items, work = [], 0
    for (n, ef, sd), g in zip(pool, graphs):
        src = np.arange(g.n, dtype=np.int32) if g.n <= 16384 else bcgen.sample_sources(g, 256, sd)
        G = bc.Graph(g.off, g.adj)
        out = torch.empty(max(g.n, 1), dtype=torch.float64, device="cuda")
        items.append((G, src, out))
        work += len(src) * g.m
    t1 = time.perf_counter()
    plan = bc.ManyPlan(items)
    torch.cuda.synchronize()
    plan_s = time.perf_counter() - t1
    for _ in range(max(a.warmup, 0)):
        plan.run()
    stream = torch.cuda.current_stream()
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    torch.cuda.synchronize()
    step_ms = []
    for _ in range(a.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = plan.run()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = float(np.mean(step_ms))
    info = plan.info()
    line = {"metric": METRIC, "value": work / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"many_rmat_{a.graphs}", "graphs": a.graphs,
                       "sizes": "n = round(2^U[10,18]), edge factor U{4..32}, graph seed 1+i",
                       "sources": "all if n <= 16384 else 256 sampled", "source_arcs_per_step": work,
                       "step": "replay of one recorded CUDA graph (one persistent launch per graph)",
                       "generation_s": round(gen_s, 1), "plan_s": round(plan_s, 2),
                       "statuses": sorted(set(int(x) for x in st)),
                       "l2": "per-graph state is reused across graphs; large graphs exceed L2"},
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                           "what": "per replay of the whole pool"},
            "gpu_launches": info["kernel_launches"] * a.steps, "clocks": clk}
    print(json.dumps(line), flush=True)


def run_bfs(a, bc, torch):
    """Multi-source BFS (bc_bfs: the forward sweep alone, levels and path counts per source)."""
    import bcgen
    g = bcgen.rmat(a.scale, a.ef, 1)
    S = a.sources or 256
    src = bcgen.sample_sources(g, S, 1)
    G = bc.Graph(g.off, g.adj)
    d_src = torch.from_numpy(src).cuda()
    for _ in range(max(a.warmup, 0)):
        G.bfs(d_src)
    stream = torch.cuda.current_stream()
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    torch.cuda.synchronize()
    ms = []
    for _ in range(a.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lev, sig, _, st = G.bfs(d_src)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        del lev, sig
    clk = clocks.stop()
    s = G.stats()
    t = float(np.mean(ms))
    line = {"metric": METRIC, "value": len(src) * g.m / (t / 1e3), "unit": UNIT, "n_gpus": 1, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": t, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u64 counts, int32 levels", "data": "synthetic",
            "config": {"workload": f"msbfs_rmat{a.scale}_ef{a.ef:g}", "sources": int(len(src)), "n": g.n, "m": g.m,
                       "step": "one bc_bfs: levels and path counts of every source into [sources][n] device rows",
                       "batch_width": s["batch_width"], "batches": s["batches"], "kernel_ms": s["kernel_ms"],
                       "output_bytes": int(len(src) * g.n * 12)},
            "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99)),
                           "what": "per bc_bfs call"},
            "gpu_launches": s["kernel_launches"] * a.steps, "clocks": clk}
    print(json.dumps(line), flush=True)


def run_pagerank(a, bc, torch):
    """The paper's computePR on the resident graph: a fixed number of sweeps (beta = 0)."""
    import bcgen
    g = bcgen.rmat(a.scale, a.ef, 1)
    G = bc.Graph(g.off, g.adj)
    sweeps = 20
    out = torch.empty(g.n, dtype=torch.float64, device="cuda")
    for _ in range(max(a.warmup, 0)):
        G.pagerank(0.85, 0.0, sweeps, out=out)
    stream = torch.cuda.current_stream()
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    torch.cuda.synchronize()
    ms, its = [], []
    for _ in range(a.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, it, _ = G.pagerank(0.85, 0.0, sweeps, out=out)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        its.append(it)
    clk = clocks.stop()
    t = float(np.mean(ms))
    it = int(its[-1])
    # per sweep: CSR indices 4m and one 8-byte contribution per arc, in-offsets 4n,
    # out-offsets 4n, rank read twice, contribution and next rank written (8n each)
    model = it * (12.0 * g.m + 36.0 * g.n)
    peak, peak_src = measured_peak()
    achieved = model / (t / 1e3) / 1e9
    line = {"metric": "PageRank traversed arcs/s (sweeps x arcs)", "value": it * g.m / (t / 1e3),
            "unit": "arc-sweeps/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": t,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"pagerank_rmat{a.scale}_ef{a.ef:g}", "n": g.n, "m": g.m, "sweeps": it,
                       "delta": 0.85, "step": "one bc_pagerank call (20 sweeps, beta = 0) incl. unpermute",
                       "l2": "CSR indices (0.5 GB) stream from HBM each sweep; contributions (34 MB) stay in L2"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "kernel": "k_pagerank", "model_bytes": model,
                         "model": "per sweep 12m + 36n bytes", "peak_source": peak_src},
            "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99)),
                           "what": "per bc_pagerank call"},
            "gpu_launches": 2 * a.steps, "clocks": clk}
    print(json.dumps(line), flush=True)


def run_weighted(a, bc, torch):
    """Weighted BC (bc_compute_weighted) on R-MAT with seeded integer weights 1..100
    (--directed: the R-MAT graph oriented, weights per arc)."""
    import bcgen
    g = bcgen.rmat(a.scale, a.ef, 1)
    if a.directed:
        g = bcgen.orient(g, seed=1)
    wt = bcgen.edge_weights(g, 1, 100, 1, per_arc=a.directed)
    src = bcgen.sample_sources(g, a.sources or 256, 1)
    t0 = time.perf_counter()
    G = bc.Graph(g.off, g.adj, weights=wt, directed=a.directed)
    torch.cuda.synchronize()
    ingest_s = time.perf_counter() - t0
    d_src = torch.from_numpy(src).cuda()
    out = torch.empty(g.n, dtype=torch.float64, device="cuda")
    for _ in range(max(a.warmup, 0)):
        G.compute_weighted(d_src, out=out)
    stream = torch.cuda.current_stream()
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    torch.cuda.synchronize()
    ms, kms, launches, statuses = [], [], 0, set()
    for _ in range(a.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, st = G.compute_weighted(d_src, out=out)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        s = G.stats()
        kms.append(s["kernel_ms"])
        launches += s["kernel_launches"]
        statuses.add(st)
    clk = clocks.stop()
    t = float(np.mean(ms))
    s = G.stats()
    # bytes the passes must move: an arc read with its neighbour's distances
    # brings its index and weight (8 B) and the neighbour's 32-column row
    # (256 B); an arc the path-count or dependency loop reads through its DAG
    # mask brings its index and mask (8 B) and 8 B per column it uses (one
    # count add or one rho);
    # every row a pass recomputes writes its 32 columns (256 B); summed over
    # the call's passes
    full = s["arcs_visited"] - s["mask_arcs"]
    model = 264.0 * full + 8.0 * s["mask_arcs"] + 8.0 * s["mask_lanes"] + 256.0 * s["rows_visited"]
    kt = float(np.mean(kms))
    peak, peak_src = measured_peak()
    achieved = model / (kt / 1e3) / 1e9
    h_src = torch.from_numpy(src).pin_memory()
    h_out = torch.empty(g.n, dtype=torch.float64).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    G.compute_weighted(h_src.numpy(), out=out)
    h_out.copy_(out, non_blocking=True)
    stream.synchronize()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    line = {"metric": "weighted BC traversed edges/s (sources x edges)", "value": len(src) * g.m / (t / 1e3),
            "unit": UNIT, "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": t,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"weighted_{'directed_' if a.directed else ''}rmat{a.scale}_ef{a.ef:g}", "n": g.n,
                       "m": g.m, "sources": len(src),
                       "graph": ("R-MAT oriented: each edge one way, a quarter of them both ways (seed 1)"
                                 if a.directed else "undirected R-MAT"),
                       "weights": ("integer 1..100 per arc (SplitMix64 of the arc, seed 1)" if a.directed else
                                   "integer 1..100 per undirected edge (SplitMix64 of the edge, seed 1)"),
                       "batches": s["batches"], "passes": {"dist": s["max_levels"], "sigma": s["pull_levels"],
                                                           "delta": s["push_levels"]},
                       "ingest_s": round(ingest_s, 3), "statuses": sorted(int(x) for x in statuses),
                       "source_grouping_ms": round(s["order_ms"], 3),
                       "step": "one bc_compute_weighted over all sources on the resident graph",
                       "l2": "per-batch state (n x 32 x 48 B) is far above L2"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "kernel": "k_wbc", "kernel_ms": kt, "model_bytes": model,
                         "model": "264 B per arc read with its neighbour's distance row, 8 B per arc read through a "
                                  "DAG mask + 8 B per column it uses, 256 B per row recomputed, over the passes the "
                                  f"call ran ({full:.3e} + {s['mask_arcs']:.3e} arcs, {s['mask_lanes']:.3e} mask "
                                  f"columns, {s['rows_visited']:.3e} rows)",
                         "peak_source": peak_src},
            "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99)),
                           "what": "per bc_compute_weighted call"},
            "e2e": {"value": len(src) * g.m / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(4 * len(src)),
                    "d2h_bytes_per_step": int(8 * g.n), "ms_per_step": e2e_ms},
            "gpu_launches": launches, "clocks": clk}
    if not a.no_cpu_baseline:
        import oracle
        sample = src[:2]
        t1 = time.perf_counter()
        oracle.wbc(g.off, g.adj, wt, sample)
        dt = time.perf_counter() - t1
        line["cpu_baseline"] = {"value": len(sample) * g.m / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{len(sample)} of the workload's sources, full graph, {dt:.1f} s on 1 thread"}
    print(json.dumps(line), flush=True)


def run_serve(a, bc, torch):
    """Serving: open-loop Poisson stream over a resident pool of R-MAT graphs."""
    import bcgen
    lo, hi = (int(x) for x in a.scales.split("-"))
    scales = list(range(lo, hi + 1))
    t0 = time.perf_counter()
    pool = [bcgen.rmat(s, 16, 1) for s in scales]
    Gs = [bc.Graph(g.off, g.adj) for g in pool]
    gen_s = time.perf_counter() - t0
    reqs = bcgen.poisson_requests(a.rate, a.duration, len(pool), seed=1)
    outs = [torch.empty(pool[gi].n, dtype=torch.float64, device="cuda") for _, gi, _ in reqs]
    srcs = [bcgen.sample_sources(pool[gi], k, 100 + i) for i, (_, gi, k) in enumerate(reqs)]
    bc.server_config(a.slots, 0)
    # warm-up: one request per graph (workspaces, tuning tables)
    for G, g in zip(Gs, pool):
        o = torch.empty(g.n, dtype=torch.float64, device="cuda")
        G.submit(bcgen.sample_sources(g, 4, 5), o).wait()
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    jobs = []
    t0 = time.perf_counter()
    for (t, gi, k), o, s in zip(reqs, outs, srcs):
        now = time.perf_counter() - t0
        if t > now:
            time.sleep(t - now)
        jobs.append(Gs[gi].submit(s, o))
    lat = [j.wait()[1] for j in jobs]
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    work = [len(s) * pool[gi].m for s, (_, gi, _) in zip(srcs, reqs)]
    arcs = sum(work)
    peak, done = bc.server_stats()
    lat_ms = np.array(lat) * 1e3
    big = np.array([pool[gi].m for _, gi, _ in reqs]) >= pool[-1].m
    line = {"metric": METRIC, "value": arcs / wall, "unit": UNIT, "n_gpus": 1, "steps": len(reqs), "warmup": len(pool),
            "ms_per_step": wall * 1e3 / max(len(reqs), 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"serve_poisson{a.rate:g}", "pool": [f"rmat{s}_ef16" for s in scales],
                       "requests": len(reqs), "k": "round(2^U[0,10]) sources, graph uniform over the pool",
                       "duration_s": a.duration, "slots": a.slots, "generation_s": round(gen_s, 1),
                       "offered_source_arcs_per_s": arcs / a.duration, "wall_s": round(wall, 2),
                       "step": "one request (submit to completion)"},
            "latency_ms": {"p50": float(np.percentile(lat_ms, 50)), "p99": float(np.percentile(lat_ms, 99)),
                           "p50_largest_graph": float(np.percentile(lat_ms[big], 50)) if big.any() else None,
                           "what": "submit to completion per request"},
            "peak_concurrency": peak, "clocks": clk}
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
