#!/usr/bin/env python
"""Benchmark of the push/pull sweep path on one R-MAT scale-22 graph.

One step runs the whole hot path once on the graph already resident in HBM:
  gp_graph_upload (validation + degree preparation + degree bins),
  gp_pagerank PULL, PUSH and AUTO, each to L1 tolerance 1e-7 (cap 300 sweeps),
  gp_bfs_multi AUTO (direction-switching) from 64 random non-isolated sources,
  all searches in one launch (groups of blocks searching concurrently).
Metric: traversed edges per second (GTEPS): m per PageRank sweep, and for BFS
the undirected edges of the reached component (Graph500 convention, the graph
being symmetric).  One JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (FP64, all host cores) on a bounded
sample of the same workload.  Under torchrun every rank runs the same per-GPU
workload (weak scaling, no data-path collective); timings are the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PR/BFS GTEPS push vs pull vs auto, batched vs serial, % HBM peak, 1 GB300"
WORKLOAD = ("R-MAT scale 22 (A/B/C/D .57/.19/.19/.05, edge factor 16, seed 1, symmetrised, no self-loops or "
            "duplicates): PageRank PULL+PUSH+AUTO to L1 tol 1e-7 (d=0.85, cap 300) and direction-switching BFS "
            "from 64 random non-isolated sources (seed 2)")


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--scale", type=int, default=22)
    p.add_argument("--sources", type=int, default=64)
    p.add_argument("--tol", type=float, default=1e-7)
    p.add_argument("--cap", type=int, default=300)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--quiet", action="store_true")
    p.add_argument("--no-batched", action="store_true")
    p.add_argument("--no-legs", action="store_true", help="skip the per-configuration push/pull legs")
    p.add_argument("--only", choices=["pr_pull", "pr_push", "bfs", "batched", "sssp", "tc", "pr_fe", "bc", "pr_shapes"],
                   default=None,
                   help="profiling case: run only this part (fixed --sweeps for PageRank), no contract line")
    p.add_argument("--sweeps", type=int, default=4)
    p.add_argument("--groups", "--bfs-groups", dest="groups", type=int, default=0,
                   help="groups of blocks of gp_bfs_multi (the step, the legs, --only bfs; 0: the library's choice)")
    p.add_argument("--batch-scale", type=int, default=None,
                   help="--only batched: one R-MAT graph of this scale instead of the 32-graph workload")
    p.add_argument("--delta", type=float, default=64.0, help="--only sssp: bucket width")
    p.add_argument("--mode", choices=["push", "pull", "auto"], default="auto",
                   help="--only sssp / --only bfs: direction mode")
    p.add_argument("--no-batch-tune", action="store_true", help="--only batched: keep the default batch options")
    p.add_argument("--opt", action="append", default=[], metavar="KEY=VALUE",
                   help="gp_options override for the profiling case (repeatable)")
    return p.parse_args(argv)


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ------------------------------------------------------------------ distributed plumbing

class Dist:
    """Rank bookkeeping; with WORLD_SIZE > 1 a process group used only for the
    timing barrier and the max-over-ranks reduction."""

    def __init__(self, backend=None):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist

            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group(backend=backend or "nccl")
            self.pg = dist

    def barrier(self):
        if self.pg:
            if self.pg.get_backend() == "nccl":
                import torch

                self.pg.barrier(device_ids=[torch.cuda.current_device()])
            else:
                self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch

        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, x: float) -> float:
        if not self.pg:
            return x
        import torch

        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def aggregate(per_rank_units: float, per_rank_ms: float, dist: Dist) -> tuple:
    """Whole-job throughput: units summed over ranks / slowest rank's time."""
    total_units = dist.sum(per_rank_units)
    ms = dist.max(per_rank_ms)
    return total_units / (ms * 1e-3) if ms > 0 else 0.0, ms


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples (every 50 ms) of SM clock and throttle reasons."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        loaded = [c for c in sm if c > 0.5 * (max(smax) if smax else 1)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ inputs

def make_graph(scale: int):
    import graphgen as gg

    t = time.time()
    g = gg.rmat(scale, 16, seed=1)
    log(f"[bench] R-MAT scale {scale}: n={g.n} m={g.m} ({time.time() - t:.1f}s)")
    return g


def pick_sources(g, count: int):
    import graphgen as gg

    return gg.pick_vertices(g, count, seed=2)


KERNEL_SOURCE = {"pull_big": "pagerank.cu", "pull_light": "pagerank.cu", "push_scatter": "pagerank.cu",
                 "push_epilogue": "pagerank.cu", "bfs_persistent": "bfs.cu", "bfs_multi": "bfs.cu"}


def source_key(cu_name: str) -> str:
    """First 16 hex digits of sha256 over the kernel's .cu file and the shared header."""
    import hashlib

    h = hashlib.sha256()
    for p in (os.path.join(ROOT, "paper_2010_16012_gb300", "csrc", cu_name),
              os.path.join(ROOT, "paper_2010_16012_gb300", "csrc", "gp_internal.cuh")):
        h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


def captured_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from profiles/traffic.md, or None when
    no capture exists or the kernel's source changed since it was taken."""
    cu = KERNEL_SOURCE.get(kernel)
    path = os.path.join(ROOT, "profiles", "traffic.md")
    if not cu or not os.path.exists(path):
        return None
    key = source_key(cu)
    for line in open(path):
        f = [x.strip() for x in line.strip().strip("|").split("|")]
        if len(f) >= 6 and f[0] == kernel and f[2] == key:
            try:
                return int(f[5])
            except ValueError:
                return None
    return None


def measured_peak_gbs():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(p))["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ algorithmic bytes per kernel launch

def kernel_bytes(g, opt, l2_bytes=None) -> dict:
    """Compulsory bytes of one (working) launch of each PageRank sweep kernel;
    random re-gathers that miss L2 are not counted.  The push accumulator is
    FP64 unless push_fp64_accum turns it off, or leaves the choice to the library
    (-1) and the library picks FP32: 8n bytes above half of `l2_bytes` and no
    vertex with more than 4096 in-edges."""
    n, m = g.n, g.m
    din, dout = g.in_degree(), g.out_degree()
    C = opt.chunk_edges
    big_in = din > opt.pull_light_max
    big_out = dout > opt.push_light_max
    e_big_in = int(din[big_in].sum())
    ch_in = int(((din[big_in] + C - 1) // C).sum())
    nb_in = int(big_in.sum())
    ch_out = int(((dout[big_out] + C - 1) // C).sum())
    mode = getattr(opt, "push_fp64_accum", -1)
    fp64 = mode == 1 or (mode == -1 and not (l2_bytes is not None and 8 * n > l2_bytes // 2
                                             and int(din.max(initial=0)) <= 4096))
    return {
        # big in-edge lists: indices + chunk table + chunk partials written
        "pull_big": 4 * e_big_in + 16 * ch_in + 4 * ch_in,
        # light in-edge lists + offsets + c (once) + x, inv_deg read + y, c' written + big-vertex combine
        "pull_light": 4 * (m - e_big_in) + 8 * (n + 1) + 4 * n * 5 + 4 * ch_in + 12 * nb_in,
        # all out-edge lists + offsets + c + y read-modify-write + chunk table
        "push_scatter": 4 * m + 8 * (n + 1) + 4 * n + 8 * n + 16 * ch_out,
        # FP64: the accumulator read and reset, x and inv_deg read, y and c' written;
        # FP32: y, x, inv_deg read, y, c' and the next accumulator (x) written
        "push_epilogue": (32 if fp64 else 24) * n,
    }


def bfs_level_bytes(n: int, direction: int, frontier: int, examined: int, candidates: int, new: int) -> tuple:
    """Compulsory bytes of one BFS level: (kernel name, bytes).  Top-down: queue
    entries, their offsets, the scanned out-edge indices, and for each newly
    visited vertex the level CAS, parent, its out- and in-degree offsets, the
    queue write and its frontier bit.  Bottom-up: the candidate bitmap, level
    and offsets of each candidate (unvisited vertex with in-edges), the scanned
    in-edge indices, level and parent of each new vertex and the new bitmap."""
    if direction == 0:
        return "bfs_topdown", 4 * frontier + 16 * frontier + 4 * examined + new * (4 + 4 + 32 + 4 + 4)
    return "bfs_bottomup", n // 8 + 20 * candidates + 4 * examined + new * 8 + n // 8


def sweep_bytes(g):
    """Compulsory bytes of one full pull sweep: 4m + 28n (+8)."""
    return 4 * g.m + 28 * g.n + 8


# ------------------------------------------------------------------ our arm

def run_ours(args, dist: Dist):
    import torch

    import paper_2010_16012_gb300 as gp

    torch.cuda.set_device(dist.local_rank)
    gp.load()
    g = make_graph(args.scale)
    srcs = pick_sources(g, args.sources)
    dev = torch.device("cuda", dist.local_rank)
    off = torch.from_numpy(g.csr_off).to(dev)
    idx = torch.from_numpy(g.csr_idx).to(dev)
    n, m = g.n, g.m
    ranks = [torch.empty(n, dtype=torch.float32, device=dev) for _ in range(3)]
    # one level and one parent vector per search (gp_bfs_multi writes all of them)
    lv_all = [torch.empty(n, dtype=torch.int32, device=dev) for _ in srcs]
    pa_all = [torch.empty(n, dtype=torch.int32, device=dev) for _ in srcs]
    modes = [(gp.PULL, "pull"), (gp.PUSH, "push"), (gp.AUTO, "auto")]

    # autotune once (outside the timed region; cached by graph statistics), then
    # every step's upload applies the tuned options
    G0 = gp.Graph(n, off, idx, symmetric=True)
    tuned = gp.autotune(G0, gp.TUNE_ALL, sources=srcs)
    tuned_opts = tuned["options"]
    opt_struct = G0.options()
    G0.free()
    kb = kernel_bytes(g, opt_struct, getattr(torch.cuda.get_device_properties(dev), "L2_cache_size", None))
    pr_kernels = {gp.PULL: ("pull_big", "pull_light"), gp.PUSH: ("push_scatter", "push_epilogue")}
    bfs_stats = {}
    n_in = int(np.count_nonzero(np.diff(g.csc_off)))  # vertices with in-edges (every reached vertex has one)

    def step(work=None):
        t0 = time.perf_counter()
        G = gp.Graph(n, off, idx, symmetric=True)
        G.set_options(**tuned_opts)
        t1 = time.perf_counter()
        edges = 0.0
        parts = {"upload_ms": (t1 - t0) * 1e3}
        for i, (mode, name) in enumerate(modes):
            ta = time.perf_counter()
            _, st = gp.pagerank(G, mode, 0.85, args.cap, args.tol, out=ranks[i])
            tb = time.perf_counter()
            k = st["iters_done"]
            edges += m * k
            parts[f"pr_{name}"] = {"sweeps": k, "ms": (tb - ta) * 1e3, "gteps": m * k / (tb - ta) / 1e9,
                                   "converged": st["converged"], "residual": st["residual"],
                                   "mode_used": "push" if st["mode_used"] == gp.PUSH else "pull"}
            if work is not None:
                for kn in pr_kernels[st["mode_used"]]:
                    w = work.setdefault(kn, [0.0, 0])
                    w[0] += kb[kn] * k
                    w[1] += k
        # The first pass (a warm-up step) runs each search on its own and keeps
        # its per-level statistics; the component sizes and level counts are
        # properties of the source (the direction decisions depend only on the
        # frontier counters), so later steps run all searches in one
        # gp_bfs_multi launch (groups of blocks searching concurrently).
        first = not bfs_stats
        ta = time.perf_counter()
        if first:
            for s in srcs:
                _, _, st = gp.bfs(G, int(s), gp.AUTO, level=lv_all[0], parent=pa_all[0])
                bfs_stats[int(s)] = st
        else:
            gp.bfs_multi(G, srcs, gp.AUTO, levels=lv_all, parents=pa_all, groups=args.groups, want_summary=False)
        torch.cuda.synchronize()
        bfs_ms = (time.perf_counter() - ta) * 1e3
        bfs_edges, switches = 0.0, 0
        for s in srcs:
            st = bfs_stats[int(s)]
            e = st["edges_reached"] / 2  # undirected edges of the component
            edges += e
            bfs_edges += e
            switches += st["switches"]
            if work is not None:  # one launch for all searches: the sum of their levels' bytes
                seen, by = 0, 0
                fr = st["frontier"] + [0]
                for L, d in enumerate(st["direction"]):
                    seen += fr[L]
                    by += bfs_level_bytes(n, d, fr[L], st["examined"][L], n_in - seen, fr[L + 1])[1]
                work.setdefault("bfs_multi", [0.0, 0])[0] += by
        if work is not None and not first:
            work["bfs_multi"][1] += 1
        parts["bfs_auto"] = {"sources": len(srcs), "ms": bfs_ms, "gteps_total": bfs_edges / bfs_ms / 1e6,
                             "switches_per_source": switches / max(len(srcs), 1),
                             "launch": "one gp_bfs_multi launch" if not first else "one gp_bfs launch per source"}
        G.free()
        return edges, parts

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(dist.local_rank)
    clocks.start()
    gp.profile_read(reset=True)
    gp.profile_enable(True)
    dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    tot_edges, parts, work = 0.0, None, {}
    for _ in range(args.steps):
        e, parts = step(work)
        tot_edges += e
    e1.record()
    torch.cuda.synchronize()
    dist.barrier()
    gp.profile_enable(False)
    kt = gp.profile_read(reset=True)
    clk = clocks.stop()
    ms_step = e0.elapsed_time(e1) / args.steps
    value_eps, ms_max = aggregate(tot_edges / args.steps, ms_step, dist)

    # roofline of the dominant kernel (largest total device time in the timed
    # region): compulsory bytes of its working launches / its total time
    # (which also contains its early-exit launches after convergence)
    peak, peak_kind = measured_peak_gbs()
    launches = int(sum(k[1] for k in kt))
    total_kernel_ms = sum(k[2] for k in kt)
    kernels = [{"name": k[0], "launches": k[1], "total_ms": round(k[2], 3),
                "share": round(k[2] / total_kernel_ms, 4) if total_kernel_ms else None} for k in kt]
    roofline = None
    if kt:
        top = kt[0]
        by, real = work.get(top[0], [0.0, 0])
        if real:
            ach = by / (top[2] * 1e-3) / 1e9
            roofline = {"kernel": top[0], "bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                        "frac": round(ach / peak, 4), "traffic": captured_traffic(top[0]), "peak_kind": peak_kind,
                        "bytes_per_launch": int(by / real), "avg_launch_ms": round(top[2] / real, 5),
                        "share": round(top[2] / total_kernel_ms, 4)}
    # the pull sweep as a whole (both pull kernels), the figure the 40%-of-HBM target is set on
    pull_sweep = None
    if "pull_light" in work and work["pull_light"][1]:
        tk = {k[0]: k for k in kt}
        sweeps = work["pull_light"][1]
        ms = (tk["pull_big"][2] + tk["pull_light"][2]) / sweeps
        ach = sweep_bytes(g) / (ms * 1e-3) / 1e9
        pull_sweep = {"sweeps": sweeps, "ms_per_sweep": round(ms, 5), "achieved": round(ach, 1), "peak": peak,
                      "unit": "GB/s", "frac": round(ach / peak, 4), "bytes_per_sweep": sweep_bytes(g),
                      "gteps": round(m / (ms * 1e-3) / 1e9, 2)}

    out = {"metric": METRIC, "value": round(value_eps / 1e9, 4), "unit": "GTEPS", "n_gpus": dist.world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n": n, "m": m, "sources": int(len(srcs)), "tuned_options": tuned_opts,
                      "l2": "inputs larger than L2 (CSR 0.55 GB > 129 MB); no flush between steps",
                      "parallelism": f"replicas{dist.world}"},
           "parts": parts, "roofline": roofline, "pull_sweep_roofline": pull_sweep,
           "gpu_launches": launches, "kernels": kernels[:14], "clocks": clk}
    if not args.no_e2e:
        out["e2e"] = run_e2e(args, g, srcs, dist, tuned_opts)
    if not args.no_legs:
        out["legs"] = run_legs(args, g, srcs, tuned_opts)
    if not args.no_batched:
        out["batched"] = run_batched(args)
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(g, srcs, args)
    return out


# ------------------------------------------------------------------ per-config legs (push against pull)

def pr_sweep_bytes(g, mode: int, weighted: bool = False) -> int:
    """Compulsory bytes of one PageRank sweep.  Pull: CSC indices, offsets, c
    read, y written, x read for the residual, inv_deg read, c' written = 4m +
    28n (+8).  Push: CSR indices, offsets, c read, y initialised, residual (x and
    y read) = 4m + 24n (+8); its m updates are L2 reductions, not HBM traffic.
    Weighted sweeps also read one float per edge."""
    base = 4 * g.m + (28 if mode == 1 else 24) * g.n + 8
    return base + (4 * g.m if weighted else 0)


def _events_ms(fn, repeats: int) -> list:
    """CUDA-event time of each of `repeats` calls of fn on the current stream."""
    import torch

    out = []
    for _ in range(repeats):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def pr_leg(gp, g, G, mode: int, sweeps: int, peak: float, repeats: int = 3, tol: float = 0.0, weighted=False):
    """PageRank in one direction: CUDA-event time of the call (host polls
    included) and the library's per-kernel device time, GTEPS (m per sweep) and
    the fraction of the measured HBM peak on the compulsory bytes."""
    import torch

    out = torch.empty(g.n, dtype=torch.float32, device="cuda")
    res = {}
    gp.pagerank(G, mode, 0.85, sweeps, tol, out=out)  # warm-up (workspace, hot sets)
    gp.profile_read(reset=True)
    gp.profile_enable(True)
    ms = _events_ms(lambda: res.update(gp.pagerank(G, mode, 0.85, sweeps, tol, out=out)[1]), repeats)
    gp.profile_enable(False)
    kt = gp.profile_read(reset=True)
    k = res["iters_done"]
    kms = sum(x[2] for x in kt) / repeats
    by = pr_sweep_bytes(g, mode, weighted) * k
    t = statistics.median(ms)
    return {"sweeps": k, "ms": round(t, 3), "gteps": round(g.m * k / t / 1e6, 2),
            "hbm_frac": round(by / (t * 1e-3) / 1e9 / peak, 4), "kernel_ms": round(kms, 3),
            "kernel_hbm_frac": round(by / (kms * 1e-3) / 1e9 / peak, 4) if kms else None,
            "bytes_per_sweep": pr_sweep_bytes(g, mode, weighted), "converged": bool(res["converged"])}


def bfs_leg(gp, g, G, srcs, mode: int, peak: float, undirected: bool, repeats: int = 3, groups=None):
    """Searches from every source in one direction mode: one gp_bfs launch per
    source enqueued back to back, or (groups not None) all of them in one
    gp_bfs_multi launch with that many groups (statistics from a first, untimed
    pass of single searches).  GTEPS: undirected edges of the reached component
    (Graph500) or, for a directed graph, out-edges of the reached vertices, over
    the time; also the adjacency entries examined per second and the fraction
    of the HBM peak on the per-level compulsory bytes."""
    import torch

    n = g.n
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    if groups is not None:
        lv_all = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in srcs]
        pa_all = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in srcs]
    n_in = int(np.count_nonzero(np.diff(g.csc_off)))
    edges = examined = by = 0.0
    levels = switches = 0
    for s in srcs:
        _, _, st = gp.bfs(G, int(s), mode, level=level, parent=parent)
        edges += st["edges_reached"] / (2 if undirected else 1)
        examined += st["edges_examined"]
        levels += st["levels"]
        switches += st["switches"]
        seen = 0
        fr = st["frontier"] + [0]
        for L, d in enumerate(st["direction"]):
            seen += fr[L]
            by += bfs_level_bytes(n, d, fr[L], st["examined"][L], n_in - seen, fr[L + 1])[1]

    def run():
        if groups is not None:
            gp.bfs_multi(G, srcs, mode, levels=lv_all, parents=pa_all, groups=groups, want_summary=False)
            return
        for s in srcs:
            gp.bfs(G, int(s), mode, level=level, parent=parent, want_stats=False)

    t = statistics.median(_events_ms(run, repeats))
    out = {"launch": "gp_bfs_multi" if groups is not None else "gp_bfs per source"}
    return {**out, "sources": len(srcs), "ms_per_search": round(t / len(srcs), 4), "gteps": round(edges / t / 1e6, 2),
            "examined_per_s_g": round(examined / t / 1e6, 2), "levels_per_search": round(levels / len(srcs), 2),
            "switches_per_search": round(switches / len(srcs), 2),
            "hbm_frac": round(by / (t * 1e-3) / 1e9 / peak, 4)}


def run_legs(args, g2, srcs2, tuned_opts):
    """The metric's push-against-pull comparison on every configuration that
    fits one GPU, outside the timed step (each leg timed on its own):
      C1  R-MAT scale 14 (seed 1): PageRank push and pull, exactly 20 sweeps
          from 1/n; BFS from vertex 0 top-down, bottom-up and switching;
      C2  R-MAT scale 22: BFS from the 64 step sources forced top-down,
          forced bottom-up and switching, one launch per search and all
          searches in one gp_bfs_multi launch;
      C3  directed Erdos-Renyi G(2^24, 16*2^24 draws) (seed 3): PageRank pull
          and push, 20 sweeps; BFS top-down, bottom-up and switching from 16
          sources with out-degree > 0 (seed 4), per source and in one launch;
      C5  weighted R-MAT scale 20 (seed 8, weights U(0,1] seed 9, normalised
          per source): forward PageRank to L1 tol 1e-10 (cap 300) and the
          adjoint for L = g.x, g ~ N(0,1) (seed 10), to the same tolerance."""
    import torch

    import graphgen as gg
    import paper_2010_16012_gb300 as gp

    peak, _ = measured_peak_gbs()
    legs = {}
    # C2: forced directions from the step's sources
    G = gp.Graph.from_graphgen(g2)
    G.set_options(**tuned_opts)
    legs["c2_bfs"] = {name: bfs_leg(gp, g2, G, srcs2, mode, peak, True, repeats=2)
                      for name, mode in (("top_down", gp.PUSH), ("bottom_up", gp.PULL), ("auto", gp.AUTO))}
    legs["c2_bfs"].update({name + "_multi": bfs_leg(gp, g2, G, srcs2, mode, peak, True, repeats=2,
                                                     groups=args.groups)
                           for name, mode in (("top_down", gp.PUSH), ("bottom_up", gp.PULL), ("auto", gp.AUTO))})
    G.free()
    # C1
    t = time.time()
    g1 = gg.rmat(14, 16, seed=1)
    G = gp.Graph.from_graphgen(g1)
    gp.autotune(G, gp.TUNE_ALL, sources=np.array([0], dtype=np.int32))
    c1 = {"n": g1.n, "m": g1.m}
    for name, mode in (("pr_pull", gp.PULL), ("pr_push", gp.PUSH)):
        c1[name] = pr_leg(gp, g1, G, mode, 20, peak, repeats=5)
    src0 = np.array([0] * 20, dtype=np.int32)  # 20 searches from vertex 0, back to back
    c1["bfs_v0"] = {name: bfs_leg(gp, g1, G, src0, mode, peak, True)
                    for name, mode in (("top_down", gp.PUSH), ("bottom_up", gp.PULL), ("auto", gp.AUTO))}
    G.free()
    legs["c1_rmat14"] = c1
    log(f"[bench] leg C1 done ({time.time() - t:.1f}s)")
    # C3
    t = time.time()
    g3 = gg.erdos_renyi(1 << 24, 16 << 24, seed=3)
    G = gp.Graph.from_graphgen(g3)
    s3 = gg.pick_vertices(g3, 16, seed=4)
    t3 = gp.autotune(G, gp.TUNE_ALL, sources=s3[:4])
    c3 = {"n": g3.n, "m": g3.m, "gen_s": round(time.time() - t, 1), "tuned_options": t3["options"]}
    for name, mode in (("pr_pull", gp.PULL), ("pr_push", gp.PUSH)):
        c3[name] = pr_leg(gp, g3, G, mode, 20, peak)
    c3["bfs"] = {name: bfs_leg(gp, g3, G, s3, mode, peak, False, repeats=2)
                 for name, mode in (("top_down", gp.PUSH), ("bottom_up", gp.PULL), ("auto", gp.AUTO))}
    c3["bfs"]["auto_multi"] = bfs_leg(gp, g3, G, s3, gp.AUTO, peak, False, repeats=2, groups=args.groups)
    G.free()
    del g3
    legs["c3_er24"] = c3
    log(f"[bench] leg C3 done ({time.time() - t:.1f}s)")
    # C5
    t = time.time()
    g5 = gg.rmat(20, 16, seed=8).with_weights(9)
    G = gp.Graph.from_graphgen(g5)
    gvec = torch.from_numpy(np.random.default_rng(10).normal(size=g5.n).astype(np.float32)).cuda()
    fwd = pr_leg(gp, g5, G, gp.PULL, 300, peak, tol=1e-10, weighted=True)
    x, _ = gp.pagerank(G, gp.PULL, 0.85, 300, 1e-10)
    res = {}
    gp.pagerank_backward(G, x, gvec, iters=300, tol=1e-10)
    ms = statistics.median(_events_ms(lambda: res.update(gp.pagerank_backward(G, x, gvec, iters=300,
                                                                                tol=1e-10)[2]), 3))
    k = res["iters_done"]
    # per adjoint iteration one weighted transposed sweep; then dL/dP over every
    # edge (indices read, gradient written) and dL/ds
    by = pr_sweep_bytes(g5, gp.PULL, True) * k + 8 * g5.m + 8 * (g5.n + 1) + 12 * g5.n
    legs["c5_adjoint_rmat20"] = {
        "n": g5.n, "m": g5.m, "forward": fwd,
        "backward": {"iters": k, "converged": bool(res["converged"]), "ms": round(ms, 3),
                     "gteps": round(g5.m * k / ms / 1e6, 2), "hbm_frac": round(by / (ms * 1e-3) / 1e9 / peak, 4)}}
    G.free()
    log(f"[bench] leg C5 done ({time.time() - t:.1f}s)")
    return legs


def run_e2e(args, g, srcs, dist: Dist, tuned_opts=None):
    """Same step through the C ABI from host memory: the CSR arrays are copied
    from pinned host memory by gp_graph_upload (GP_UPLOAD_COPY) and every result
    (three rank vectors, 64 level + parent vectors) is read back into its own
    pinned host buffer, all inside the timed region.  The searches run first, in
    one gp_bfs_multi launch; their results (2.15 GB) are copied out on a second
    stream while the three PageRank runs compute (PageRank polls its status
    through mapped memory, so it never waits behind those copies), and the rank
    vectors follow on the same stream.  Uploads are pipelined: a worker thread
    uploads the next step's graph on a third stream while this step computes
    (the first step's upload is not overlapped; every step's upload is inside
    the timed region).  The edge count of a search is a property of its
    source: taken from one untimed step."""
    import concurrent.futures

    import torch

    import paper_2010_16012_gb300 as gp

    n, m = g.n, g.m
    pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
    off_h, idx_h = pin(g.csr_off), pin(g.csr_idx)
    ranks_h = [torch.empty(n, dtype=torch.float32).pin_memory() for _ in range(3)]
    ranks_d = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
    lv_h = [torch.empty(n, dtype=torch.int32).pin_memory() for _ in srcs]
    pa_h = [torch.empty(n, dtype=torch.int32).pin_memory() for _ in srcs]
    lv_d = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in srcs]
    pa_d = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in srcs]
    main = torch.cuda.current_stream()
    copy = torch.cuda.Stream()
    up = torch.cuda.Stream()
    worker = concurrent.futures.ThreadPoolExecutor(max_workers=1)
    h2d = off_h.nbytes + idx_h.nbytes
    d2h = 3 * 4 * n + len(srcs) * 8 * n
    bfs_edges = {}

    def upload():
        torch.cuda.set_device(dist.local_rank)  # the worker thread's device
        G = gp.Graph(n, off_h, idx_h, symmetric=True, copy=True, stream=up)
        if tuned_opts:
            G.set_options(stream=up, **tuned_opts)
        ready = torch.cuda.Event()
        ready.record(up)
        return G, ready

    def step(pending, prefetch):
        G, ready = pending.result()
        main.wait_event(ready)
        nxt = worker.submit(upload) if prefetch else None  # the next step's graph, beside this step
        edges = 0.0
        first = not bfs_edges  # untimed first step: the sources' component sizes
        _, _, summ = gp.bfs_multi(G, srcs, gp.AUTO, levels=lv_d, parents=pa_d, groups=args.groups,
                                  want_summary=first)
        if first:
            for s, st in zip(srcs, summ):
                bfs_edges[int(s)] = st["edges_reached"] / 2
        done = torch.cuda.Event()
        done.record(main)
        copy.wait_event(done)
        with torch.cuda.stream(copy):
            for i in range(len(srcs)):
                lv_h[i].copy_(lv_d[i], non_blocking=True)
                pa_h[i].copy_(pa_d[i], non_blocking=True)
        edges += sum(bfs_edges[int(s)] for s in srcs)
        for i, mode in enumerate((gp.PULL, gp.PUSH, gp.AUTO)):
            _, st = gp.pagerank(G, mode, 0.85, args.cap, args.tol, out=ranks_d[i])
            edges += m * st["iters_done"]
        done = torch.cuda.Event()
        done.record(main)
        copy.wait_event(done)
        with torch.cuda.stream(copy):
            for i in range(3):
                ranks_h[i].copy_(ranks_d[i], non_blocking=True)
        copy.synchronize()
        G.free()
        return edges, nxt

    step(worker.submit(upload), False)
    torch.cuda.synchronize()
    steps = args.steps
    dist.barrier()
    t0 = time.perf_counter()
    tot = 0.0
    step_ms = []
    pending = worker.submit(upload)
    for k in range(steps):
        ts = time.perf_counter()
        e, pending = step(pending, k + 1 < steps)
        tot += e
        step_ms.append((time.perf_counter() - ts) * 1e3)
    torch.cuda.synchronize()
    dist.barrier()
    ms = (time.perf_counter() - t0) * 1e3 / steps
    worker.shutdown()
    v, _ = aggregate(tot / steps, ms, dist)
    # the results read back are the searches' own: spot-check the last step's first and last
    for i in (0, len(srcs) - 1):
        lv = lv_h[i].numpy()
        assert lv[int(srcs[i])] == 0 and (lv >= -1).all()
    assert all(bool((r >= 0).all()) and float(r.max()) > 0 for r in ranks_h)
    return {"value": round(v / 1e9, 4), "unit": "GTEPS", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "steps": steps, "ms_per_step": round(ms, 3),
            "median_step_ms": round(statistics.median(step_ms), 3), "max_step_ms": round(max(step_ms), 3),
            "overlap": "next step's upload on a worker thread and stream; searches in one launch first, their results "
                       "copied out on a second stream during PageRank"}


# ------------------------------------------------------------------ CPU oracle (baseline and reference arm)

def oracle_sample(g, srcs, O, sweeps: int, nsrc: int, threads: int):
    """One bounded sample of the workload on the CPU oracle: `sweeps` pull
    PageRank sweeps, one push sweep, and FIFO BFS from `nsrc` sources."""
    import oracle

    t = time.perf_counter()
    O.pagerank(oracle.PULL, 0.85, iters=sweeps, nthreads=threads)
    O.pagerank(oracle.PUSH, 0.85, iters=1)
    edges = g.m * (sweeps + 1)
    for s in srcs[:nsrc]:
        lv, _ = O.bfs(int(s))
        edges += float(g.out_degree()[lv >= 0].sum()) / 2
    return edges, time.perf_counter() - t


def cpu_baseline(g, srcs, args):
    """The oracle on the host cores, on a bounded sample of the step's workload
    (the headline figure, GTEPS over the whole sample), with per-operation
    figures: the pull sweep on all cores and on one thread, the push sweep and
    the FIFO BFS on one thread (the oracle's push and BFS are sequential), on
    the step's graph and on R-MAT scale 14."""
    import graphgen as gg
    import oracle

    threads = oracle.max_threads()
    O = oracle.OracleGraph.from_graph(g)
    sweeps, nsrc = 8, 2
    edges, sec = oracle_sample(g, srcs, O, sweeps, nsrc, threads)
    per_op = {}
    for gname, gg_, O_, s_ in (("rmat22", g, O, srcs[:2]), ("rmat14", None, None, None)):
        if gg_ is None:
            gg_ = gg.rmat(14, 16, seed=1)
            O_ = oracle.OracleGraph.from_graph(gg_)
            s_ = np.array([0], dtype=np.int32)
        reps = 1 if gname == "rmat22" else 20
        for key, var, th, k in (("pull_sweep_all_cores", oracle.PULL, threads, 4),
                                ("pull_sweep_1_thread", oracle.PULL, 1, 1), ("push_sweep_1_thread", oracle.PUSH, 1, 1)):
            t = time.perf_counter()
            for _ in range(reps):
                O_.pagerank(var, 0.85, iters=k, nthreads=th)
            per_op[f"{gname}_{key}_gteps"] = round(gg_.m * k * reps / (time.perf_counter() - t) / 1e9, 5)
        t = time.perf_counter()
        be = 0.0
        for _ in range(reps):
            for src in s_:
                lv, _ = O_.bfs(int(src))
                be += float(gg_.out_degree()[lv >= 0].sum()) / 2
        per_op[f"{gname}_bfs_fifo_1_thread_gteps"] = round(be / (time.perf_counter() - t) / 1e9, 5)
    return {"value": round(edges / sec / 1e9, 5), "unit": "GTEPS", "cores": threads, "kind": "oracle",
            "sample": f"{sweeps} pull PageRank sweeps ({threads} threads) + 1 push sweep (1 thread) + FIFO BFS "
                      f"from {nsrc} of the sources, on the full scale-{args.scale} graph; {sec:.1f} s",
            "per_op": per_op}


def run_reference(args, dist: Dist):
    import oracle

    if dist.rank != 0:
        return None
    g = make_graph(args.scale)
    srcs = pick_sources(g, args.sources)
    threads = oracle.max_threads()
    O = oracle.OracleGraph.from_graph(g)
    sweeps, nsrc = 3, 1
    for _ in range(args.warmup):
        oracle_sample(g, srcs, O, 1, 0, threads)
    tot, sec = 0.0, 0.0
    for _ in range(args.steps):
        e, s = oracle_sample(g, srcs, O, sweeps, nsrc, threads)
        tot += e
        sec += s
    v = tot / sec / 1e9
    sample = (f"per step {sweeps} pull PageRank sweeps ({threads} threads) + 1 push sweep + FIFO BFS from "
              f"{nsrc} source on the full scale-{args.scale} graph")
    return {"impl": "reference", "metric": METRIC, "value": round(v, 5), "unit": "GTEPS", "n_gpus": dist.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(sec / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": g.n, "m": g.m, "parallelism": "cpu oracle"},
            "cpu_baseline": {"value": round(v, 5), "unit": "GTEPS", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(v, 5), "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def batched_workload(nscale_lo=12, nscale_hi=18, ngraphs=32):
    """32 R-MAT graphs, scales uniform in [12, 18] (seed 5), graph i with seed 100 + i."""
    import graphgen as gg

    scales = [nscale_lo + int(gg.draw(5, i) % (nscale_hi - nscale_lo + 1)) for i in range(ngraphs)]
    return [gg.rmat(s, 16, seed=100 + i) for i, s in enumerate(scales)], scales


def run_batched(args, graphs_scales=None):
    """Batched personalised PageRank (256 one-hot vectors per graph, tol 1e-6) and
    64-source BFS over 32 graphs in one persistent launch each, against
    one-at-a-time gp_pagerank / gp_bfs calls on the same stream, each vector
    started at its seed's one-hot vector on both sides (timed on a
    sample of vectors and sources per graph, scaled to all of them; CUDA-graph
    capture is excluded from the batched side, launch overheads are included on
    both sides)."""
    import torch

    import graphgen as gg
    import paper_2010_16012_gb300 as gp

    K, NSRC, SAMPLE, REPS = 256, 64, 16, 3
    graphs, scales = graphs_scales or batched_workload()
    G = [gp.Graph.from_graphgen(g) for g in graphs]
    B = gp.Batch(G, k_ppr=K)
    seeds = np.stack([np.resize(gg.pick_vertices(g, K, seed=6 + 1000 * i), K) for i, g in enumerate(graphs)])
    srcs = np.stack([np.resize(gg.pick_vertices(g, NSRC, seed=7 + 1000 * i), NSRC) for i, g in enumerate(graphs)])
    tuned = {"trials": 0} if getattr(args, "no_batch_tune", False) else B.autotune(seeds, srcs)  # outside the timed region
    B.ppr(seeds, iters=1000, tol=1e-6)  # captures the CUDA graph
    B.msbfs(srcs)
    torch.cuda.synchronize()
    tp, tb, tk = [], [], []
    for _ in range(REPS):
        t = time.perf_counter()
        outs, done, st = B.ppr(seeds, iters=1000, tol=1e-6)
        tp.append(time.perf_counter() - t)
        tk.append(st["ms"])
        t = time.perf_counter()
        louts, bst = B.msbfs(srcs)
        tb.append(time.perf_counter() - t)
    ppr_batched_s, bfs_batched_s = statistics.median(tp), statistics.median(tb)
    # one at a time, on a sample
    e = [torch.zeros(g.n, device="cuda") for g in graphs]
    x = [torch.empty(g.n, device="cuda") for g in graphs]
    lv = [torch.empty(g.n, dtype=torch.int32, device="cuda") for g in graphs]
    for i in range(len(graphs)):  # warm-up of the per-graph workspaces
        gp.pagerank(G[i], gp.PULL, 0.85, 5, 0.0, out=x[i])
        gp.bfs(G[i], int(srcs[i, 0]), gp.AUTO, level=lv[i], want_parent=False)
    torch.cuda.synchronize()
    ev = [[torch.zeros(g.n, device="cuda") for _ in range(SAMPLE)] for g in graphs]
    xs = [[torch.empty(g.n, device="cuda") for _ in range(SAMPLE)] for g in graphs]
    for i in range(len(graphs)):
        for j in range(SAMPLE):
            ev[i][j][int(seeds[i, j])] = 1.0
    ts, tsb = [], []
    for _ in range(REPS):
        torch.cuda.synchronize()
        t = time.perf_counter()
        for i in range(len(graphs)):
            for j in range(SAMPLE):
                gp.pagerank(G[i], gp.PULL, 0.85, 1000, 1e-6, personalization=ev[i][j], x0=ev[i][j], out=xs[i][j])
        torch.cuda.synchronize()
        ts.append((time.perf_counter() - t) * K / SAMPLE)
        t = time.perf_counter()
        for i in range(len(graphs)):
            for j in range(SAMPLE):
                gp.bfs(G[i], int(srcs[i, j]), gp.AUTO, level=lv[i], want_parent=False)
        torch.cuda.synchronize()
        tsb.append((time.perf_counter() - t) * NSRC / SAMPLE)
    ppr_serial_s, bfs_serial_s = statistics.median(ts), statistics.median(tsb)
    max_err = max(float((xs[i][j] - outs[i][:, j]).abs().max()) for i in range(len(graphs)) for j in range(SAMPLE))
    nvec = len(graphs) * K
    edges = sum(g.m * int(done[i].sum()) for i, g in enumerate(graphs))
    # roofline: compulsory bytes, whatever the slicing and packing: a graph's
    # index stream and offsets (4m + 8n) once per sweep of its slowest column,
    # and each column's iterate read once, written once and read for the
    # residual (12 n) per sweep of its own.  Row gathers (4m bytes per column
    # sweep) come from L2 by design and are reported as a rate beside it.
    bo = B.options()
    comp_bytes = gath_bytes = 0.0
    for i, g in enumerate(graphs):
        col_sweeps = float(done[i].sum())
        comp_bytes += int(done[i].max()) * (4 * g.m + 8 * (g.n + 1)) + 12 * g.n * col_sweeps
        gath_bytes += 4.0 * g.m * col_sweeps
    peak, peak_kind = measured_peak_gbs()
    kms = statistics.median(tk) if tk else None
    B.free()
    return {"graphs": len(graphs), "scales": scales, "n_total": int(sum(g.n for g in graphs)),
            "m_total": int(sum(g.m for g in graphs)), "ppr_vectors": nvec,
            "ppr_batched_ms": round(ppr_batched_s * 1e3, 2), "ppr_batched_sweeps": st["sweeps"],
            "ppr_serial_ms_extrapolated": round(ppr_serial_s * 1e3, 1),
            "ppr_speedup": round(ppr_serial_s / ppr_batched_s, 2),
            "ppr_batched_gteps": round(edges / ppr_batched_s / 1e9, 2),
            "ppr_max_abs_diff_vs_serial": max_err,
            "bfs_sources": len(graphs) * NSRC, "bfs_batched_ms": round(bfs_batched_s * 1e3, 2),
            "bfs_serial_ms_extrapolated": round(bfs_serial_s * 1e3, 1),
            "bfs_speedup": round(bfs_serial_s / bfs_batched_s, 2), "bfs_levels": bst["levels"],
            "serial_sample_per_graph": SAMPLE, "repeats": REPS, "options": bo, "tune_trials": tuned["trials"],
            "ppr_jobs": st["jobs"],
            "ppr_roofline": {"bound": "hbm", "kernel_ms": round(kms, 2), "compulsory_bytes": int(comp_bytes),
                             "achieved": round(comp_bytes / (kms * 1e-3) / 1e9, 1), "peak": peak, "unit": "GB/s",
                             "frac": round(comp_bytes / (kms * 1e-3) / 1e9 / peak, 4), "peak_kind": peak_kind,
                             "l2_gather_gbs": round(gath_bytes / (kms * 1e-3) / 1e9, 1)},
            "ppr_sweeps_per_vector": {"median": float(np.median(done)), "p90": float(np.percentile(done, 90)),
                                      "max": int(done.max()),
                                      "graph_max_median": float(np.median(done.max(axis=1)))},
            "ppr_batched_ms_all": [round(x * 1e3, 2) for x in tp],
            "ppr_serial_ms_all": [round(x * 1e3, 1) for x in ts]}


def run_only(args):
    """A reduced run for profilers: one part of the step on the same kind of
    graph, --warmup + --steps repetitions, then a short JSON summary."""
    import torch

    import paper_2010_16012_gb300 as gp

    gp.load()
    if args.only == "pr_shapes":
        return run_only_pr_shapes(args)
    if args.only == "batched":
        import graphgen as gg

        gs = None
        if args.batch_scale:
            gs = ([gg.rmat(args.batch_scale, 16, seed=100)], [args.batch_scale])
        print(json.dumps({"profile_case": "batched", **run_batched(args, gs)}), flush=True)
        return 0
    if args.only == "sssp":
        return run_only_sssp(args)
    if args.only == "tc":
        return run_only_tc(args)
    if args.only == "bc":
        return run_only_bc(args)
    if args.only == "pr_fe":
        return run_only_fe(args)
    g = make_graph(args.scale)
    off = torch.from_numpy(g.csr_off).cuda()
    idx = torch.from_numpy(g.csr_idx).cuda()
    G = gp.Graph(g.n, off, idx, symmetric=True)
    opts = {}
    for kv in args.opt:
        k, v = kv.split("=")
        opts[k] = float(v) if k.endswith("_alpha") or k.endswith("_beta") else int(v)
    if opts:
        G.set_options(**opts)
    out = torch.empty(g.n, dtype=torch.float32, device="cuda")
    srcs = pick_sources(g, args.sources)
    res = {}
    for i in range(args.warmup + args.steps):
        if i == args.warmup:
            torch.cuda.synchronize()
            gp.profile_read(reset=True)
            gp.profile_enable(True)
        if args.only == "bfs" and args.groups > 0:
            # all sources in one gp_bfs_multi launch with --groups groups
            bmode = {"push": gp.PUSH, "pull": gp.PULL, "auto": gp.AUTO}[args.mode]
            _, _, summ = gp.bfs_multi(G, srcs, bmode, groups=args.groups)
            res = {"searches": len(summ), "levels": [x["levels"] for x in summ],
                   "reached": [x["reached"] for x in summ]}
        elif args.only == "bfs":
            bmode = {"push": gp.PUSH, "pull": gp.PULL, "auto": gp.AUTO}[args.mode]
            for s in srcs:
                _, _, st = gp.bfs(G, int(s), bmode)
            # the last search's levels: direction, frontier, edges examined, device time
            res = {"levels": st["levels"], "reached": st["reached"], "init_us": round(st["init_us"], 1),
                   "level_table": [[d, f, e, round(t, 1)] for d, f, e, t in
                                   zip(st["direction"], st["frontier"], st["examined"], st["level_us"])]}
        else:
            mode = gp.PULL if args.only == "pr_pull" else gp.PUSH
            _, st = gp.pagerank(G, mode, 0.85, args.sweeps, 0.0, out=out)
            res = {"sweeps": st["iters_done"], "push_updates_l2": st["push_updates_l2"],
                   "push_updates_shared": st["push_updates_shared"], "push_updates_merged": st["push_updates_merged"],
                   "push_flush_l2": st["push_flush_l2"], "m": g.m}
    torch.cuda.synchronize()
    gp.profile_enable(False)
    kt = gp.profile_read(reset=True)
    G.free()
    per = {k[0]: round(k[2] / max(k[1], 1), 4) for k in kt}
    print(json.dumps({"profile_case": args.only, "scale": args.scale, "n": g.n, "m": g.m, "opts": opts,
                      "avg_launch_ms": per, **res}), flush=True)
    return 0


def run_only_sssp(args):
    """Delta-Stepping SSSP on the R-MAT graph with integer weights uniform in
    [1, 255] (seed 3), from --sources sources (seed 2): traversed edges per
    second, Graph500 convention (undirected edges of the reached component)."""
    import torch

    import graphgen as gg
    import paper_2010_16012_gb300 as gp

    g = gg.with_int_weights(make_graph(args.scale), seed=3, lo=1, hi=255)
    G = gp.Graph.from_graphgen(g)
    opts = {}
    for kv in args.opt:
        k, v = kv.split("=")
        opts[k] = float(v) if k.endswith("_alpha") or k.endswith("_beta") else int(v)
    if opts:
        G.set_options(**opts)
    srcs = pick_sources(g, args.sources)
    mode = {"push": gp.PUSH, "pull": gp.PULL, "auto": gp.AUTO}[args.mode]
    dist = torch.empty(g.n, dtype=torch.float32, device="cuda")
    deg = np.diff(g.csr_off)
    edges, stats = [], []
    for s in srcs:  # component sizes and iteration counts, outside the timed runs
        d, _, st = gp.sssp(G, int(s), args.delta, mode, dist=dist, want_pred=False)
        edges.append(float(deg[np.isfinite(d.cpu().numpy())].sum()) / 2)
        stats.append(st)
    for i in range(args.warmup + args.steps):
        if i == args.warmup:
            torch.cuda.synchronize()
            gp.profile_read(reset=True)
            gp.profile_enable(True)
        for s in srcs:
            gp.sssp(G, int(s), args.delta, mode, dist=dist, want_pred=False, want_stats=False)
    torch.cuda.synchronize()
    gp.profile_enable(False)
    kt = {k[0]: k for k in gp.profile_read(reset=True)}
    k = kt["sssp_persistent"]
    ms = k[2] / k[1]
    # compulsory bytes of a search: every examined edge's index and weight (8 B)
    # and one 8-byte key read per relaxation, over the event-timed search
    ex = float(np.mean([s["edges_examined"] for s in stats]))
    peak, peak_kind = measured_peak_gbs()
    ach = 16.0 * ex / (ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4),
            "peak_kind": peak_kind, "bytes_per_search": int(16 * ex)}
    cpu = None
    if not args.no_cpu_baseline:  # the oracle's Dijkstra on the host cores, one source
        import oracle

        O = oracle.OracleGraph.from_graph(g)
        t0 = time.perf_counter()
        O.sssp(int(srcs[0]))
        dt = time.perf_counter() - t0
        cpu = {"kind": "oracle", "what": "Dijkstra (binary heap, FP64), 1 thread, first source",
               "ms": round(dt * 1e3, 1), "cores": 1, "gteps": round(edges[0] / dt / 1e9, 4)}
    print(json.dumps({"profile_case": "sssp", "scale": args.scale, "n": g.n, "m": g.m, "weights": "int [1, 255]",
                      "delta": args.delta, "mode": args.mode, "opts": opts, "sources": len(srcs),
                      "avg_launch_ms": round(ms, 4), "gteps": round(sum(edges) / (ms * 1e-3 * len(srcs)) / 1e9, 2),
                      "roofline": roof, "cpu_oracle": cpu,
                      "iterations": round(float(np.mean([s["iterations"] for s in stats])), 1),
                      "epochs": round(float(np.mean([s["epochs"] for s in stats])), 1),
                      "pulls": round(float(np.mean([s["pulls"] for s in stats])), 1),
                      "edges_examined": round(float(np.mean([s["edges_examined"] for s in stats]))),
                      # the last source: per iteration direction, bucket, active vertices, edges, device time
                      "init_us": round(stats[-1]["init_us"], 1),
                      "iter_table": [[d, b, a, e, round(t, 1)] for d, b, a, e, t in
                                     zip(stats[-1]["direction"], stats[-1]["bucket"], stats[-1]["active"],
                                         stats[-1]["examined"], stats[-1]["iter_us"])]}), flush=True)
    return 0


def run_only_fe(args):
    """Frontier-Exploit PageRank on the R-MAT graph of --scale for a range of
    frontier thresholds and each mode: ms per run, iterations, push/pull split,
    the a-posteriori L1 error bound; beside it the Jacobi pull PageRank to L1
    tol 1e-7 on the same graph."""
    import torch

    import paper_2010_16012_gb300 as gp

    g = make_graph(args.scale)
    off = torch.from_numpy(g.csr_off).cuda()
    idx = torch.from_numpy(g.csr_idx).cuda()
    G = gp.Graph(g.n, off, idx, symmetric=True)
    x = torch.empty(g.n, dtype=torch.float32, device="cuda")
    rows = []
    for eps in (1e-9, 1e-10, 1e-11, 1e-12):
        for name, mode in (("auto", gp.AUTO), ("pull", gp.PULL), ("push", gp.PUSH)):
            for _ in range(args.warmup):
                gp.pagerank_fe(G, mode, 0.85, eps=eps, iters=1000, out=x)
            ms = []
            for _ in range(args.steps):
                _, st = gp.pagerank_fe(G, mode, 0.85, eps=eps, iters=1000, out=x)
                ms.append(st["ms"])
            rows.append({"eps": eps, "mode": name, "ms": round(statistics.median(ms), 3),
                         "iterations": st["iterations"], "pushes": st["pushes"], "pulls": st["pulls"],
                         "edges_examined": int(sum(st["examined"])), "error_bound_l1": st["error_bound"]})
    for _ in range(args.warmup):
        gp.pagerank(G, gp.PULL, 0.85, 300, 1e-7, out=x)
    ms = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _, st = gp.pagerank(G, gp.PULL, 0.85, 300, 1e-7, out=x)
        torch.cuda.synchronize()
        ms.append((time.perf_counter() - t0) * 1e3)
    jac = {"ms": round(statistics.median(ms), 3), "sweeps": st["iters_done"], "residual_l1": st["residual"],
           "error_bound_l1": st["residual"] * 0.85 / 0.15}
    print(json.dumps({"profile_case": "pr_fe", "scale": args.scale, "n": g.n, "m": g.m, "runs": rows,
                      "jacobi_pull_tol_1e-7": jac}), flush=True)
    return 0


def run_only_tc(args):
    """Triangle counting (NodeIterator, push and pull) on the R-MAT graph of
    --scale: per-vertex counts, ms per run, edges per second; the oracle's
    threaded pull form timed beside it (unless --no-cpu-baseline)."""
    import torch

    import paper_2010_16012_gb300 as gp

    g = make_graph(args.scale)
    G = gp.Graph.from_graphgen(g)
    opts = {}
    for kv in args.opt:
        k, v = kv.split("=")
        opts[k] = float(v) if k.endswith("_alpha") or k.endswith("_beta") else int(v)
    if opts:
        G.set_options(**opts)
    out = {}
    counts = {}
    for name, mode in (("pull", gp.PULL), ("push", gp.PUSH)):
        tc = torch.empty(g.n, dtype=torch.int64, device="cuda")
        for _ in range(args.warmup):
            gp.triangles(G, mode, out=tc)
        torch.cuda.synchronize()
        ms = []
        for _ in range(args.steps):
            _, total, st = gp.triangles(G, mode, out=tc)
            ms.append(st["ms"])
        counts[name] = tc.cpu().numpy()
        t = statistics.median(ms)
        out[name] = {"ms": round(t, 3), "triangles": total, "probes": st["probes"],
                     "gteps": round(g.m / (t * 1e-3) / 1e9, 3)}
    out["push_equals_pull"] = bool(np.array_equal(counts["push"], counts["pull"]))
    if not args.no_cpu_baseline:
        import oracle

        O = oracle.OracleGraph.from_graph(g)
        t0 = time.perf_counter()
        ref, rtot = O.triangles(oracle.PULL, nthreads=oracle.max_threads())
        dt = time.perf_counter() - t0
        out["cpu_oracle"] = {"kind": "oracle", "what": "NodeIterator pull, OpenMP", "cores": oracle.max_threads(),
                             "ms": round(dt * 1e3, 1), "gteps": round(g.m / dt / 1e9, 4)}
        out["equals_oracle"] = bool(np.array_equal(counts["pull"], ref))
    print(json.dumps({"profile_case": "tc", "scale": args.scale, "n": g.n, "m": g.m, "opts": opts, **out}), flush=True)
    return 0


def run_only_pr_shapes(args):
    """PageRank push against pull on graphs of several shapes, with the default
    options and after gp_autotune (the calibration of GP_AUTO): CUDA-event time
    of --sweeps fixed sweeps, median of 3, per sweep."""
    import torch

    import graphgen as gg
    import paper_2010_16012_gb300 as gp

    def per_sweep(G, n, mode, sweeps):
        out = torch.empty(n, device="cuda")
        gp.pagerank(G, mode, 0.85, sweeps, 0.0, out=out)
        ts = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            gp.pagerank(G, mode, 0.85, sweeps, 0.0, out=out)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return round(statistics.median(ts) / sweeps, 4)

    shapes = [
        ("rmat20_sym", lambda: gg.rmat(20, 16, seed=1)),
        ("rmat20_dir", lambda: gg.rmat(20, 16, seed=1, symmetrize=False)),
        ("rmat20_ef64_sym", lambda: gg.rmat(20, 64, seed=1)),
        ("rmat16_sym", lambda: gg.rmat(16, 16, seed=1)),
        ("dst_skew20_dir", lambda: gg.rmat(20, 16, a=0.45, b=0.05, c=0.45, seed=1, symmetrize=False)),
        ("dst_skew22_dir", lambda: gg.rmat(22, 16, a=0.45, b=0.05, c=0.45, seed=1, symmetrize=False)),
        ("src_skew20_dir", lambda: gg.rmat(20, 16, a=0.45, b=0.45, c=0.05, seed=1, symmetrize=False)),
        ("er22", lambda: gg.erdos_renyi(1 << 22, 16 << 22, seed=3)),
    ]
    sweeps = max(args.sweeps, 20)
    out = {}
    for name, make in shapes:
        g = make()
        G = gp.Graph.from_graphgen(g)
        r = {"n": g.n, "m": g.m, "pull_default_ms": per_sweep(G, g.n, gp.PULL, sweeps),
             "push_default_ms": per_sweep(G, g.n, gp.PUSH, sweeps)}
        t = gp.autotune(G, gp.TUNE_PULL | gp.TUNE_PUSH | gp.TUNE_AUTO, use_cache=False)
        r["pull_tuned_ms"] = per_sweep(G, g.n, gp.PULL, sweeps)
        r["push_tuned_ms"] = per_sweep(G, g.n, gp.PUSH, sweeps)
        r["auto_tuned"] = "push" if t["options"]["pr_auto_mode"] == gp.PUSH else "pull"
        _, st = gp.pagerank(G, gp.AUTO, 0.85, 1, 0.0)
        G.free()
        G = gp.Graph.from_graphgen(g)
        _, st = gp.pagerank(G, gp.AUTO, 0.85, 1, 0.0)
        r["auto_untuned"] = "push" if st["mode_used"] == gp.PUSH else "pull"
        G.free()
        out[name] = r
        log(f"[bench] {name}: {r}")
    print(json.dumps({"profile_case": "pr_shapes", "sweeps": sweeps, **out}), flush=True)
    return 0


def run_only_bc(args):
    """Betweenness centrality (Brandes, push/pull steps) on the R-MAT graph of
    --scale from 16 sources per run, each mode: ms per source, the traversed
    edges per second (m times the sources over the time, the usual rate for
    BC), adjacency entries examined; the first source's step table; the
    oracle's sequential Brandes timed on two of the sources and compared
    (unless --no-cpu-baseline)."""
    import torch

    import paper_2010_16012_gb300 as gp

    g = make_graph(args.scale)
    G = gp.Graph.from_graphgen(g)
    opts = {}
    for kv in args.opt:
        k, v = kv.split("=")
        opts[k] = float(v) if k.endswith("_alpha") or k.endswith("_beta") else int(v)
    if opts:
        G.set_options(**opts)
    src = np.ascontiguousarray(pick_sources(g, 16).astype(np.int32))
    src_dev = torch.from_numpy(src).cuda()
    bc = torch.empty(g.n, dtype=torch.float64, device="cuda")
    out = {}
    res = {}
    for name, mode in (("auto", gp.AUTO), ("pull", gp.PULL), ("push", gp.PUSH)):
        for _ in range(args.warmup):
            gp.bc(G, src_dev, mode, out=bc)
        ms = []
        for _ in range(args.steps):
            _, st = gp.bc(G, src_dev, mode, out=bc)
            ms.append(st["ms"])
        t = statistics.median(ms)
        res[name] = bc.cpu().numpy()
        out[name] = {"ms": round(t, 3), "ms_per_source": round(t / len(src), 4),
                     "gteps": round(g.m * len(src) / (t * 1e-3) / 1e9, 2),
                     "examined_per_source": int(st["edges_examined"] // len(src)),
                     "pushes": st["pushes"], "pulls": st["pulls"]}
        if name == "auto":
            out["steps_first_source"] = [[p, l, d, f, e, round(u, 1)] for p, l, d, f, e, u in
                                         zip(st["phase"], st["level"], st["direction"], st["frontier"],
                                             st["examined"], st["step_us"])]
    ref = res["auto"]
    out["max_rel_diff_modes"] = float(max(np.max(np.abs(res[k] - ref) / np.maximum(np.abs(ref), 1e-300))
                                          for k in ("pull", "push")))
    if not args.no_cpu_baseline:
        import oracle

        O = oracle.OracleGraph.from_graph(g)
        t0 = time.perf_counter()
        r2 = O.bc(src[:2])
        dt = time.perf_counter() - t0
        x2, _ = gp.bc(G, src[:2], gp.AUTO)
        x2 = x2.cpu().numpy()
        out["cpu_oracle"] = {"kind": "oracle", "what": "sequential Brandes, 2 sources", "cores": 1,
                             "ms_per_source": round(dt * 1e3 / 2, 1), "gteps": round(g.m * 2 / dt / 1e9, 4)}
        out["oracle_max_rel_diff"] = float(np.max(np.abs(x2 - r2) / np.maximum(np.abs(r2), 1e-9 * np.abs(r2).max())))
    print(json.dumps({"profile_case": "bc", "scale": args.scale, "n": g.n, "m": g.m, "sources": len(src),
                      "opts": opts, **out}), flush=True)
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.only:
        return run_only(args)
    if args.impl == "reference":
        dist = Dist(backend="gloo") if int(os.environ.get("WORLD_SIZE", "1")) > 1 else Dist()
        out = run_reference(args, dist)
        if out is not None:
            print(json.dumps(out), flush=True)
        dist.close()
        return 0
    import torch

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dist = Dist()
    out = run_ours(args, dist)
    if dist.rank == 0:
        print(json.dumps(out), flush=True)
    dist.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
