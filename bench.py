"""Benchmark: USTs sampled+aggregated per second and diag(L^+) wall time.

One step = the whole path of Algorithm 1 on one workload, by default the
largest single-GPU one: R-MAT scale 22, edge factor 16, a,b,c,d =
0.57,0.19,0.19,0.05, symmetrised, deduplicated, self-loops removed, largest
component (n = 2,394,915, m = 64.2M), max-degree pivot. The step computes
the BFS tree B_u, tau(eps = 0.3) = 9,475 Wilson trees with their Algorithm 2
counts, the exact reduction into R, the FP32-PCG + FP64-refinement column
solve and the FP64 diagonal. Inputs are resident on the device when a timed
step starts; L2 is flushed (256 MB write) between timed steps, outside the
timed region. Other workloads: --workload (grid48, rmat16, hyperbolic20,
batch256, and the profiling cases rmat17 and rmat19).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line. With N > 1 (torchrun, one rank per GPU) rank r
samples the tree ids [T r, T (r + 1)) under the common seed (weak scaling),
the integer counts are summed across ranks (the paper's final reduction of
R; the sum equals one GPU sampling all T N trees) and the max step time over
ranks is reported.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "USTs sampled+aggregated/sec and diag(L†) wall time on 1 GB300; % of L2/HBM roofline"
SEED = 0
# DRAM traffic of the sampler from ncu captures of the sampler kernel: bytes per
# vertex-tree of the captured launch, the workloads it is scaled to, and the sha1 of
# the sampler's code (the kernel and the relabelling that orders its memory, without
# comments; sampler_sha1) when it was taken.
TRAFFIC_CAPTURES = [
    # R-MAT scale 22, one launch of 1,520 trees: 877.8 GB read + 341.1 GB written
    {"applies_to": ["rmat22"], "sha1": "7cebea6f53a1855be183fd46c529cdd07dbd6d37",
     "bytes_per_vertex_tree": 1218.95e9 / (1520 * 2394915)},
]
SAMPLER_SOURCES = ("ust_wilson.cu", "ust_relabel.cu")

# workload -> (description, oracle sample in trees for the CPU baseline; None = all)
WORKLOADS = {
    "rmat22": ("R-MAT scale 22, edge factor 16, (0.57,0.19,0.19,0.05), LCC, max-degree pivot, tau(eps=0.3)", 48),
    "rmat16": ("R-MAT scale 16, edge factor 16, (0.57,0.19,0.19,0.05), LCC, max-degree pivot, 4096 trees", None),
    "grid48": ("48x48 4-neighbour grid, pivot (24,24), 1000 trees", None),
    "rmat17": ("R-MAT scale 17, edge factor 16, LCC, max-degree pivot, 1024 trees (a small case of the "
               "large-graph sampler, for profiling)", None),
    "rmat19": ("R-MAT scale 19, edge factor 16, LCC, max-degree pivot, 1024 trees (a case of the large-graph "
               "sampler whose per-tree state, like R-MAT 22's, is far larger than L2, for profiling)", 256),
    "hyperbolic20": ("random hyperbolic graph n=2^20, avg degree 20, exponent 3, T=0, LCC, max-degree pivot, "
                     "tau(eps=0.3)", 128),
    "batch256": ("256 graphs: even index Barabasi-Albert (k = avg/2), odd index Erdos-Renyi, n ~ U[1000, 64000], "
                 "average degree ~ U[8, 32], LCC, per-graph max-degree pivot, 1024 trees each", None),
}
BATCH_GRAPHS = 256
BATCH_TREES = 1024
# Upper vertex counts of the library's batch size classes (kClassMaxN in
# csrc/ust_common.cuh); --per-class times each class as a batch of its own.
BATCH_CLASS_MAX_N = (4096, 8192, 14336, 28672, 56 * 1024, 0xFFFF, 2 ** 31 - 1)
# CPU baseline sample of the batch workload: the first graphs, this many trees each
BATCH_CPU_GRAPHS = 16
BATCH_CPU_TREES = 64

# Algorithmic bytes (what the method must touch, no cache effects):
#   per Wilson draw: row_ptr pair 8 B + col_idx 4 B + successor write 4 B + stack depth 4 B
#   per vertex per tree (intervals + aggregation bookkeeping): 40 B
#   per pair test of Algorithm 2 (f^c(u) per tree): bfs_parent 4 B + successor 4 B + interval 8 B
BYTES_PER_DRAW = 20
BYTES_PER_VERTEX = 40
BYTES_PER_PAIR = 16


def algorithmic_bytes(draws: int, trees: int, n: int, farness: int) -> int:
    return BYTES_PER_DRAW * draws + trees * (BYTES_PER_VERTEX * n + BYTES_PER_PAIR * farness)


def phase_names(n: int):
    """Names of the sampler's per-tree cycle counters (thread 0's clock per
    phase), which depend on the kernel that serves a graph of n vertices."""
    if n <= 0xFFFF:
        return ["first_draws", "in_degrees", "leaf_queue", "peeling", "cycle_list", "pop_rounds", "child_counts",
                "sizes_offsets", "preorder", "aggregation", "tree_total"]
    return ["first_draws_in_degrees", "peeling", "cycle_list", "pop_rounds", "sizes_offsets", "preorder",
            "aggregation", "tree_total"]


# One-tree-per-launch comparator: trees timed (the rest extrapolated); fewer on
# graphs above 65,535 vertices, where one tree on one CTA takes tens of milliseconds.
COMPARATOR_TREES = 1024
COMPARATOR_TREES_LARGE = 64


def sampler_kernel(n: int) -> str:
    return "sample_aggregate_smem_kernel" if n <= 0xFFFF else "sample_aggregate_large_kernel"


def code_of(text: str) -> str:
    """C++ source without its comments and blank lines (what a capture's
    validity depends on)."""
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(line.rstrip() for line in text.splitlines() if line.strip())


def sampler_sha1():
    """sha1 over the code (comments left out) of the sampler's sources, in
    SAMPLER_SOURCES order."""
    import hashlib
    h = hashlib.sha1()
    try:
        for name in SAMPLER_SOURCES:
            path = os.path.join(ROOT, "paper_2006_13679_gb300", "csrc", name)
            h.update(code_of(open(path, encoding="utf-8").read()).encode())
    except OSError:
        return None
    return h.hexdigest()


def traffic_per_launch(workload: str, n: int, trees: int):
    """DRAM bytes (read + write) of one sampler launch: an ncu capture's
    dram__bytes_read.sum + dram__bytes_write.sum per vertex-tree, times this
    launch's n x trees. A capture counts only while the sampler sources hash
    as they did when the counters were taken; None otherwise."""
    sha = sampler_sha1()
    if sha is None:
        return None
    for cap in TRAFFIC_CAPTURES:
        if workload in cap["applies_to"] and cap["sha1"] == sha:
            return cap["bytes_per_vertex_tree"] * n * trees
    return None


def gather_peaks(pkg, stream) -> dict:
    """Random 4-byte access rates of this GPU, measured by the library's probe
    (ust_probe_random_access) before the timed region: loads over a 32 MB
    array (served by L2) and over a 4 GB array (served by HBM). Bytes are
    counted as 4 per access (what an algorithmic byte count charges one
    gather), sectors as 32."""
    l2 = pkg.probe_random_access(32 << 20, 0, 3, stream)
    hbm = pkg.probe_random_access(4 << 30, 0, 3, stream)
    return {"l2_gather_gbs": l2 * 4 / 1e9, "l2_sector_gbs": l2 * 32 / 1e9,
            "hbm_gather_gbs": hbm * 4 / 1e9, "hbm_sector_gbs": hbm * 32 / 1e9,
            "how": "ust_probe_random_access: 2048 threads per SM, 8 independent random 4-byte loads each in "
                   "flight (L1 bypassed), best of 3 launches; 32 MB array (L2) and 4 GB array (HBM)"}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


def gpu_index(local_rank: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    parts = [p for p in vis.split(",") if p.strip()]
    if parts and parts[min(local_rank, len(parts) - 1)].strip().isdigit():
        return int(parts[min(local_rank, len(parts) - 1)])
    return local_rank


def oracle_tau(g, u, T, eps):
    """Trees per step for the oracle arm: the workload's fixed count, else
    tau(eps) of Algorithm 1 from the oracle's own BFS."""
    if T is not None:
        return T
    import oracle
    ecc, _, _ = oracle.bfs(g, u)
    return oracle.tau(ecc, g.m, eps, 1.0 / g.n, 0.3)


def oracle_step(g, u, T, sample, threads, walk=None):
    """One step of the oracle on the host cores: BFS, trees [0, sample) of the
    T (OpenMP over trees, thread-local R, then the reduction), the FP64
    Jacobi-CG column solve and the combination. Returns (seconds measured,
    seconds with the tree part scaled to all T trees)."""
    import oracle
    t0 = time.perf_counter()
    ecc, dist, par = oracle.bfs(g, u)
    t1 = time.perf_counter()
    R, _ = oracle.sample_aggregate(walk if walk is not None else g, u, par, 0, sample, SEED, threads=threads)
    t2 = time.perf_counter()
    x, _, _, _ = oracle.cg(g, u, tol=1e-9)
    oracle.combine(R, sample, x, u)
    t3 = time.perf_counter()
    return t3 - t0, (t1 - t0) + (t2 - t1) * T / sample + (t3 - t2)


def sample_label(T, sample, threads):
    if sample == T:
        return f"one full step (BFS + {T} trees + FP64 CG + combine), OpenMP over trees on {threads} cores"
    return (f"BFS + trees [0, {sample}) of the {T} + FP64 CG + combine per step, OpenMP over trees on {threads} "
            f"cores; the tree part extrapolated to all {T} trees (value = {T} / extrapolated step time)")


def run_reference(args, rank: int, world: int) -> None:
    """The oracle (plain C, OpenMP over trees) on the host cores."""
    if rank != 0:
        return
    import oracle
    import synth
    if args.workload == "batch256":
        run_reference_batch(args, world)
        return
    g, u, T0, eps = synth.workload(args.workload)
    T = oracle_tau(g, u, T0, eps)
    threads = oracle.max_threads()
    sample = min(T, WORKLOADS[args.workload][1] or T)
    for _ in range(args.warmup):
        oracle_step(g, u, T, sample, threads)
    measured, extrapolated = [], []
    for _ in range(args.steps):
        a, b = oracle_step(g, u, T, sample, threads)
        measured.append(a)
        extrapolated.append(b)
    sec = statistics.mean(extrapolated)
    value = T / sec
    label = sample_label(T, sample, threads)
    line = {"metric": METRIC, "value": value, "unit": "trees/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload][0]}; n={g.n} m={g.m}, pivot {u}, "
                                   f"{T} trees per GPU (tree ids rank*{T} onwards), seed {SEED}",
                       "sample": label},
            "measured_ms_per_sample_step": statistics.mean(measured) * 1e3,
            "cpu_baseline": {"value": value, "unit": "trees/s", "cores": threads, "kind": "oracle",
                             "sample": label, "extrapolated": sample != T},
            "e2e": {"value": value, "unit": "trees/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batch_workload():
    import synth
    gs = [synth.batch_graph(sp) for sp in synth.batch_specs(BATCH_GRAPHS)]
    return gs, [synth.max_degree_vertex(g) for g in gs]


def oracle_batch_sample(gs, pivots, threads):
    """The oracle on the CPU sample of the batch: BFS, trees, FP64 CG and the
    combination for the first BATCH_CPU_GRAPHS graphs, BATCH_CPU_TREES trees
    each (graph id = index). Returns (trees, seconds)."""
    import oracle
    t0 = time.perf_counter()
    for i in range(BATCH_CPU_GRAPHS):
        g, u = gs[i], pivots[i]
        _, _, par = oracle.bfs(g, u)
        R, _ = oracle.sample_aggregate(g, u, par, 0, BATCH_CPU_TREES, SEED, graph=i, threads=threads)
        x, _, _, _ = oracle.cg(g, u, tol=1e-9)
        oracle.combine(R, BATCH_CPU_TREES, x, u)
    return BATCH_CPU_GRAPHS * BATCH_CPU_TREES, time.perf_counter() - t0


def run_reference_batch(args, world: int) -> None:
    import oracle
    gs, pivots = batch_workload()
    threads = oracle.max_threads()
    for _ in range(args.warmup):
        oracle_batch_sample(gs, pivots, threads)
    times = []
    trees = 0
    for _ in range(args.steps):
        trees, sec = oracle_batch_sample(gs, pivots, threads)
        times.append(sec)
    sec = statistics.mean(times)
    value = trees / sec
    sample = (f"BFS + {BATCH_CPU_TREES} trees + FP64 CG + combine for each of the first {BATCH_CPU_GRAPHS} "
              f"of the {BATCH_GRAPHS} graphs per step")
    line = {"metric": METRIC, "value": value, "unit": "trees/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"batch256: {WORKLOADS['batch256'][0]}; total n={sum(g.n for g in gs)}",
                       "sample": sample},
            "cpu_baseline": {"value": value, "unit": "trees/s", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "trees/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batch_gpu(args, rank: int, world: int, local_rank: int, dist) -> None:
    """The batch workload: one step = B_u of every graph, 1024 trees of every
    graph through the batched sampler launches, every graph's column solve
    and the diagonals. The comparator loops the single-graph path over the
    same graphs (same tree ids and graph words, so the counts must match)."""
    import numpy as np
    import torch

    import paper_2006_13679_gb300 as pkg

    gs, pivots = batch_workload()
    T = BATCH_TREES
    seed = SEED + rank
    ntot = sum(g.n for g in gs)
    stream = torch.cuda.Stream()
    b = pkg.USTBatch([(g.row_ptr, g.col_idx) for g in gs], pivots, stream=stream, skip_validation=True, autotune=1)
    diag_d = torch.empty(ntot, dtype=torch.float64, device="cuda")
    counts_d = torch.empty(ntot, dtype=torch.int64, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def step():
        b.reset()                     # B_u of every graph, clear R and columns
        b.sample_aggregate(T, seed)   # T trees of every graph (seed offset by rank)
        if dist is not None:          # counts summed over ranks and installed
            b.counts(counts_d)
            with torch.cuda.stream(stream):
                dist.all_reduce(counts_d)
            b.set_counts(counts_d, world * T)
        if dist is None or rank == 0:  # every graph's column solve + combination, on one rank
            b.diag(0.0, diag_d)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    sample_ms, bfs_ms, solve_ms, draws = [], [], [], []
    launches0 = b.info()["kernel_launches"]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(gpu_index(local_rank)) as clk:
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            ev0[k].record(stream)
            step()
            ev1[k].record(stream)
            inf = b.info()
            sample_ms.append(inf["sample_ms"])
            bfs_ms.append(inf["bfs_ms"])
            solve_ms.append(inf["solve_ms"])
            draws.append(inf["last_draws"])
        torch.cuda.synchronize()
    launches = b.info()["kernel_launches"] - launches0
    if dist is not None:
        dist.barrier()
    ms = statistics.mean(a.elapsed_time(c) for a, c in zip(ev0, ev1))
    if dist is not None:
        t = torch.tensor([ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    trees_step = len(gs) * T
    value = world * trees_step / (ms / 1e3)
    clocks = clk.summary()
    info = b.info()
    kernel_ms = statistics.mean(sample_ms)
    farness = [b.graph_info(i)["farness"] for i in range(len(gs))]
    alg = BYTES_PER_DRAW * int(statistics.mean(draws)) + sum(
        T * (BYTES_PER_VERTEX * g.n + BYTES_PER_PAIR * f) for g, f in zip(gs, farness))
    peak, peak_kind = peaks()
    achieved = alg / (kernel_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "kernel": "sample_aggregate_smem_kernel + sample_aggregate_kernel (batch launches)",
                "kernel_ms": kernel_ms, "algorithmic_bytes": alg, "peak_kind": peak_kind}
    R_batch = b.counts()

    # comparator: the single-graph path looped over the graphs (contexts
    # created outside the timed regions; each graph timed on the same stream)
    comparator = None
    if not args.no_comparator:
        loop_ms = 0.0
        same = True
        off = b.offsets()
        for i, (g, u) in enumerate(zip(gs, pivots)):
            with pkg.UST(g.row_ptr, g.col_idx, u, stream=stream, skip_validation=True, graph_id=i) as h:
                out = diag_d[off[i]:off[i + 1]]
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                h.reset(u)
                h.sample_aggregate(T, seed)
                h.diag(0.0, out)
                e1.record(stream)
                torch.cuda.synchronize()
                loop_ms += e0.elapsed_time(e1)
                same = same and bool(np.array_equal(h.counts(), R_batch[off[i]:off[i + 1]]))
        comparator = {"form": "single-graph path looped over the 256 graphs (one context per graph)",
                      "ms_per_step": loop_ms, "value": trees_step / (loop_ms / 1e3), "unit": "trees/s",
                      "batched_speedup": loop_ms / ms, "counts_equal_to_batch": same}

    # each size class on its own (outside the timed region): where the
    # sampler time of the batch goes
    per_class = None
    if args.per_class:
        per_class = []
        lo = 0
        for hi in BATCH_CLASS_MAX_N:
            idx = [i for i, g in enumerate(gs) if lo < g.n <= hi]
            lo = hi
            if not idx:
                continue
            with pkg.USTBatch([(gs[i].row_ptr, gs[i].col_idx) for i in idx], [pivots[i] for i in idx],
                              stream=stream, skip_validation=True) as sb:
                times = []
                for k in range(3):  # the first run warms up
                    sb.reset()
                    sb.sample_aggregate(T, seed)
                    torch.cuda.synchronize()
                    if k > 0:
                        times.append(sb.info()["sample_ms"])
                shape = sb.graph_info(0)
                per_class.append({"max_n": hi, "graphs": len(idx), "vertices": sum(gs[i].n for i in idx),
                                  "arcs": sum(gs[i].nnz for i in idx), "trees": len(idx) * T,
                                  "sample_ms": statistics.mean(times),
                                  "draws_per_tree": sb.info()["last_draws"] / (len(idx) * T),
                                  "sampler": f"{shape['sample_ctas']} CTAs x {shape['sample_threads']} threads"})

    # end to end through the public API with host buffers
    e2e = None
    if args.e2e_steps > 0:
        h2d = sum((g.n + 1) * 4 + g.nnz * 4 for g in gs)
        d2h = ntot * 8
        secs = []
        for k in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with pkg.USTBatch([(g.row_ptr, g.col_idx) for g in gs], pivots) as be:
                be.sample_aggregate(T, seed)
                be.diag()
            if k > 0:
                secs.append(time.perf_counter() - t0)
        e2e = {"value": trees_step / statistics.mean(secs), "unit": "trees/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": statistics.mean(secs) * 1e3}

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            import oracle
            threads = oracle.max_threads()
            trees_cpu, sec = oracle_batch_sample(gs, pivots, threads)
            cpu = {"value": trees_cpu / sec, "unit": "trees/s", "cores": threads, "kind": "oracle",
                   "sample": f"BFS + {BATCH_CPU_TREES} trees + FP64 CG + combine for each of the first "
                             f"{BATCH_CPU_GRAPHS} of the {len(gs)} graphs, OpenMP over trees", "seconds": sec}
        line = {"metric": METRIC, "value": value, "unit": "trees/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                "config": {"workload": f"batch256: {WORKLOADS['batch256'][0]}; total n={ntot}, "
                                       f"total arcs={sum(g.nnz for g in gs)}, {T} trees per graph per GPU, "
                                       f"seed {SEED}+rank",
                           "l2": "flushed between timed steps (256 MB write); inputs exceed L2",
                           "sampler": f"{info['sample_ctas']} CTAs x {info['sample_threads']} threads"},
                "diag_ms": ms, "phase_ms": {"bfs": statistics.mean(bfs_ms), "sample_kernel": kernel_ms,
                                            "solve": statistics.mean(solve_ms)},
                "draws_per_tree": statistics.mean(draws) / trees_step, "cg_iters": info["cg_iters"],
                "cg_relres": info["cg_relres"], "roofline": roofline, "clocks": clocks, "gpu_launches": launches,
                "gpu_launches_per_step": launches / args.steps, "e2e": e2e, "cpu_baseline": cpu,
                "comparator": comparator}
        if per_class is not None:
            line["per_class"] = per_class
        print(json.dumps(line), flush=True)
    b.close()
    if dist is not None:
        dist.destroy_process_group()


def cpu_baseline(g, u, T, sample, wilson_blocks: bool = False) -> dict:
    import oracle
    threads = oracle.max_threads()
    _, _, par = oracle.bfs(g, u)
    walk = oracle.parent_block_graph(g, u, par) if wilson_blocks else g  # rows built before the timed step
    oracle.sample_aggregate(walk, u, par, 0, min(16, sample), SEED, threads=threads)  # warm
    measured, extrapolated = oracle_step(g, u, T, sample, threads, walk)
    label = sample_label(T, sample, threads)
    if wilson_blocks:
        label += "; walks on the parent-block rows (built outside the timed step)"
    # the sequential oracle on one core, over a share of the sample that
    # takes about as long as the run above
    k = max(1, min(sample, sample // max(1, threads)))
    t1 = time.perf_counter()
    _, _, par1 = oracle.bfs(g, u)
    oracle.sample_aggregate(walk, u, par1, 0, k, SEED, threads=1)
    sec1 = time.perf_counter() - t1
    return {"value": T / extrapolated, "unit": "trees/s", "cores": threads, "kind": "oracle",
            "sample": label, "extrapolated": sample != T, "seconds": measured,
            "one_core": {"value": k / sec1, "unit": "trees/s", "trees": k,
                         "sample": f"BFS + {k} trees, sequential (the sampling loop of Algorithm 1)"}}


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="rmat22", choices=sorted(WORKLOADS))
    ap.add_argument("--wilson-blocks", action="store_true",
                    help="single-graph workloads: walks inside each vertex's parent block "
                         "(the biconnected-component variant)")
    ap.add_argument("--block-threads", type=int, default=0,
                    help="single-graph workloads: threads per sampling CTA (0 = the library's choice)")
    ap.add_argument("--ctas-per-sm", type=int, default=0,
                    help="single-graph workloads: sampling CTAs per SM (0 = the library's choice)")
    ap.add_argument("--trees", type=int, default=0,
                    help="single-graph workloads: trees per step instead of the workload's own count")
    ap.add_argument("--per-class", action="store_true",
                    help="batch256: also time each size class of the batch on its own")
    ap.add_argument("--no-comparator", action="store_true",
                    help="skip the one-tree-per-launch + all-FP64-solve comparison")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch

    import paper_2006_13679_gb300 as pkg
    import synth

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    pkg.build()
    from paper_2006_13679_gb300 import parallel
    if args.workload == "batch256":
        if args.wilson_blocks:
            raise SystemExit("--wilson-blocks applies to the single-graph workloads")
        run_batch_gpu(args, rank, world, local_rank, dist)
        return
    g, u, T0, eps = synth.workload(args.workload)
    seed = SEED
    stream = torch.cuda.Stream()
    rp_d = torch.from_numpy(g.row_ptr).cuda()
    ci_d = torch.from_numpy(g.col_idx).cuda()
    shape = dict(block_threads=args.block_threads, ctas_per_sm=args.ctas_per_sm)
    h = pkg.UST(rp_d, ci_d, u, stream=stream, skip_validation=True, wilson_blocks=args.wilson_blocks, **shape)
    # trees per step: the workload's fixed count, else tau(eps) of Algorithm 1 (ust_tau)
    T = args.trees if args.trees > 0 else (T0 if T0 is not None else h.tau(eps))
    gather = gather_peaks(pkg, stream)
    diag_d = torch.empty(g.n, dtype=torch.float64, device="cuda")
    counts_d = torch.empty(g.n, dtype=torch.int64, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def step():
        h.reset(u)                    # B_u, ecc, clear R
        if dist is None:
            h.sample_aggregate(T, seed)   # Wilson + intervals + Algorithm 2 + exact reduction
            h.diag(0.0, diag_d)           # column solve + combination
        else:                         # rank 0 solves the column; every rank samples its tree ids;
            with torch.cuda.stream(stream):  # counts summed and installed; rank 0 combines
                parallel.diag_sharded(h, T, seed, out=diag_d, counts_out=counts_d)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    sample_ms, bfs_ms, solve_ms, draws = [], [], [], []
    launches0 = h.info()["kernel_launches"]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(gpu_index(local_rank)) as clk:
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            ev0[k].record(stream)
            step()
            ev1[k].record(stream)
            inf = h.info()
            sample_ms.append(inf["sample_ms"])
            bfs_ms.append(inf["bfs_ms"])
            solve_ms.append(inf["solve_ms"])
            draws.append(inf["last_draws"])
        torch.cuda.synchronize()
    launches = h.info()["kernel_launches"] - launches0
    if dist is not None:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    ms = statistics.mean(step_ms)
    if dist is not None:
        t = torch.tensor([ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * T / (ms / 1e3)
    clocks = clk.summary()

    info = h.info()
    kernel_ms = statistics.mean(sample_ms)
    alg = algorithmic_bytes(int(statistics.mean(draws)), T, g.n, info["farness"])
    peak, peak_kind = peaks()
    achieved = alg / (kernel_ms / 1e3) / 1e9
    traffic = traffic_per_launch(args.workload, g.n, T) if not args.wilson_blocks else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": sampler_kernel(g.n), "kernel_ms": kernel_ms,
                "algorithmic_bytes": alg, "peak_kind": peak_kind,
                # the same algorithmic bytes against the random-gather ceilings of this GPU
                "peak_l2": gather["l2_gather_gbs"], "frac_l2": achieved / gather["l2_gather_gbs"],
                "peak_hbm_gather": gather["hbm_gather_gbs"], "frac_hbm_gather": achieved / gather["hbm_gather_gbs"],
                # the measured DRAM bytes of the launch against the HBM copy peak
                "frac_dram": (traffic / (kernel_ms / 1e3) / 1e9 / peak) if traffic else None,
                "gather_probe": gather}

    # end to end through the public API with host buffers in pinned memory
    # (validation included): the CSR goes in, the diagonal comes out
    e2e_times = []
    if args.e2e_steps > 0:
        rp_pin = torch.from_numpy(g.row_ptr).pin_memory()
        ci_pin = torch.from_numpy(g.col_idx).pin_memory()
        d_pin = torch.empty(g.n, dtype=torch.float64).pin_memory()
    for k in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with pkg.UST(rp_pin, ci_pin, u, wilson_blocks=args.wilson_blocks, **shape) as he:
            he.sample_aggregate(T, seed)
            he.diag(out=d_pin)
        t1 = time.perf_counter()
        if k > 0:
            e2e_times.append(t1 - t0)
    e2e_sec = statistics.mean(e2e_times) if e2e_times else None
    h2d = (g.n + 1) * 4 + g.nnz * 4
    d2h = g.n * 8

    # In-GPU comparator: the same kernels launched for one tree at a time (one
    # CTA per launch) and the column solved entirely in FP64 - the form the
    # batched persistent launch and the mixed-precision solve replace. Timed
    # once, on the same stream and events, outside the measured steps.
    # (on the large workloads a sample of the trees, one per launch, scaled
    # to all T trees)
    comparator = None
    if not args.no_comparator:
        hc = pkg.UST(rp_d, ci_d, u, stream=stream, skip_validation=True, solve_fp64=True,
                     wilson_blocks=args.wilson_blocks, **shape)
        tc = min(T, COMPARATOR_TREES if g.n <= 0xFFFF else COMPARATOR_TREES_LARGE)
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        hc.reset(u)
        e1.record(stream)
        for _ in range(tc):
            hc.sample_aggregate(1, seed)
        e2.record(stream)
        hc.diag(0.0, diag_d)
        e3 = torch.cuda.Event(enable_timing=True)
        e3.record(stream)
        torch.cuda.synchronize()
        trees_ms = e1.elapsed_time(e2) * T / tc
        cms = e0.elapsed_time(e1) + trees_ms + e2.elapsed_time(e3)
        ci = hc.info()
        comparator = {"form": "one tree per launch (1 CTA) + all-FP64 Jacobi-PCG column solve",
                      "ms_per_step": cms, "value": T / (cms / 1e3), "unit": "trees/s",
                      "trees_timed": tc, "extrapolated": tc != T,
                      "solve_ms": ci["solve_ms"], "cg_iters": ci["cg_iters"],
                      "batched_speedup": cms / ms}
        hc.close()

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline(g, u, T, min(T, WORKLOADS[args.workload][1] or T), args.wilson_blocks)
        line = {"metric": METRIC, "value": value, "unit": "trees/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload][0]}; n={g.n} m={g.m}, "
                                       f"pivot {u}, {T} trees per GPU (tree ids rank*{T} onwards), seed {SEED}",
                           "l2": "flushed between timed steps (256 MB write)",
                           "sampler": f"{info['sample_ctas']} CTAs x {info['sample_threads']} threads",
                           "walks": ("inside each vertex's parent block (biconnected-component variant; "
                                     "the step's reset rebuilds the rows)" if args.wilson_blocks
                                     else "plain Wilson rooted at the pivot")},
                "diag_ms": ms, "phase_ms": {"bfs": statistics.mean(bfs_ms), "sample_kernel": kernel_ms,
                                            "solve": statistics.mean(solve_ms)},
                "sampler_cycles_per_tree": dict(zip(phase_names(g.n),
                                                    [c / max(1, info["last_trees"]) for c in info["last_phase_cycles"]])),
                "draws_per_tree": statistics.mean(draws) / T, "cg_iters": info["cg_iters"],
                "cg_refinements": info["cg_refinements"], "cg_relres": info["cg_relres"],
                "roofline": roofline, "clocks": clocks, "gpu_launches": launches,
                "gpu_launches_per_step": launches / args.steps,
                "e2e": ({"value": T / e2e_sec, "unit": "trees/s", "h2d_bytes_per_step": h2d,
                         "d2h_bytes_per_step": d2h, "ms_per_step": e2e_sec * 1e3} if e2e_sec else None),
                "cpu_baseline": cpu, "comparator": comparator}
        print(json.dumps(line), flush=True)
    h.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
