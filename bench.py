#!/usr/bin/env python3
"""Order+count throughput of the GB300 k-clique counter (exact counts) on the R-MAT scale-20
workload: 2^20 vertices, edge factor 16, (a,b,c,d) = (0.57,0.19,0.19,0.05), deduplicated,
symmetrised, seeded.

One step = for every k of the step: degree ordering (citron_order) + relabelled DAG
(citron_build_dag, with its largest row) + exact count (citron_count_ex), i.e. one full
order+count job per k.  value = edges of all jobs (m undirected edges per job, all ranks) / device
time of the steps.  At N = 1 the same line carries the rest of the metric, each timed on its own:
R-MAT k = 7 (one job) and k = 8 (under a time budget), the 4M-vertex Chung-Lu graph at k = 5, 6,
the 4,096-graph batch (graphs/s against one launch sequence per graph) and the serving loop
(p50/p99 and requests/s at 100 and 1,000 req/s).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--ks 4,5,6] [--impl ours|reference]
                  [--extras all|none|k7,k8,chunglu,batch,serve]

--impl reference times the oracle (plain C, CPU) on the host cores on a bounded sample of the
same workload.  N > 1 (torchrun) runs independent replicas (the counting of one graph is not
sharded here), one per GPU, with a barrier and the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "order+count edges/s at k=4..9 (exact, 1 GB300); batched graphs/s; serve p50/p99"
UNIT = "edges/s"
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2
# Nominal ceiling of 32-bit AND+POPC word operations: 16 POPC results per clock per SM, 152 SMs,
# 2070 MHz.  The roofline's peak is the rate citron_probe_word_ops measures on the device.
POPC_NOMINAL_OPS = 16 * 152 * 2.070e9
EXTRAS = ("k7", "k8", "chunglu", "batch", "serve")
TUNED = ROOT / "paper_2112_10913_gb300" / "tuned_plans.json"


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--ks", default="4,5,6")
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--cpu-budget", type=float, default=20.0,
                   help="wall seconds of sampled oracle counting per k (bands in parallel processes)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--workload", default="rmat20",
                   choices=["rmat20", "batch", "serve", "orderings", "list", "chunglu", "count", "order"],
                   help="rmat20: order+count edges/s (default); batch: 4,096-graph batched graphs/s; "
                        "serve: request loop at every rate; orderings: degree vs core ordering; "
                        "list: clique listing; chunglu: the 4M-vertex power-law graph, k=5..; "
                        "count: one timed count per k (for profilers); order: the ordering "
                        "phase's calls timed apart (for profilers)")
    p.add_argument("--batch-graphs", type=int, default=4096)
    p.add_argument("--extras", default="all",
                   help="extra measurements of the default line (N = 1 only), comma list of "
                        + ",".join(EXTRAS) + ", or all / none")
    p.add_argument("--k8-budget-s", type=float, default=30.0, help="time budget of the k = 8 count")
    p.add_argument("--chunglu-ks", default="5,6")
    p.add_argument("--chunglu-budget-s", type=float, default=0.0,
                   help="device-time budget of each Chung-Lu count (0: none)")
    p.add_argument("--retune", action="store_true", help="batch: time every plan instead of the cache")
    return p.parse_args(argv)


def extras_of(args) -> set:
    if args.extras == "all":
        return set(EXTRAS)
    if args.extras == "none":
        return set()
    return {e for e in args.extras.split(",") if e in EXTRAS}


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def max_over_ranks(x: float, device="cpu") -> float:
    """The largest of every rank's value (the slowest replica sets the job time); x itself on
    one rank.  Uses the initialised process group (NCCL on GPUs, gloo on the CPU)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job throughput of N independent replicas: all ranks' units over the slowest time."""
    return units_per_rank * world / (ms_max / 1e3)


def workload():
    from paper_2112_10913_gb300 import graphgen as gg

    return gg.config2_rmat()


# ---------------------------------------------------------------------------------------------
# CPU side: the oracle (whole jobs where it finishes, else a stratified sample of edge tasks)

BANDS = [(0, 8), (8, 16), (16, 32), (32, 64), (64, 128), (128, 256), (256, 512), (512, 1 << 30)]


def oracle_order(g):
    """The oracle's degree ordering and relabelled DAG of the whole graph: (dag, seconds)."""
    import oracle

    t0 = time.perf_counter()
    rank = oracle.degree_rank(g.off, g.n)
    dag = oracle.dag_by_rank(g.off, g.cols, g.n, rank, True)
    return dag, time.perf_counter() - t0


def _band_worker(dag_off, dag_cols, n, k, plan, q):
    """Runs in a spawned process: times the oracle's edge tasks on one thread, one group of
    sampled DAG arcs at a time in the plan's order, and reports each group as soon as it is
    done."""
    import oracle

    oracle.build()
    # the cost of a call that counts nothing (row-width scan, scratch set-up): subtracted per group
    none = np.zeros(0, dtype=np.uint64)
    cost = []
    for _ in range(7):
        t0 = time.perf_counter()
        oracle.count_arcs(dag_off, dag_cols, n, k, none)
        cost.append(time.perf_counter() - t0)
    q.put(("call", 0, float(np.median(cost))))
    for band, arcs in plan:
        t0 = time.perf_counter()
        oracle.count_arcs(dag_off, dag_cols, n, k, arcs)
        q.put((band, int(arcs.size), time.perf_counter() - t0))
    q.put(None)


def _group_size(lo: int) -> int:
    """Arcs per timed group in a band whose roots have out-degree above lo: many cheap edge tasks
    per call in light bands (so the call's own cost stays small against them), few in heavy
    ones (an edge task of a heavy root can take a tenth of a second at k = 6)."""
    return max(4, min(256, 4096 // max(lo, 16)))


def oracle_stratified(dag, n, k, budget_s, seed=2, groups=8, per=None):
    """Single-thread oracle counting time of one k (k >= 3), estimated from a stratified sample
    of edge tasks.  The unit is the edge-parallel form's task: the k-cliques whose first two
    vertices are the ends of one DAG arc (the oracle's count_arcs; a root's time is the sum of
    its arcs' times).  Arcs of the roots that can hold a k-clique are split into bands by their
    root's out-degree; every band gets up to `groups` seeded groups of arcs (per arcs each, else
    a size set by the band), timed on one thread in one worker process, round-robin over the
    bands from the heaviest down, so that every band is sampled early.  A band's time is its arc
    count times its mean time per sampled arc (inverse-probability weighting), with a standard
    error from the spread of its groups.  Sampling stops budget_s after the worker is ready (the
    worker is stopped): a band with no group done by then is left out, and the estimate is then a
    lower bound.  Returns (seconds on one thread, standard error, sampled arcs, bands left out)."""
    import multiprocessing as mp
    import queue as queue_mod

    from paper_2112_10913_gb300 import graphgen as gg

    dag_off, dag_cols = dag
    outdeg = np.diff(dag_off).astype(np.int64)
    chunks, sizes, takes = {}, {}, {}
    for b, (lo, hi) in enumerate(BANDS):
        roots = np.nonzero((outdeg >= max(k - 1, lo + 1)) & (outdeg <= hi))[0]
        if not roots.size:
            continue
        starts = dag_off[roots].astype(np.int64)
        lens = outdeg[roots]
        total = int(lens.sum())
        # every arc of the band's roots, then a seeded sample of them
        ids = np.repeat(starts - np.concatenate(([0], np.cumsum(lens)[:-1])), lens) + np.arange(total)
        ids = ids[gg.permutation(seed, 20 + b, total)]
        gsize = per if per is not None else _group_size(lo)
        take = min(total, gsize * groups)
        nch = max(1, -(-take // gsize))
        chunks[b] = [c.astype(np.uint64) for c in np.array_split(ids[:take], nch) if c.size]
        sizes[b], takes[b] = total, take
    plan = []
    for r in range(max((len(c) for c in chunks.values()), default=0)):
        for b in sorted(chunks, reverse=True):
            if r < len(chunks[b]):
                plan.append((b, chunks[b][r]))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    proc = ctx.Process(target=_band_worker, args=(dag_off, dag_cols, n, k, plan, q), daemon=True)
    proc.start()
    done = {b: [] for b in sizes}
    # the budget counts from the worker's first report: its start-up (interpreter, arrays) is not
    # sampling time; a worker that never reports is given up after a minute
    deadline = time.perf_counter() + 60.0
    finished, call_s = False, 0.0
    while not finished and time.perf_counter() < deadline:
        try:
            item = q.get(timeout=min(0.5, max(0.01, deadline - time.perf_counter())))
        except queue_mod.Empty:
            continue
        if item is None:
            finished = True
        elif item[0] == "call":
            call_s = item[2]
            deadline = time.perf_counter() + budget_s
        else:
            done[item[0]].append((item[1], max(0.0, item[2] - call_s)))
    if not finished:
        proc.terminate()
    proc.join(timeout=10)
    est, var, sampled, missing = 0.0, 0.0, 0, []
    for b, res in done.items():
        if not res:
            missing.append(BANDS[b])
            continue
        rates = [t / c for c, t in res]
        sampled += sum(c for c, _ in res)
        est += sizes[b] * float(np.mean(rates))
        if len(rates) > 1 and takes[b] < sizes[b]:
            var += (sizes[b] ** 2) * float(np.var(rates, ddof=1)) / len(rates)
    return est, var ** 0.5, sampled, missing


def cpu_baseline_obj(g, ks, budget_s, gpu_counts=None):
    """The oracle on this host's cores for the same jobs: ordering + DAG on the whole graph;
    counting on the whole graph, all threads, for k <= 4 (checked against the GPU's count); for
    larger k, the single-thread time estimated from a stratified sample of edge tasks
    (oracle_stratified) over the thread count (the oracle's roots are independent tasks taken
    dynamically: ideal scaling is assumed)."""
    import oracle

    oracle.build()
    threads = oracle.default_threads()
    dag, t_order = oracle_order(g)
    per_k, total, se2, samples = {}, 0.0, 0.0, []
    lower = False
    for k in ks:
        if k <= 4:
            t0 = time.perf_counter()
            c = oracle.count(dag[0], dag[1], g.n, k, threads)
            t_count = time.perf_counter() - t0
            if gpu_counts is not None:
                assert c == gpu_counts[k], f"oracle k={k}: {c} != GPU {gpu_counts[k]}"
            per_k[str(k)] = dict(seconds=t_order + t_count, order_s=t_order, count_s=t_count,
                                 count=c, count_equal_gpu=gpu_counts is not None, sample="whole graph")
            total += t_order + t_count
            samples.append(f"k={k} on the whole graph, all threads")
        else:
            t1, se1, m, missing = oracle_stratified(dag, g.n, k, budget_s)
            scale = 1.0 / threads
            est, se = t1 * scale, se1 * scale
            per_k[str(k)] = dict(seconds=t_order + est, order_s=t_order, count_s=est, count_se_s=se,
                                 single_thread_s=t1,
                                 sample=f"{m} edge tasks (DAG arcs) stratified by their root's out-degree",
                                 bands_not_sampled=[list(b) for b in missing],
                                 lower_bound=bool(missing))
            total += t_order + est
            se2 += se * se
            lower = lower or bool(missing)
            samples.append(f"k={k} from {m} edge tasks (DAG arcs) stratified by their root's out-degree, "
                           "single-thread times "
                           "weighted by inverse sampling probability, over the thread count"
                           + (f" (out-degree bands {missing} not sampled within {budget_s:.0f} s: "
                              "a lower bound on the time)" if missing else ""))
    se = se2 ** 0.5
    units = g.m * len(ks)
    return dict(value=units / total, unit=UNIT, cores=threads, kind="oracle",
                sample="oracle ordering + DAG on the whole graph per job; counting " + "; ".join(samples),
                seconds_per_step=total, seconds_se=se,
                seconds_is_lower_bound=lower,
                value_1se_range=[units / (total + se), units / max(total - se, 1e-9)], per_k=per_k)


# ---------------------------------------------------------------------------------------------
# Clocks during the timed region


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[4:8]):
                if flag.lower() in ("active", "1", "yes"):
                    reasons.add(name)
        if not sm:
            return None
        return dict(sm_mhz=statistics.median(sm), sm_max_mhz=max(smax), reasons=sorted(reasons),
                    samples=len(sm))



# ---------------------------------------------------------------------------------------------
# GPU side


def _hbm_peak() -> float:
    try:
        return float(json.loads((ROOT / "MEASURED_PEAKS.json").read_text())["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def run_ours(args, ks):
    import torch

    rank, local_rank, world = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    from paper_2112_10913_gb300 import build as B

    B.build()
    import paper_2112_10913_gb300 as cg

    g = workload()
    n, arcs, m = g.n, g.arcs, g.m
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    off = torch.from_numpy(g.off.view(np.int64)).to(dev)
    cols = torch.from_numpy(g.cols.view(np.int32)).to(dev)
    rank_t = torch.empty(n, dtype=torch.int32, device=dev)
    dag_off = torch.empty(n + 1, dtype=torch.int64, device=dev)
    dag_cols = torch.empty(arcs // 2, dtype=torch.int32, device=dev)
    ws = cg.alloc_workspace(n, arcs, 1, device=dev)
    cg.citron_order(n, off, rank_t, None, ws)
    max_outdeg = cg.citron_build_dag(n, off, cols, rank_t, dag_off, dag_cols, ws)
    ws = cg.alloc_workspace(n, arcs, max_outdeg, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    def job(k, timed, **kw):
        """One order+count job; returns (count, order_ms, count_ms, kernel_ms, opts)."""
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        cg.citron_order(n, off, rank_t, None, ws)
        mx = cg.citron_build_dag(n, off, cols, rank_t, dag_off, dag_cols, ws)
        e1.record(stream)
        c, o = cg.citron_count_ex(n, dag_off, dag_cols, k, ws, mx, time_kernels=timed, **kw)
        e2.record(stream)
        e2.synchronize()
        return c, e0.elapsed_time(e1), e1.elapsed_time(e2), list(o.kernel_ms), o

    def step(timed=False):
        return [job(k, timed) for k in ks]

    ref = None
    for _ in range(max(args.warmup, 0)):
        flush.fill_(1)
        out = step()
        counts = [r[0] for r in out]
        assert ref is None or counts == ref, "counts changed between runs"
        ref = counts
    # instrumented (untimed) launch per k: word operations of the bitmap kernel (the instrumented
    # kernel is built for k <= 8)
    work = {k: (cg.citron_count_ex(n, dag_off, dag_cols, k, ws, max_outdeg, count_work=True)[1].work_ops
                if k <= 8 else None)
            for k in ks}
    # measured peak of the word operation on this device (registers only, all SMs)
    peak_ops, peak_ms = cg.citron_probe_word_ops(2, 200000)

    clocks = ClockSampler(local_rank)
    launches0 = cg.citron_kernel_launches()
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    per_step, per_job = [], {k: [] for k in ks}
    for _ in range(args.steps):
        flush.fill_(2)  # L2 flush between timed steps (outside the step's events)
        out = step(timed=True)
        assert [r[0] for r in out] == (ref or [r[0] for r in out]), "counts changed between runs"
        ref = [r[0] for r in out]
        per_step.append(sum(r[1] + r[2] for r in out))
        for k, r in zip(ks, out):
            per_job[k].append(r)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = cg.citron_kernel_launches() - launches0
    ms_step = statistics.mean(per_step) if per_step else float("nan")
    if world > 1:
        import torch.distributed as dist

        ms_step = max_over_ranks(ms_step, dev)
        dist.barrier()

    # end to end through the host-buffer entry point: H2D of the CSR + order + DAG + count + D2H
    h_off = torch.from_numpy(g.off.view(np.int64)).pin_memory()
    h_cols = torch.from_numpy(g.cols.view(np.int32)).pin_memory()
    dbuf = torch.empty(cg.citron_host_buffer_bytes(n, arcs), dtype=torch.uint8, device=dev)
    e2e_steps = max(1, min(args.steps, 3))
    cg.citron_count_host(n, h_off, h_cols, [ks[0]], dbuf, ws)
    torch.cuda.synchronize()
    e2e_ms = []
    for _ in range(e2e_steps):
        flush.fill_(3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        got = [cg.citron_count_host(n, h_off, h_cols, [k], dbuf, ws)[0] for k in ks]
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        assert got == ref, "end-to-end counts differ"
    e2e_step = statistics.mean(e2e_ms)
    if world > 1:
        e2e_step = max_over_ranks(e2e_step, dev)
    del dbuf

    if rank != 0:
        return None
    units = m * len(ks) * world
    value = replica_throughput(m * len(ks), world, ms_step)
    # dominant kernel: the bitmap counting kernel of the largest k with a word-op count
    kd = max([k for k in ks if work[k] is not None] or ks, key=lambda k: statistics.mean(r[3][1] for r in per_job[k]))
    kern_ms = statistics.mean(r[3][1] for r in per_job[kd])
    achieved = work[kd] / (kern_ms / 1e3) if work[kd] is not None else None
    order_ms = statistics.mean(r[1] for k in ks for r in per_job[k])
    order_bytes = 8 * (n + 1) + 4 * arcs + 8 * (n + 1) + 4 * (arcs // 2) + 4 * n
    sm_mhz = clk["sm_mhz"] if clk else None
    per_k = {str(k): {"count": per_job[k][-1][0],
                      "order_ms": statistics.mean(r[1] for r in per_job[k]),
                      "count_ms": statistics.mean(r[2] for r in per_job[k]),
                      "bitmap_kernel_ms": statistics.mean(r[3][1] for r in per_job[k]),
                      "small_kernel_ms": statistics.mean(r[3][0] for r in per_job[k]),
                      "edges_per_s": m / ((statistics.mean(r[1] + r[2] for r in per_job[k])) / 1e3),
                      "word_ops": work[k], "repeats": args.steps}
             for k in ks}
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32/u64 (exact integer)",
        "data": "synthetic (seeded R-MAT)",
        "config": {
            "workload": f"rmat20-ef16 k={','.join(map(str, ks))}",
            "n": n, "m_undirected": m, "arcs": arcs, "max_outdeg": max_outdeg,
            "ks": ks, "counts": {str(k): c for k, c in zip(ks, ref)},
            "step": "per k: citron_order + citron_build_dag (relabelled, largest row) + citron_count_ex",
            "l2": "flushed between steps (256 MB write outside the step events); CSR 134 MB > L2",
            "parallelism": "replicas" if world > 1 else "single GPU",
        },
        "per_k": per_k,
        "roofline": {"kernel": f"k_count_mid<{kd}> (bitmap path)", "bound": "alu",
                     "achieved": achieved / 1e12 if achieved is not None else None, "peak": peak_ops / 1e12,
                     "unit": "T word-ops/s (32-bit AND+POPC)",
                     "frac": achieved / peak_ops if achieved is not None else None, "traffic": None,
                     "peak_source": ("measured: citron_probe_word_ops (AND+POPC+add on registers, "
                                     f"all SMs, {peak_ms:.1f} ms) before the timed steps; nominal "
                                     f"{POPC_NOMINAL_OPS / 1e12:.2f} T/s at 2070 MHz"),
                     "sm_mhz_median": sm_mhz},
        "roofline_order": {"kernels": "citron_order + citron_build_dag (relabelled)", "bound": "hbm",
                           "achieved": order_bytes / (order_ms / 1e3) / 1e9, "unit": "GB/s",
                           "peak": _hbm_peak(), "frac": order_bytes / (order_ms / 1e3) / 1e9 / _hbm_peak(),
                           "algorithmic_bytes": order_bytes, "ms": order_ms},
        "e2e": {"value": units / (e2e_step / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": len(ks) * (g.off.nbytes + g.cols.nbytes),
                "d2h_bytes_per_step": len(ks) * 8, "ms_per_step": e2e_step,
                "api": "citron_count_host (pinned host CSR)"},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    extras = extras_of(args) if world == 1 else set()
    if "k7" in extras:
        flush.fill_(4)
        c, o_ms, c_ms, kms, o = job(7, True, balance=True)
        per_k["7"] = {"count": c, "order_ms": o_ms, "count_ms": c_ms, "bitmap_kernel_ms": kms[1],
                      "edges_per_s": m / ((o_ms + c_ms) / 1e3), "repeats": 1,
                      "bitmap_kernel_tail_frac": o.busy_ms[1] / o.busy_ms[0] if o.busy_ms[0] else None,
                      "note": "timed once outside the step (order + DAG + count, CUDA events)"}
    if "k8" in extras:
        budget = float(args.k8_budget_s)
        t0 = time.perf_counter()
        try:
            c, o_ms, c_ms, _, _ = job(8, True, budget_ms=int(budget * 1000))
            per_k["8"] = {"count": c, "order_ms": o_ms, "count_ms": c_ms,
                          "edges_per_s": m / ((o_ms + c_ms) / 1e3), "repeats": 1}
        except cg.CitronError as exc:
            if exc.name != "CITRON_E_BUDGET":
                raise
            per_k["8"] = {"count": None, "did_not_finish_within_s": budget,
                          "stopped_after_s": time.perf_counter() - t0,
                          "note": "the count's time budget ran out (CITRON_E_BUDGET); no count"}
    del flush, ws, dag_off, dag_cols, rank_t, off, cols
    torch.cuda.empty_cache()
    if "chunglu" in extras:
        line["chunglu"] = chunglu_obj(cg, [int(k) for k in args.chunglu_ks.split(",") if k],
                                      args.chunglu_budget_s)
        torch.cuda.empty_cache()
    if "batch" in extras:
        line["batch"] = batch_obj(args, cg)
        torch.cuda.empty_cache()
    if "serve" in extras:
        line["serve"] = serve_obj(cg, rates=(100, 1000), per_rate=400)
        torch.cuda.empty_cache()
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_obj(g, ks, args.cpu_budget,
                                                gpu_counts={k: c for k, c in zip(ks, ref)})
    return line


def chunglu_obj(cg, ks, budget_s: float = 0.0):
    """The 4M-vertex Chung-Lu graph (exponent 2.1, average degree 30, degrees capped at 20,000,
    50 planted cliques of 20-40 vertices): order + relabelled DAG + count per k, CUDA events.
    budget_s > 0 bounds each count's device time (a k that runs out is recorded without a
    count)."""
    import torch

    from paper_2112_10913_gb300 import graphgen as gg

    t0 = time.perf_counter()
    g = gg.config3_chung_lu()
    t_gen = time.perf_counter() - t0
    G = cg.DeviceGraph(g)

    def order_dag():
        cg.citron_order(g.n, G.off, G.rank, None, G.ws)
        return cg.citron_build_dag(g.n, G.off, G.cols, G.rank, G.dag_off, G.dag_cols, G.ws)

    t_order = _events_ms(order_dag)
    per_k = {}
    for k in ks:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        a.record()
        try:
            c, o = cg.citron_count_ex(g.n, G.dag_off, G.dag_cols, k, G.ws, G.max_outdeg, time_kernels=True,
                                      balance=True, budget_ms=int(budget_s * 1000))
        except cg.CitronError as exc:
            if exc.name != "CITRON_E_BUDGET":
                raise
            per_k[str(k)] = {"count": None, "did_not_finish_within_s": budget_s,
                             "stopped_after_s": time.perf_counter() - t0}
            continue
        b.record()
        b.synchronize()
        ms = a.elapsed_time(b)
        per_k[str(k)] = dict(count=c, count_ms=ms, order_ms=t_order, edges_per_s=g.m / ((ms + t_order) / 1e3),
                             bitmap_kernel_ms=o.kernel_ms[1],
                             bitmap_kernel_tail_frac=o.busy_ms[1] / o.busy_ms[0] if o.busy_ms[0] else None)
    tot = sum(per_k[str(k)]["count_ms"] + t_order for k in ks if per_k[str(k)]["count"] is not None)
    return {"workload": "chunglu-4M beta=2.1 avg30 cap20000 + 50 planted cliques (seed 3)",
            "n": g.n, "m_undirected": g.m, "max_outdeg": G.max_outdeg, "ks": ks,
            "edges_per_s": (g.m * sum(per_k[str(k)]["count"] is not None for k in ks) / (tot / 1e3)
                            if tot > 0 else None),
            "order_dag_ms": t_order, "per_k": per_k,
            "generation_s": t_gen}


def _batch_plan(bc, args):
    """The autotuner's plan for this batch: the cached choice for this device and batch, or a new
    timing of the candidate plans (kept in the cache)."""
    import torch

    from paper_2112_10913_gb300.batch import tune

    key = f"{torch.cuda.get_device_name()}|config4-seed4-{len(bc.ks)}graphs"
    if args.retune and TUNED.exists():
        known = json.loads(TUNED.read_text())
        known.pop(key, None)
        TUNED.write_text(json.dumps(known, indent=1))
    return tune(bc, repeats=1, cache=TUNED, key=key), key


def batch_obj(args, cg):
    """Batched graphs/s on the 4,096-graph workload: n log-uniform in [50, 50000], ER and R-MAT
    half and half, average degree U[8, 64], k U{3..7}, seed 4.  One step = degree ordering and
    DAG of the union + the batched count replayed from its CUDA graph; compared with counting
    every graph through its own launches (upload, order, DAG, count)."""
    import torch

    from paper_2112_10913_gb300 import graphgen as gg
    from paper_2112_10913_gb300.batch import BatchCounter

    t0 = time.perf_counter()
    items = gg.config4_batch_parallel(seed=4, count=args.batch_graphs)
    t_gen = time.perf_counter() - t0
    graphs, ks = [it.graph for it in items], [it.k for it in items]
    bc = BatchCounter(graphs, ks)
    tuned, key = _batch_plan(bc, args)
    bc.capture()
    bc.replay()
    ref = bc.result()
    torch.cuda.synchronize()
    steps = []
    for _ in range(1):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record()
        bc.build()  # ordering + DAG of the union (synchronises once for the largest row)
        e[1].record()
        bc.replay()
        e[2].record()
        e[2].synchronize()
        assert bc.result() == ref, "batched counts changed between replays"
        steps.append((e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])))
    order_ms = statistics.mean(a for a, _ in steps)
    count_ms = statistics.mean(b for _, b in steps)
    del bc
    torch.cuda.empty_cache()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    single = [cg.DeviceGraph(g).count(k) for g, k in zip(graphs, ks)]
    torch.cuda.synchronize()
    t_single = time.perf_counter() - t1
    assert single == ref, "batched and one-graph counts differ"
    return {"workload": f"{len(graphs)} graphs, n log-uniform [50,50000], ER/R-MAT, avg degree U[8,64], "
                        "k U{3..7}, seed 4",
            "graphs_per_s": len(graphs) / ((order_ms + count_ms) / 1e3), "unit": "graphs/s",
            "ms_per_step": order_ms + count_ms, "steps": len(steps),
            "order_dag_ms": order_ms, "batched_count_replay_ms": count_ms,
            "one_launch_per_graph": {"seconds": t_single, "graphs_per_s": len(graphs) / t_single,
                                     "counts_equal": True},
            "speedup_vs_one_launch_per_graph": (len(graphs) / ((order_ms + count_ms) / 1e3)) / (len(graphs) / t_single),
            "tuned_plan": {k: v for k, v in tuned.items() if k not in ("tried",)}, "plan_cache_key": key,
            "k_histogram": {str(k): int(c) for k, c in enumerate(np.bincount(ks)) if c},
            "generation_s": t_gen}


def _serve_pool(per_rate):
    from paper_2112_10913_gb300 import graphgen as gg

    pool = gg.config4_batch_parallel(seed=5, count=per_rate)
    big = [gg.config2_rmat(seed=50 + i, scale=18, edge_factor=16) for i in range(2)]
    for j in range(0, per_rate, 50):  # 2 % of the requests
        pool[j] = gg.BatchItem(big[(j // 50) % 2], pool[j].k)
    return pool


def _alone_summary(pool, alone_ms, heavy_arcs: int) -> dict:
    """Latency of every request served alone (its floor): p50/p99 of all requests and of the
    light ones (below the heavy lane's arc threshold), and the sum."""
    light = [t for it, t in zip(pool, alone_ms) if not (heavy_arcs and it.graph.arcs >= heavy_arcs)]
    out = {"p50": float(np.percentile(alone_ms, 50)), "p99": float(np.percentile(alone_ms, 99)),
           "sum_s": float(sum(alone_ms) / 1e3)}
    if light:
        out["light_p50"] = float(np.percentile(light, 50))
        out["light_p99"] = float(np.percentile(light, 99))
    return out


def serve_obj(cg, rates=(100, 1000), per_rate=400):
    """The request loop (continuous batching) on Poisson arrivals at the given rates: requests
    drawn from the batch distribution (seed 5) plus 2 % R-MAT scale-18 graphs; p50/p99 of all
    requests and of the light lane, achieved requests/s; every count equal to the graph counted
    alone, whose own latency is the floor."""
    from paper_2112_10913_gb300.serve import Request, ServeConfig, ServeEngine, poisson_arrivals, summarize

    pool = _serve_pool(per_rate)
    alone, alone_ms = [], []
    for it in pool:
        t0 = time.perf_counter()
        alone.append(cg.DeviceGraph(it.graph).count(it.k))
        alone_ms.append((time.perf_counter() - t0) * 1e3)
    cfg = ServeConfig()
    per = {}
    for rate in rates:
        arrivals = poisson_arrivals(float(rate), per_rate, seed=rate)
        reqs = [Request(i, it.graph, it.k, arrival=float(a)) for i, (it, a) in enumerate(zip(pool, arrivals))]
        eng = ServeEngine(cfg)
        try:
            done = eng.run(reqs, timeout_s=600)
        finally:
            eng.close()
        assert [r.count for r in sorted(done, key=lambda r: r.rid)] == alone, "serving changed a count"
        per[str(rate)] = summarize(done)
        per[str(rate)]["host_ms_by_phase"] = {k: round(v, 1) for k, v in eng.phase_ms.items()}
        per[str(rate)]["cache_hits"] = eng.cache.hits if eng.cache else 0
    return {"workload": f"{per_rate} requests per rate from the batch distribution (seed 5) + 2% R-MAT "
                        "scale 18, Poisson arrivals",
            "per_rate": per, "counts_equal_alone": True,
            "alone_latency_ms": _alone_summary(pool, alone_ms, cfg.heavy_arcs),
            "config": {k: getattr(cfg, k) for k in ("slots", "max_batch_requests", "heavy_arcs",
                                                    "heavy_sm_fraction", "hbm_budget_bytes")}}


def run_reference(args, ks):
    """The oracle arm: the oracle on this host's cores, on the same workload, metric and unit.
    Every step orders the whole graph and estimates each k's counting time from a stratified
    sample of roots sized so that the whole run ends within a few minutes."""
    rank, _, world = dist_env()
    if rank != 0:
        return None
    import oracle

    oracle.build()
    threads = oracle.default_threads()
    g = workload()
    budget = max(0.5, min(args.cpu_budget, 150.0 / max(1, (args.steps + args.warmup) * len(ks))))
    times, last, lower = [], None, False
    for i in range(args.warmup + args.steps):
        dag, t_order = oracle_order(g)
        t = 0.0
        for k in ks:
            t1, _, sampled, missing = oracle_stratified(dag, g.n, k, budget, seed=2 + i)
            t += t_order + t1 / threads
            lower = lower or (bool(missing) and i >= args.warmup)
        if i >= args.warmup:
            times.append(t)
        last = sampled
    t = statistics.mean(times)
    value = g.m * len(ks) / t
    sample = (f"oracle ordering + DAG on the whole graph per job; counting time per k estimated from "
              f"edge tasks (DAG arcs) stratified by their root's out-degree ({budget:.1f} s of "
              f"single-thread sampling per k, inverse-probability weighted, divided by {threads} "
              f"threads; last k: {last} arcs)"
              + ("; some out-degree bands were not reached within the budget in a timed step: the "
                 "time is a lower bound" if lower else ""))
    return {
        "impl": "reference",
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32/u64 (exact integer)", "data": "synthetic (seeded R-MAT)",
        "config": {"workload": f"rmat20-ef16 k={','.join(map(str, ks))}", "n": g.n, "m_undirected": g.m,
                   "ks": ks},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_batch(args):
    """The batch measurement alone, as its own line."""
    from paper_2112_10913_gb300 import build as B

    B.build()
    import paper_2112_10913_gb300 as cg

    b = batch_obj(args, cg)
    return {"metric": "batched graphs/s (exact per-graph k-clique counts)", "value": b["graphs_per_s"],
            "unit": "graphs/s", "n_gpus": 1, "steps": b["steps"], "warmup": 1,
            "ms_per_step": b["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32/u64 (exact integer)", "data": "synthetic (seeded ER/R-MAT)",
            "config": {"workload": b["workload"]}, "batch": b}


def run_serve(args):
    """Serving with continuous batching: Poisson arrivals at 100..5000 req/s of (graph, k)
    requests drawn from the batch workload's distribution (seed 5) plus 2 % R-MAT scale-18 graphs
    (edge factor 16), and one rate below the device's capacity (25 req/s); p50/p99 latency (all,
    light lane, heavy lane), queueing delay and achieved requests/s per rate; every count is
    checked against the same graph counted alone."""
    import torch

    from paper_2112_10913_gb300 import build as B

    B.build()
    import paper_2112_10913_gb300 as cg
    from paper_2112_10913_gb300 import graphgen as gg
    from paper_2112_10913_gb300.serve import Request, ServeConfig, ServeEngine, poisson_arrivals, summarize

    per_rate = 400
    pool = _serve_pool(per_rate)
    alone, alone_ms = [], []
    for it in pool:  # each request served alone (upload, order, DAG, count): the latency floor
        t0 = time.perf_counter()
        alone.append(cg.DeviceGraph(it.graph).count(it.k))
        alone_ms.append((time.perf_counter() - t0) * 1e3)
    results = {}
    cfg = ServeConfig(slots=4, max_batch_requests=64)
    for rate in (25, 100, 500, 1000, 2000, 5000):
        arrivals = poisson_arrivals(float(rate), per_rate, seed=rate)
        reqs = [Request(i, it.graph, it.k, arrival=float(a)) for i, (it, a) in enumerate(zip(pool, arrivals))]
        eng = ServeEngine(cfg)
        try:
            done = eng.run(reqs, timeout_s=600)
        finally:
            eng.close()
        assert [r.count for r in sorted(done, key=lambda r: r.rid)] == alone, "serving changed a count"
        results[str(rate)] = summarize(done)
        results[str(rate)]["host_ms_by_phase"] = {k: round(v, 1) for k, v in eng.phase_ms.items()}
        results[str(rate)]["cache_hits"] = eng.cache.hits if eng.cache else 0
    top = results["5000"]
    return {
        "metric": "serve p50/p99 latency and requests/s (exact counts, continuous batching)",
        "value": top["req_per_s"], "unit": "requests/s", "n_gpus": 1, "steps": len(results),
        "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32/u64 (exact integer)", "data": "synthetic (seeded ER/R-MAT)",
        "config": {"workload": f"{per_rate} requests per rate from the batch distribution (seed 5) "
                               "+ 2% R-MAT scale 18; rates 25 and 100..5000 req/s (Poisson)",
                   "slots": cfg.slots, "max_batch_requests": cfg.max_batch_requests,
                   "heavy_arcs": cfg.heavy_arcs, "heavy_sm_fraction": cfg.heavy_sm_fraction},
        "per_rate": results, "counts_equal_alone": True,
        "alone_latency_ms": _alone_summary(pool, alone_ms, cfg.heavy_arcs),
    }


def _events_ms(fn, reps: int = 3) -> float:
    """Mean device time (ms) of fn() over reps runs, CUDA events on the current stream."""
    import torch

    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    b.synchronize()
    return a.elapsed_time(b) / reps


def run_orderings(args):
    """Degree ordering (CITRON, Sec. IV) against the core ordering (Sec. III, computed in
    synchronous rounds) on R-MAT scale 20: ordering time, DAG time, maximum out-degree and the
    counting time it leads to (the comparison of Table II and Table III)."""
    import torch

    from paper_2112_10913_gb300 import build as B

    B.build()
    import paper_2112_10913_gb300 as cg

    g = workload()
    dev = torch.device("cuda")
    off = torch.from_numpy(g.off.view(np.int64)).to(dev)
    cols = torch.from_numpy(g.cols.view(np.int32)).to(dev)
    ws = cg.alloc_workspace(g.n, g.arcs, 1024, device=dev)
    rank = torch.empty(g.n, dtype=torch.int32, device=dev)
    dag_off = torch.empty(g.n + 1, dtype=torch.int64, device=dev)
    dag_cols = torch.empty(g.arcs // 2, dtype=torch.int32, device=dev)
    ks = [int(x) for x in args.ks.split(",") if x]
    out = {}
    for name in ("degree", "core"):
        info = {}
        if name == "degree":
            order = lambda: cg.citron_order(g.n, off, rank, None, ws)
        else:
            def order():
                info["degeneracy"], info["rounds"] = cg.citron_core_order(g.n, off, cols, rank, None, ws)
        t_order = _events_ms(order)
        t_dag = _events_ms(lambda: cg.citron_build_dag(g.n, off, cols, rank, dag_off, dag_cols, ws,
                                                      want_max_outdeg=False))
        mx = cg.citron_build_dag(g.n, off, cols, rank, dag_off, dag_cols, ws)
        counts = {}
        for k in ks:
            c, o = cg.citron_count_ex(g.n, dag_off, dag_cols, k, ws, mx, None, None, time_kernels=True)
            t = _events_ms(lambda: cg.citron_count(g.n, dag_off, dag_cols, k, ws, mx), reps=1)
            counts[str(k)] = dict(count=c, count_ms=t)
        out[name] = dict(order_ms=t_order, dag_ms=t_dag, max_outdeg=mx, per_k=counts, **info)
    for k in ks:
        assert out["degree"]["per_k"][str(k)]["count"] == out["core"]["per_k"][str(k)]["count"]
    d, c = out["degree"], out["core"]
    return {
        "metric": "ordering comparison (Table II/III analogue): order ms, max out-degree, count ms",
        "value": c["order_ms"] / d["order_ms"], "unit": "core/degree ordering time ratio",
        "n_gpus": 1, "steps": 3, "warmup": 1, "ms_per_step": None, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64 (exact integer)",
        "data": "synthetic (seeded R-MAT)",
        "config": {"workload": "rmat20-ef16", "n": g.n, "m_undirected": g.m, "ks": ks},
        "orderings": out,
    }


def run_list(args):
    """Listing (Sec. VIII): every k-clique written out as k ids, on R-MAT scale 20 for k = 3 and
    4 (the output must fit in HBM).  Bound: the output writes (k x 4 bytes per clique)."""
    import torch

    from paper_2112_10913_gb300 import build as B

    B.build()
    import paper_2112_10913_gb300 as cg

    g = workload()
    dg = cg.DeviceGraph(g)
    peak = _hbm_peak()
    res = {}
    for k in (3, 4):
        total = cg.citron_list(dg.n, dg.dag_off, dg.dag_cols, k, dg.ws)
        if total * k * 4 > (64 << 30):
            res[str(k)] = dict(cliques=total, skipped="output above 64 GiB")
            continue
        out_t = torch.empty((total, k), dtype=torch.int32, device="cuda")
        ms = _events_ms(lambda: cg.citron_list(dg.n, dg.dag_off, dg.dag_cols, k, dg.ws, out_t), reps=3)
        assert total == dg.count(k)
        gbs = total * k * 4 / (ms * 1e-3) / 1e9
        res[str(k)] = dict(cliques=total, ms=ms, cliques_per_s=total / (ms * 1e-3), out_gb_s=gbs,
                           frac_of_hbm=gbs / peak)
        del out_t
        torch.cuda.empty_cache()
    top = res.get("4", res["3"])
    return {
        "metric": "k-clique listing (cliques/s; output GB/s)", "value": top.get("cliques_per_s"),
        "unit": "cliques/s", "n_gpus": 1, "steps": 3, "warmup": 1, "ms_per_step": top.get("ms"),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32 ids", "data": "synthetic (seeded R-MAT)",
        "config": {"workload": "rmat20-ef16 listing k=3,4 (DAG ids mapped to none)", "n": g.n},
        "roofline": {"bound": "hbm", "achieved": top.get("out_gb_s"), "peak": peak, "unit": "GB/s",
                     "frac": top.get("frac_of_hbm"), "traffic": None,
                     "note": "algorithmic bytes = the rows written (k x 4 B per clique)"},
        "per_k": res,
    }


def run_chunglu(args):
    """The 4M-vertex Chung-Lu workload (exponent 2.1, avg degree 30, degrees capped at 20,000,
    50 planted cliques of 20-40 vertices): order + relabelled DAG + count per k, k = 5..9 while a
    count stays under a minute; per-root share of the heaviest roots (load balance)."""
    import torch

    from paper_2112_10913_gb300 import build as B

    B.build()
    import paper_2112_10913_gb300 as cg
    from paper_2112_10913_gb300 import graphgen as gg

    g = gg.config3_chung_lu()
    dev = torch.device("cuda")
    off = torch.from_numpy(g.off.view(np.int64)).to(dev)
    cols = torch.from_numpy(g.cols.view(np.int32)).to(dev)
    ws = cg.alloc_workspace(g.n, g.arcs, 1, device=dev)
    rank = torch.empty(g.n, dtype=torch.int32, device=dev)
    dag_off = torch.empty(g.n + 1, dtype=torch.int64, device=dev)
    dag_cols = torch.empty(g.arcs // 2, dtype=torch.int32, device=dev)

    def order_dag():
        cg.citron_order(g.n, off, rank, None, ws)
        return cg.citron_build_dag(g.n, off, cols, rank, dag_off, dag_cols, ws)

    mx = order_dag()
    if cg.citron_workspace_bytes(g.n, g.arcs, mx) > ws.numel():
        ws = cg.alloc_workspace(g.n, g.arcs, mx, device=dev)
    t_order = _events_ms(order_dag)
    per_k = {}
    prev_ms = None
    for k in range(5, 10):
        if prev_ms is not None and len(per_k) >= 2:
            ks_done = sorted(per_k, key=int)
            growth = per_k[ks_done[-1]]["count_ms"] / max(per_k[ks_done[-2]]["count_ms"], 1e-3)
            if prev_ms * growth > 60000:  # the next k would take over a minute: stop here
                break
        pr = torch.zeros(g.n, dtype=torch.int64, device=dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        c = cg.citron_count(g.n, dag_off, dag_cols, k, ws, mx, pr)
        b.record()
        b.synchronize()
        ms = a.elapsed_time(b)
        p = np.sort(pr.cpu().numpy().view(np.uint64).astype(np.float64))[::-1]
        per_k[str(k)] = dict(count=c, count_ms=ms, order_ms=t_order,
                             edges_per_s=g.m / ((ms + t_order) * 1e-3),
                             top_root_share=float(p[0] / max(p.sum(), 1)),
                             top100_share=float(p[:100].sum() / max(p.sum(), 1)))
        prev_ms = ms
        if ms > 60000:
            break
    ks = list(per_k)
    tot = sum(per_k[k]["count_ms"] + t_order for k in ks)
    return {
        "metric": "order+count edges/s on the Chung-Lu 4M graph (exact)",
        "value": g.m * len(ks) / (tot * 1e-3), "unit": "edges/s", "n_gpus": 1, "steps": 1,
        "warmup": 1, "ms_per_step": tot, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32/u64 (exact integer)", "data": "synthetic (seeded Chung-Lu)",
        "config": {"workload": "chunglu-4M beta=2.1 avg30 cap20000 + 50 planted cliques", "n": g.n,
                   "m_undirected": g.m, "max_outdeg": mx, "ks": [int(k) for k in ks]},
        "per_k": per_k,
    }


def run_count_only(args):
    """One timed count per k of --ks on R-MAT scale 20, after the DAG is built: the launch a
    profiler captures for the counting kernels."""
    from paper_2112_10913_gb300 import build as B

    B.build()
    import paper_2112_10913_gb300 as cg

    g = workload()
    G = cg.DeviceGraph(g)
    per_k = {}
    for k in [int(x) for x in args.ks.split(",") if x]:
        for _ in range(max(1, args.steps)):
            c, o = cg.citron_count_ex(g.n, G.dag_off, G.dag_cols, k, G.ws, G.max_outdeg, time_kernels=True)
        per_k[str(k)] = dict(count=c, bitmap_kernel_ms=o.kernel_ms[1], small_kernel_ms=o.kernel_ms[0])
    return {"metric": "counting kernels (one count per k)", "value": None, "unit": "ms",
            "config": {"workload": "rmat20-ef16", "n": g.n}, "per_k": per_k}


def run_order_only(args):
    """The ordering phase's calls timed apart on R-MAT scale 20 (CUDA events, median of --steps):
    the degree ordering, the relabelled DAG, Algorithm GenOrdering's DAG."""
    import torch

    from paper_2112_10913_gb300 import build as B

    B.build()
    import paper_2112_10913_gb300 as cg

    g = workload()
    n, arcs = g.n, g.arcs
    dev = torch.device("cuda")
    off = torch.from_numpy(g.off.view(np.int64)).to(dev)
    cols = torch.from_numpy(g.cols.view(np.int32)).to(dev)
    rank = torch.empty(n, dtype=torch.int32, device=dev)
    dag_off = torch.empty(n + 1, dtype=torch.int64, device=dev)
    dag_cols = torch.empty(arcs // 2, dtype=torch.int32, device=dev)
    ws = cg.alloc_workspace(n, arcs, 1024, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    def timed(fn):
        ts = []
        for i in range(max(1, args.steps)):
            flush.fill_(i)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    res = {
        "order_ms": timed(lambda: cg.citron_order(n, off, rank, None, ws)),
        "dag_relabel_ms": timed(lambda: cg.citron_build_dag(n, off, cols, rank, dag_off, dag_cols, ws,
                                                             want_max_outdeg=False)),
        "dag_genordering_ms": timed(lambda: cg.citron_build_dag(n, off, cols, None, dag_off, dag_cols, ws,
                                                                want_max_outdeg=False)),
    }
    order_bytes = 8 * (n + 1) + 4 * arcs + 8 * (n + 1) + 4 * (arcs // 2) + 4 * n
    gen_bytes = 8 * (n + 1) + 4 * arcs + 8 * (n + 1) + 4 * (arcs // 2)
    t = res["order_ms"] + res["dag_relabel_ms"]
    return {"metric": "ordering phase (degree ordering + DAG), GB/s of algorithmic bytes",
            "value": order_bytes / (t / 1e3) / 1e9, "unit": "GB/s", "ms_per_step": t,
            "frac_of_hbm": order_bytes / (t / 1e3) / 1e9 / _hbm_peak(),
            "genordering_gb_s": gen_bytes / (res["dag_genordering_ms"] / 1e3) / 1e9,
            "config": {"workload": "rmat20-ef16", "n": n, "arcs": arcs, "l2": "flushed between reps"},
            **res}


def main():
    args = parse()
    ks = [int(x) for x in args.ks.split(",") if x]
    if args.workload == "batch":
        line = run_batch(args)
    elif args.workload == "serve":
        line = run_serve(args)
    elif args.workload == "orderings":
        line = run_orderings(args)
    elif args.workload == "list":
        line = run_list(args)
    elif args.workload == "chunglu":
        line = run_chunglu(args)
    elif args.workload == "count":
        line = run_count_only(args)
    elif args.workload == "order":
        line = run_order_only(args)
    elif args.impl == "reference":
        line = run_reference(args, ks)
    else:
        line = run_ours(args, ks)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
