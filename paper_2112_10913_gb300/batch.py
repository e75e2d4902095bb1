"""Batched counting: many graphs, each with its own k, in one capturable launch sequence.

The graphs are concatenated into one CSR (their disjoint union).  Degree ordering and the DAG are
built once for the union (no edge crosses two graphs, so the union's DAG is the union of the
graphs' DAGs), and ``citron_count_batch`` counts every graph's cliques for its own k, adding each
root's count to its graph's total.  That call never synchronises the host, so the whole batch
count is captured into one CUDA graph and replayed.

Every step runs in the CUDA library; this module only assembles inputs and marshals calls.
"""
from __future__ import annotations

import json
import time
from pathlib import Path

import numpy as np

from . import (CountOpts, alloc_workspace, citron_build_dag, citron_count_batch, citron_order,
               citron_workspace_bytes, citron_workspace_status)
from .graphgen import Csr


def union_csr(graphs: list[Csr]):
    """Disjoint union of CSR graphs (ids shifted) and the graph of each vertex."""
    n = sum(g.n for g in graphs)
    arcs = sum(g.arcs for g in graphs)
    if n >= (1 << 32) - 1:
        raise ValueError("the union has too many vertices for uint32 ids")
    off = np.zeros(n + 1, dtype=np.uint64)
    cols = np.empty(arcs, dtype=np.uint32)
    group = np.empty(n, dtype=np.uint32)
    vbase, abase = 0, 0
    for i, g in enumerate(graphs):
        off[vbase + 1: vbase + g.n + 1] = g.off[1:] + np.uint64(abase)
        cols[abase: abase + g.arcs] = g.cols + np.uint32(vbase)
        group[vbase: vbase + g.n] = i
        vbase += g.n
        abase += g.arcs
    return Csr(n=n, off=off, cols=cols, name=f"union{len(graphs)}"), group


class BatchCounter:
    """A batch of (graph, k) requests resident on one device."""

    def __init__(self, graphs: list[Csr], ks: list[int], device="cuda", opts: CountOpts | None = None,
                 max_blocks: int = 0):
        import torch

        if len(graphs) != len(ks):
            raise ValueError("one k per graph")
        self.dev = torch.device(device)
        u, group = union_csr(graphs)
        self.n, self.arcs, self.ngroups = u.n, u.arcs, len(graphs)
        self.ks = np.asarray(ks, dtype=np.uint32)
        self.kmask = 0
        for k in set(int(k) for k in ks):
            self.kmask |= 1 << k
        self.max_blocks = max_blocks
        self.opts = opts if opts is not None else (
            CountOpts(0, 0, 0, 0, 0, max_blocks, None, 0) if max_blocks else None)
        t = torch
        self.off = t.from_numpy(u.off.view(np.int64)).to(self.dev)
        self.cols = t.from_numpy(u.cols.view(np.int32)).to(self.dev)
        self.group = t.from_numpy(group.view(np.int32)).to(self.dev)
        self.group_k = t.from_numpy(self.ks.view(np.int32)).to(self.dev)
        self.counts = t.zeros(self.ngroups, dtype=t.int64, device=self.dev)
        self.ws = alloc_workspace(self.n, self.arcs, 1, device=self.dev)
        self.rank = t.empty(max(1, self.n), dtype=t.int32, device=self.dev)
        self.dag_off = t.empty(self.n + 1, dtype=t.int64, device=self.dev)
        self.dag_cols = t.empty(max(1, self.arcs // 2), dtype=t.int32, device=self.dev)
        self.build()
        if citron_workspace_bytes(self.n, self.arcs, self.max_outdeg) > self.ws.numel():
            self.ws = alloc_workspace(self.n, self.arcs, self.max_outdeg, device=self.dev)
        self.graph = None

    def build(self):
        """Degree ordering and relabelled DAG of the union (synchronises once for max_outdeg)."""
        citron_order(self.n, self.off, self.rank, None, self.ws)
        self.max_outdeg = citron_build_dag(self.n, self.off, self.cols, self.rank, self.dag_off,
                                           self.dag_cols, self.ws)

    def launch(self, stream=None):
        """Enqueue the batched count (asynchronous)."""
        citron_count_batch(self.n, self.dag_off, self.dag_cols, self.rank, self.group, self.group_k,
                           self.ngroups, self.kmask, self.max_outdeg, self.counts, self.ws, stream,
                           self.opts)

    def capture(self):
        """Record the batched count into a CUDA graph (after one warm-up launch)."""
        import torch

        self.launch()
        citron_workspace_status(self.ws)
        side = torch.cuda.Stream(device=self.dev)
        side.wait_stream(torch.cuda.current_stream(self.dev))
        with torch.cuda.stream(side):
            self.launch()
        torch.cuda.current_stream(self.dev).wait_stream(side)
        citron_workspace_status(self.ws)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, capture_error_mode="relaxed"):
            self.launch()
        return self.graph

    def replay(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()

    def result(self) -> list[int]:
        """Synchronise, check the device error word and return the per-graph counts."""
        citron_workspace_status(self.ws)
        return [int(x) for x in self.counts.cpu().numpy().view(np.uint64)]


# ---------------------------------------------------------------------------------------------
# Autotuner: picks the path thresholds for a batch by timing candidate plans on it.


def plan_opts(plan: dict, max_blocks: int = 0) -> CountOpts:
    return CountOpts(plan["small_max"], 0, plan["warps_per_cta"], 0, plan["compact_max"], max_blocks,
                     None, 0)

CANDIDATES = [
    dict(small_max=32, warps_per_cta=32, compact_max=0),
    dict(small_max=32, warps_per_cta=16, compact_max=0),
    dict(small_max=32, warps_per_cta=8, compact_max=0),
    dict(small_max=16, warps_per_cta=16, compact_max=0),
    dict(small_max=32, warps_per_cta=16, compact_max=1),
]


def tune(counter: BatchCounter, candidates=CANDIDATES, repeats: int = 2, cache: str | Path | None = None,
         key: str | None = None) -> dict:
    """Time each candidate plan on the batch (CUDA events, best of `repeats`) and keep the
    fastest in counter.opts.  With `cache` and `key`, a previous choice is reused and new ones
    are stored (JSON)."""
    import torch

    if cache and key:
        p = Path(cache)
        if p.exists():
            known = json.loads(p.read_text())
            if key in known:
                best = known[key]
                counter.opts = plan_opts(best, counter.max_blocks)
                counter.graph = None
                return dict(best, cached=True)
    results = []
    ref = None
    for cand in candidates:
        counter.opts = plan_opts(cand, counter.max_blocks)
        best_ms = float("inf")
        for _ in range(repeats):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            counter.launch()
            b.record()
            b.synchronize()
            best_ms = min(best_ms, a.elapsed_time(b))
        got = counter.result()
        if ref is None:
            ref = got
        elif got != ref:
            raise RuntimeError("tuning candidates disagree on the counts")
        results.append((best_ms, cand))
    best_ms, best = min(results, key=lambda r: r[0])
    counter.opts = plan_opts(best, counter.max_blocks)
    counter.graph = None
    out = dict(best, ms=best_ms, tried=[dict(c, ms=m) for m, c in results])
    if cache and key:
        p = Path(cache)
        known = json.loads(p.read_text()) if p.exists() else {}
        known[key] = dict(best)
        p.write_text(json.dumps(known, indent=1))
    return out


def time_replays(counter: BatchCounter, replays: int = 3) -> float:
    """Mean device time (ms) of graph replays of the batched count."""
    import torch

    counter.replay()
    counter.result()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(replays):
        counter.replay()
    b.record()
    b.synchronize()
    return a.elapsed_time(b) / replays
