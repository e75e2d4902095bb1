"""Serving: a request loop over (graph, k) queries with continuous batching.

Requests arrive over time.  A dispatcher groups the requests waiting in the queue into
micro-batches (FIFO, bounded by request count, vertices and arcs), admits a micro-batch only when
a slot is free and its estimated device footprint fits the HBM budget, and hands it to a slot.
Each slot owns a CUDA stream, a host thread and an arena: device buffers and pinned host staging
buffers sized once for the largest micro-batch, so that no micro-batch allocates.  Requests that
arrive while others are on the GPU join the next micro-batch of the next free slot; the work of
different slots overlaps on the device.

State stays resident: the relabelled DAG of every graph counted recently is kept on the device
(``DagCache``, least recently used out first, bounded in bytes).  A micro-batch uploads, orders
(``citron_order_grouped``: every graph in its own degree order, graph after graph) and
directionalises only the graphs it has not seen; the DAGs of the others are copied into the
micro-batch's union DAG from the cache (``citron_dag_append``), and one batched count
(``citron_count_batch``) answers every request, each with its own k.

Large requests (at least ``heavy_arcs`` arcs) take a separate lane: their own queue and slot, a
low-priority stream, and counting launches capped at part of the SMs (``citron_count_opts``
max_blocks).  The counting kernels are persistent (one block per SM taking roots from a shared
counter), so an uncapped heavy launch would hold every SM until it ends and the small requests
queued behind it would wait for its whole run; with the cap the light lane keeps the remaining
SMs, on high-priority streams.

Every step of the counting runs in the CUDA library; this module only schedules and marshals.
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass

import numpy as np

from .graphgen import Csr


@dataclass
class Request:
    rid: int
    graph: Csr
    k: int
    arrival: float = 0.0       # seconds since the start of the run
    admitted: float = -1.0
    done: float = -1.0
    count: int | None = None
    batch: int = -1            # micro-batch it was served in
    heavy: bool = False        # served in the heavy lane
    cached: bool = False       # its graph's DAG came from the device cache
    key: object = None         # graph identity for the cache (default: the graph object)

    @property
    def latency(self) -> float:
        return self.done - self.arrival

    @property
    def graph_key(self):
        return self.key if self.key is not None else id(self.graph)


def footprint_bytes(n: int, arcs: int) -> int:
    """Device bytes a micro-batch uses: CSR, rank, DAG, kept-row buffers and counting lists."""
    return int(8 * (n + 1) * 3 + 4 * arcs * 2 + 4 * n * 8 + (64 << 20))


@dataclass
class ServeConfig:
    slots: int = 4                    # light micro-batches in flight (one stream each)
    max_batch_requests: int = 64
    max_batch_arcs: int = 16 << 20
    max_batch_vertices: int = 4 << 20
    hbm_budget_bytes: int = 64 << 30
    poll_s: float = 0.0002
    heavy_arcs: int = 1 << 22         # requests with at least this many arcs use the heavy lane (0: no lane)
    heavy_slots: int = 1
    heavy_sm_fraction: float = 0.75   # share of the SMs a heavy counting launch may hold
    cache_bytes: int = 8 << 30        # device bytes of cached DAGs (0: no cache)
    max_outdeg_cap: int = 4096        # the arenas' workspaces cover DAG rows up to this length


class DagCache:
    """Relabelled DAGs of graphs counted before, on the device: key -> (n, arcs, max_outdeg,
    dag_off (n+1, from 0), dag_cols (ranks 0..n-1)), the oldest stored out first.

    The DAGs live in one device buffer allocated once (a ring: new DAGs go after the last one,
    wrapping around to the start and pushing out the DAGs they overlap, i.e. the ones stored
    longest ago), so that caching never calls the device allocator, which would synchronise the
    device under the other slots' work.
    A DAG that a micro-batch in flight still reads is never overwritten: the new one is then not
    kept."""

    def __init__(self, capacity_bytes: int, device=None):
        self.capacity = capacity_bytes
        self.device = device
        self.buf = None  # uint8 device buffer, allocated on first use
        self.head = 0
        self.bytes = 0
        self.entries: collections.OrderedDict = collections.OrderedDict()  # key -> (entry, start, nbytes)
        self.in_use: collections.Counter = collections.Counter()
        self.lock = threading.Lock()
        self.hits = self.misses = 0

    def get(self, key):
        """The entry of key (marked in use until release(key)), or None."""
        with self.lock:
            e = self.entries.get(key)
            if e is None:
                return None
            self.in_use[key] += 1
            return e[0]

    def release(self, key):
        with self.lock:
            self.in_use[key] -= 1
            if self.in_use[key] <= 0:
                del self.in_use[key]

    def reserve(self, key, n: int, arcs: int):
        """Device storage (dag_off, dag_cols) for a new entry, or None when the key is cached
        already or the room it needs is in use.  The entry is readable after commit()."""
        import torch

        nbytes = (8 * (n + 1) + 4 * max(1, arcs) + 255) // 256 * 256
        if nbytes > self.capacity:
            return None
        with self.lock:
            if key in self.entries:
                return None
            if self.buf is None:
                self.buf = torch.empty(self.capacity, dtype=torch.uint8, device=self.device)
            start = self.head if self.head + nbytes <= self.capacity else 0
            end = start + nbytes
            clash = [k for k, (_, s0, nb) in self.entries.items() if s0 < end and start < s0 + nb]
            if any(self.in_use.get(k) for k in clash):
                return None
            for k in clash:
                self.bytes -= self.entries.pop(k)[2]
            self.head = end
            region = self.buf[start:end]
            off = region[: 8 * (n + 1)].view(torch.int64)
            cols = region[8 * (n + 1): 8 * (n + 1) + 4 * max(1, arcs)].view(torch.int32)
            return off, cols, start, nbytes

    def commit(self, key, entry, start: int, nbytes: int):
        with self.lock:
            self.entries[key] = (entry, start, nbytes)
            self.bytes += nbytes


class SlotArena:
    """Device buffers and pinned host staging of one slot, sized for the largest micro-batch."""

    def __init__(self, device, max_n: int, max_arcs: int, max_groups: int, max_outdeg_cap: int):
        import torch

        from . import alloc_workspace

        d, t = device, torch
        self.max_n, self.max_arcs, self.max_groups = max_n, max_arcs, max_groups
        self.off = t.empty(max_n + 1, dtype=t.int64, device=d)
        self.cols = t.empty(max(1, max_arcs), dtype=t.int32, device=d)
        self.group = t.empty(max(1, max_n), dtype=t.int32, device=d)
        self.rank = t.empty(max(1, max_n), dtype=t.int32, device=d)
        self.dag_off = t.empty(max_n + 1, dtype=t.int64, device=d)
        self.dag_cols = t.empty(max(1, max_arcs // 2), dtype=t.int32, device=d)
        self.group_k = t.empty(max_groups, dtype=t.int32, device=d)
        self.counts = t.empty(max_groups, dtype=t.int64, device=d)
        self.ws = alloc_workspace(max_n, max_arcs, max_outdeg_cap, device=d)
        pin = dict(pin_memory=True)
        self.h_off = t.empty(max_n + 1, dtype=t.int64, **pin)
        self.h_cols = t.empty(max(1, max_arcs), dtype=t.int32, **pin)
        self.h_group = t.empty(max(1, max_n), dtype=t.int32, **pin)
        self.h_k = t.empty(max_groups, dtype=t.int32, **pin)
        self.h_counts = t.empty(max_groups, dtype=t.int64, **pin)

    def fits(self, n: int, arcs: int, groups: int) -> bool:
        return n <= self.max_n and arcs <= self.max_arcs and groups <= self.max_groups


class _Slot:
    def __init__(self, engine: "ServeEngine", index: int, heavy: bool = False):
        import torch

        self.engine = engine
        self.index = index
        self.heavy = heavy
        # lower numbers are higher priorities; 0 is the default (lowest) one
        self.stream = torch.cuda.Stream(device=engine.device, priority=0 if heavy else -1)
        self.max_blocks = engine.heavy_max_blocks if heavy else 0
        self.arena = None  # created on first use, on the slot's thread
        self.work: list[Request] | None = None
        self.cv = threading.Condition()
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.thread.start()

    def _loop(self):
        import torch

        try:
            torch.cuda.set_device(self.engine.device)
        except Exception as exc:  # reported by the engine's run loop
            self.engine.errors.append(exc)
            return
        while True:
            with self.cv:
                while self.work is None:
                    self.cv.wait()
                batch = self.work
            if batch == []:
                return
            try:
                with torch.cuda.stream(self.stream):
                    counts = self.engine._run_batch(batch, self.stream, self.max_blocks, slot=self)
                now = self.engine.now()
                for r, c in zip(batch, counts):
                    r.count, r.done = c, now
            except Exception as exc:  # reported by the engine, never swallowed
                self.engine.errors.append(exc)
                now = self.engine.now()
                for r in batch:
                    r.done = now
            # the slot must be idle before it goes back on the free list: once released, the
            # dispatcher may hand it the next micro-batch at any moment
            with self.cv:
                self.work = None
            self.engine._release(self, batch)

    def give(self, batch: list[Request]):
        with self.cv:
            self.work = batch
            self.cv.notify()


class ServeEngine:
    def __init__(self, config: ServeConfig | None = None, device="cuda"):
        import torch

        self.cfg = config or ServeConfig()
        dev = torch.device(device)
        self.device = dev if dev.index is not None else torch.device(dev.type, torch.cuda.current_device())
        sms = torch.cuda.get_device_properties(self.device).multi_processor_count
        self.heavy_max_blocks = max(1, int(sms * self.cfg.heavy_sm_fraction))
        self.queue: collections.deque[Request] = collections.deque()
        self.heavy_queue: collections.deque[Request] = collections.deque()
        self.lock = threading.Lock()
        self.in_flight_bytes = 0
        self.errors: list[Exception] = []
        self.t0 = time.perf_counter()
        self.batches = 0
        self.cache = DagCache(self.cfg.cache_bytes, self.device) if self.cfg.cache_bytes else None
        self.phase_ms = collections.defaultdict(float)  # host time per phase, all micro-batches
        self.slots = [_Slot(self, i) for i in range(self.cfg.slots)]
        self.heavy_slots = ([_Slot(self, self.cfg.slots + i, heavy=True)
                             for i in range(self.cfg.heavy_slots)] if self.cfg.heavy_arcs else [])
        self.free = list(self.slots)
        self.heavy_free = list(self.heavy_slots)

    def now(self) -> float:
        return time.perf_counter() - self.t0

    # -- the work of one micro-batch (runs on the slot's thread and stream) --------------------
    def _arena(self, slot: _Slot, n: int, arcs: int, groups: int) -> SlotArena:
        cfg = self.cfg
        if slot.arena is None or not slot.arena.fits(n, arcs, groups):
            slot.arena = None
            slot.arena = SlotArena(self.device, max(cfg.max_batch_vertices, n), max(cfg.max_batch_arcs, arcs),
                                   max(cfg.max_batch_requests, groups), cfg.max_outdeg_cap)
        return slot.arena

    def _run_batch(self, batch: list[Request], stream, max_blocks: int = 0, slot: _Slot | None = None) -> list[int]:
        from . import (CountOpts, citron_build_dag, citron_count_batch, citron_dag_append,
                       citron_order_grouped, citron_workspace_bytes)

        t0 = time.perf_counter()
        cache = self.cache
        entries = [cache.get(r.graph_key) if cache else None for r in batch]
        miss = [i for i, e in enumerate(entries) if e is None]
        hit = [i for i, e in enumerate(entries) if e is not None]
        for i in hit:
            batch[i].cached = True
        if cache:
            cache.hits += len(hit)
            cache.misses += len(miss)
        n_miss = sum(batch[i].graph.n for i in miss)
        arcs_miss = sum(batch[i].graph.arcs for i in miss)
        n_all = n_miss + sum(entries[i][0] for i in hit)
        dag_arcs = arcs_miss // 2 + sum(entries[i][1] for i in hit)
        a = self._arena(slot, n_all, max(arcs_miss, 2 * dag_arcs), len(batch))
        # union CSR of the graphs not seen before, staged in pinned memory
        h_off = a.h_off.numpy().view(np.uint64)
        h_cols = a.h_cols.numpy().view(np.uint32)
        h_group = a.h_group.numpy().view(np.uint32)
        h_off[0] = 0
        vb = ab = 0
        for gi, i in enumerate(miss):
            g = batch[i].graph
            np.add(g.off[1:], np.uint64(ab), out=h_off[vb + 1: vb + g.n + 1])
            np.add(g.cols, np.uint32(vb), out=h_cols[ab: ab + g.arcs])
            h_group[vb: vb + g.n] = gi
            vb += g.n
            ab += g.arcs
        t1 = time.perf_counter()
        max_outdeg = 0
        if n_miss:
            a.off[: n_miss + 1].copy_(a.h_off[: n_miss + 1], non_blocking=True)
            if arcs_miss:
                a.cols[:arcs_miss].copy_(a.h_cols[:arcs_miss], non_blocking=True)
            a.group[:n_miss].copy_(a.h_group[:n_miss], non_blocking=True)
            citron_order_grouped(n_miss, a.off, a.group, len(miss), a.rank, None, a.ws, stream)
            # the arc count is taken from the columns' length: pass exactly this batch's arcs
            max_outdeg = citron_build_dag(n_miss, a.off, a.cols[:arcs_miss], a.rank, a.dag_off, a.dag_cols,
                                          a.ws, stream)
        else:
            a.dag_off[:1].zero_()
        t2 = time.perf_counter()
        # the cached DAGs follow, each copied to its place in the union DAG
        order = miss + hit
        vb, ab = n_miss, arcs_miss // 2
        for i in hit:
            n, arcs, mx, e_off, e_cols = entries[i][:5]
            citron_dag_append(n, e_off, e_cols, 0, a.dag_off[vb: vb + n + 1], a.dag_cols, vb, ab, stream)
            max_outdeg = max(max_outdeg, mx)
            vb += n
            ab += arcs
        # the graph of every union row (rows of the new graphs hold it already: rank space keeps
        # each graph's rows together, in union order), and every graph's k
        if hit:
            sizes = np.array([entries[i][0] for i in hit], dtype=np.int64)
            h_group[n_miss:n_all] = np.repeat(np.arange(len(miss), len(order), dtype=np.uint32), sizes)
            a.group[n_miss:n_all].copy_(a.h_group[n_miss:n_all], non_blocking=True)
        hk = a.h_k.numpy().view(np.uint32)
        hk[: len(order)] = [batch[i].k for i in order]
        a.group_k[: len(order)].copy_(a.h_k[: len(order)], non_blocking=True)
        kmask = 0
        for i in order:
            kmask |= 1 << batch[i].k
        if max_outdeg > self.cfg.max_outdeg_cap and citron_workspace_bytes(n_all, 2 * ab, max_outdeg) > a.ws.numel():
            raise RuntimeError("a DAG row exceeds the serving arena's workspace bound")
        opts = CountOpts(0, 0, 0, 0, 0, max_blocks, None, 0) if max_blocks else None
        citron_count_batch(n_all, a.dag_off, a.dag_cols, None, a.group, a.group_k, len(order), kmask,
                           max_outdeg, a.counts, a.ws, stream, opts)
        a.h_counts[: len(order)].copy_(a.counts[: len(order)], non_blocking=True)
        # keep the new graphs' DAGs (cut out of the union) for later requests; they become
        # visible once the stream has finished the copies, so that other slots never see them early
        new_entries = []
        if cache:
            vb = 0
            for i in miss:
                g = batch[i].graph
                m = int(g.arcs // 2)
                room = cache.reserve(batch[i].graph_key, g.n, m)
                if room is not None:
                    e_off, e_cols, start, nbytes = room
                    citron_dag_append(g.n, a.dag_off[vb: vb + g.n + 1], a.dag_cols, vb, e_off, e_cols, 0, 0, stream)
                    new_entries.append((batch[i].graph_key, (g.n, m, max_outdeg, e_off, e_cols), start, nbytes))
                vb += g.n
        t3 = time.perf_counter()
        from . import citron_workspace_status

        try:
            citron_workspace_status(a.ws, stream)  # synchronises the stream, reports device errors
        finally:
            if cache:
                for i in hit:
                    cache.release(batch[i].graph_key)
        for key, entry, start, nbytes in new_entries:
            cache.commit(key, entry, start, nbytes)
        got = a.h_counts.numpy().view(np.uint64)[: len(order)]
        counts = [0] * len(batch)
        for j, i in enumerate(order):
            counts[i] = int(got[j])
        t4 = time.perf_counter()
        ph = self.phase_ms
        ph["assemble"] += (t1 - t0) * 1e3
        ph["order_dag"] += (t2 - t1) * 1e3
        ph["enqueue_count"] += (t3 - t2) * 1e3
        ph["wait"] += (t4 - t3) * 1e3
        return counts

    def _release(self, slot: _Slot, batch: list[Request]):
        with self.lock:
            self.in_flight_bytes -= sum(getattr(r, "_bytes", 0) for r in batch[:1])
            (self.heavy_free if slot.heavy else self.free).append(slot)

    # -- scheduling ------------------------------------------------------------------------------
    def is_heavy(self, r: Request) -> bool:
        return bool(self.cfg.heavy_arcs) and r.graph.arcs >= self.cfg.heavy_arcs

    def submit(self, r: Request):
        r.heavy = self.is_heavy(r)
        with self.lock:
            (self.heavy_queue if r.heavy else self.queue).append(r)

    def _take_batch(self, heavy: bool = False) -> list[Request]:
        """FIFO micro-batch from one lane's queue head, bounded by count, vertices, arcs and the
        HBM budget."""
        queue, free = (self.heavy_queue, self.heavy_free) if heavy else (self.queue, self.free)
        with self.lock:
            if not queue or not free:
                return []
            batch, n, arcs = [], 0, 0
            while queue and len(batch) < self.cfg.max_batch_requests:
                r = queue[0]
                if batch and (arcs + r.graph.arcs > self.cfg.max_batch_arcs
                              or n + r.graph.n > self.cfg.max_batch_vertices):
                    break
                fp = footprint_bytes(n + r.graph.n, arcs + r.graph.arcs)
                if self.in_flight_bytes + fp > self.cfg.hbm_budget_bytes and (batch or self.in_flight_bytes):
                    break  # wait for memory to free up
                batch.append(queue.popleft())
                n += r.graph.n
                arcs += r.graph.arcs
            if not batch:
                return []
            fp = footprint_bytes(n, arcs)
            batch[0]._bytes = fp
            self.in_flight_bytes += fp
            slot = free.pop()
        now = self.now()
        for r in batch:
            r.admitted = now
            r.batch = self.batches
        self.batches += 1
        slot.give(batch)
        return batch

    def run(self, requests: list[Request], timeout_s: float = 600.0) -> list[Request]:
        """Feed the requests at their arrival times and serve them; returns them completed."""
        self.t0 = time.perf_counter()
        pending = sorted(requests, key=lambda r: r.arrival)
        i = 0
        deadline = time.perf_counter() + timeout_s
        while True:
            now = self.now()
            while i < len(pending) and pending[i].arrival <= now:
                self.submit(pending[i])
                i += 1
            while self._take_batch(heavy=False):
                pass
            while self._take_batch(heavy=True):
                pass
            if self.errors:
                raise self.errors[0]
            if i == len(pending) and all(r.done >= 0 for r in pending):
                break
            if time.perf_counter() > deadline:
                raise TimeoutError("serving run exceeded its time limit")
            time.sleep(self.cfg.poll_s)
        if self.errors:
            raise self.errors[0]
        return pending

    def close(self):
        for s in self.slots + self.heavy_slots:
            s.give([])
        for s in self.slots + self.heavy_slots:
            s.thread.join(timeout=10)


def poisson_arrivals(rate: float, count: int, seed: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process: exponential gaps from seeded uniforms."""
    from .graphgen import uniform

    u = uniform(seed, 77, count)
    gaps = -np.log1p(-u) / rate
    return np.cumsum(gaps)


def _lat(rs: list[Request]) -> dict:
    lat = np.array([r.latency for r in rs]) * 1e3
    wait = np.array([r.admitted - r.arrival for r in rs]) * 1e3
    return dict(requests=len(rs), p50_ms=float(np.percentile(lat, 50)),
                p99_ms=float(np.percentile(lat, 99)), mean_ms=float(lat.mean()),
                queue_p50_ms=float(np.percentile(wait, 50)))


def summarize(done: list[Request]) -> dict:
    """Latency percentiles (all requests and per lane), queueing share and achieved requests/s."""
    span = max(r.done for r in done) - min(r.arrival for r in done)
    out = _lat(done)
    out.update(req_per_s=len(done) / span if span > 0 else float("inf"),
               batches=len(set(r.batch for r in done)),
               cached=sum(1 for r in done if r.cached))
    for name, rs in (("light", [r for r in done if not r.heavy]), ("heavy", [r for r in done if r.heavy])):
        if rs:
            out[name] = _lat(rs)
    return out
