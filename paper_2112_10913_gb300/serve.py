"""Serving: a request loop over (graph, k) queries with continuous batching.

Requests arrive over time.  A dispatcher groups the requests waiting in the queue into
micro-batches (FIFO, bounded by request count and arcs), admits a micro-batch only when a slot is
free and its estimated device footprint fits the HBM budget, and hands it to a slot.  Each slot
owns a CUDA stream and a host thread: it uploads the micro-batch as one union CSR, builds the
ordering and DAG and runs the batched count (``citron_count_batch``), all on its stream, so the
work of different slots overlaps on the device; a slot takes new work as soon as it finishes.
Requests that arrive while others are on the GPU join the next micro-batch of the next free slot.

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
from dataclasses import dataclass, field

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

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def footprint_bytes(n: int, arcs: int) -> int:
    """Device bytes a micro-batch holds: CSR, rank, DAG, kept-row buffers and counting lists."""
    return int(8 * (n + 1) * 3 + 4 * arcs * 2 + 4 * n * 8 + (64 << 20))


@dataclass
class ServeConfig:
    slots: int = 4                    # light micro-batches in flight (one stream each)
    max_batch_requests: int = 64
    max_batch_arcs: int = 16 << 20
    hbm_budget_bytes: int = 64 << 30
    poll_s: float = 0.0002
    heavy_arcs: int = 1 << 22         # requests with at least this many arcs use the heavy lane (0: no lane)
    heavy_slots: int = 1
    heavy_sm_fraction: float = 0.75   # share of the SMs a heavy counting launch may hold


class _Slot:
    def __init__(self, engine: "ServeEngine", index: int, heavy: bool = False):
        import torch

        self.engine = engine
        self.index = index
        self.heavy = heavy
        # lower numbers are higher priorities; 0 is the default (lowest) one
        self.stream = torch.cuda.Stream(device=engine.device, priority=0 if heavy else -1)
        self.max_blocks = engine.heavy_max_blocks if heavy else 0
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
                    counts = self.engine._run_batch(batch, self.stream, self.max_blocks)
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
        self.slots = [_Slot(self, i) for i in range(self.cfg.slots)]
        self.heavy_slots = ([_Slot(self, self.cfg.slots + i, heavy=True)
                             for i in range(self.cfg.heavy_slots)] if self.cfg.heavy_arcs else [])
        self.free = list(self.slots)
        self.heavy_free = list(self.heavy_slots)

    def now(self) -> float:
        return time.perf_counter() - self.t0

    # -- the work of one micro-batch (runs on the slot's thread and stream) --------------------
    def _run_batch(self, batch: list[Request], stream, max_blocks: int = 0) -> list[int]:
        from .batch import BatchCounter

        bc = BatchCounter([r.graph for r in batch], [r.k for r in batch], device=self.device,
                          max_blocks=max_blocks)
        bc.launch(stream)
        return bc.result()

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
        """FIFO micro-batch from one lane's queue head, bounded by count, arcs and the HBM budget."""
        queue, free = (self.heavy_queue, self.heavy_free) if heavy else (self.queue, self.free)
        with self.lock:
            if not queue or not free:
                return []
            batch, n, arcs = [], 0, 0
            while queue and len(batch) < self.cfg.max_batch_requests:
                r = queue[0]
                if batch and arcs + r.graph.arcs > self.cfg.max_batch_arcs:
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
               batches=len(set(r.batch for r in done)))
    for name, rs in (("light", [r for r in done if not r.heavy]), ("heavy", [r for r in done if r.heavy])):
        if rs:
            out[name] = _lat(rs)
    return out
