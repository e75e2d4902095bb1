"""Host logic of the serving engine, on the CPU: lanes, FIFO micro-batches bounded by request
count and arcs, admission by the HBM-footprint budget, and every request answered once.  The
CUDA pieces (streams, device selection) are replaced by stand-ins and each micro-batch is
counted by the oracle, so no GPU is needed."""
import contextlib
import threading
import time

import pytest
import torch

import oracle
from paper_2112_10913_gb300 import graphgen as gg


class _FakeStream:
    def __init__(self, device=None, priority=0):
        self.priority = priority


class _Props:
    multi_processor_count = 152


@pytest.fixture
def engine_cls(monkeypatch):
    monkeypatch.setattr(torch.cuda, "Stream", _FakeStream)
    monkeypatch.setattr(torch.cuda, "set_device", lambda d: None)
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda d: _Props())
    from paper_2112_10913_gb300 import serve

    class Recording(serve.ServeEngine):
        def __init__(self, *a, **kw):
            self.seen = []
            self.max_bytes = 0
            self.rec_lock = threading.Lock()
            super().__init__(*a, **kw)

        def _run_batch(self, batch, stream, max_blocks=0, **kw):
            with self.rec_lock:
                self.seen.append(([r.rid for r in batch], stream.priority, max_blocks))
                self.max_bytes = max(self.max_bytes, self.in_flight_bytes)
            time.sleep(0.002)
            return [oracle.count_graph(r.graph, r.k, threads=1) for r in batch]

    return serve, Recording


def test_lanes_batches_and_answers(engine_cls):
    serve, Recording = engine_cls
    light = [gg.small_er(i, 300, 6.0) for i in range(30)]
    heavy = gg.small_rmat(99, 3000, 30.0)
    reqs = [serve.Request(i, g, 3 + i % 3, arrival=0.0005 * i) for i, g in enumerate(light)]
    reqs += [serve.Request(100 + j, heavy, 4, arrival=0.004 * j) for j in range(3)]
    cfg = serve.ServeConfig(slots=2, max_batch_requests=4, heavy_arcs=heavy.arcs, heavy_slots=1,
                            heavy_sm_fraction=0.5, cache_bytes=0)
    eng = Recording(cfg, device="cuda:0")
    try:
        done = eng.run(reqs, timeout_s=60)
    finally:
        eng.close()
    assert eng.heavy_max_blocks == 76
    assert sorted(r.rid for r in done) == sorted(r.rid for r in reqs)
    for r in done:
        assert r.count == oracle.count_graph(r.graph, r.k, threads=1)
        assert r.done >= r.admitted >= r.arrival - 1e-9
    by_rid = {r.rid: r for r in done}
    for rids, prio, mb in eng.seen:
        assert 1 <= len(rids) <= 4
        kinds = {by_rid[i].heavy for i in rids}
        assert len(kinds) == 1  # a micro-batch never mixes the lanes
        if kinds == {True}:
            assert prio == 0 and mb == 76
        else:
            assert prio == -1 and mb == 0
    # FIFO within each lane: micro-batches are numbered as they are admitted, and a later
    # arrival never lands in an earlier micro-batch (slots may still finish out of order)
    for heavy_lane in (False, True):
        lane_reqs = sorted((r for r in done if r.heavy == heavy_lane), key=lambda r: r.arrival)
        ids = [r.batch for r in lane_reqs]
        assert ids == sorted(ids)
    s = serve.summarize(done)
    assert s["requests"] == len(reqs) and "light" in s and "heavy" in s


def test_admission_keeps_the_footprint_under_budget(engine_cls):
    serve, Recording = engine_cls
    graphs = [gg.small_er(i, 400, 8.0) for i in range(8)]
    arcs = max(g.arcs for g in graphs)
    one = serve.footprint_bytes(400, arcs)
    extra = serve.footprint_bytes(800, 2 * arcs) - one
    budget = one + extra // 2  # room for one request in flight, never two
    cfg = serve.ServeConfig(slots=3, max_batch_requests=8, hbm_budget_bytes=budget, heavy_arcs=0,
                            cache_bytes=0)
    eng = Recording(cfg, device="cuda:0")
    try:
        done = eng.run([serve.Request(i, g, 3, arrival=0.0) for i, g in enumerate(graphs)],
                       timeout_s=60)
    finally:
        eng.close()
    assert eng.max_bytes <= budget
    assert len({r.batch for r in done}) == len(graphs)  # admitted one by one
    assert eng.heavy_slots == []


def test_slot_handoff_never_loses_a_request(engine_cls):
    """A slot returns to the free list only once it is idle: with one slot and many one-request
    micro-batches handed over back to back, every request is answered.  The release is slowed
    down so that the dispatcher hands over the next micro-batch while the slot's thread is still
    inside it: a slot that clears its work after the release loses that micro-batch."""
    serve, _ = engine_cls

    class Instant(serve.ServeEngine):
        def _run_batch(self, batch, stream, max_blocks=0, **kw):
            return [r.k for r in batch]

        def _release(self, slot, batch):
            super()._release(slot, batch)
            time.sleep(0.001)

    g = gg.fig1()
    reqs = [serve.Request(i, g, 3, arrival=0.0) for i in range(2000)]
    eng = Instant(serve.ServeConfig(slots=1, max_batch_requests=1, heavy_arcs=0, poll_s=0.0),
                  device="cuda:0")
    try:
        done = eng.run(reqs, timeout_s=60)
    finally:
        eng.close()
    assert len(done) == len(reqs) and all(r.count == 3 for r in done)
    assert len({r.batch for r in done}) == len(reqs)


def test_dag_cache_ring_keeps_what_is_in_use():
    """The cache's ring of DAGs: new entries push out the ones they overlap, least recently
    written first, never one that a micro-batch in flight still reads, and never more bytes
    than its capacity."""
    from paper_2112_10913_gb300.serve import DagCache

    c = DagCache(4096, device="cpu")
    def add(key, n, arcs):
        room = c.reserve(key, n, arcs)
        if room is None:
            return False
        off, cols, start, nbytes = room
        assert off.numel() == n + 1 and cols.numel() == max(1, arcs)
        c.commit(key, (n, arcs, 0, off, cols), start, nbytes)
        return True

    assert add("a", 100, 200)       # 1,808 bytes -> 2,048
    assert add("b", 100, 200)       # fills the ring
    assert not add("a", 100, 200)   # cached already
    assert c.get("a")[0] == 100     # "a" is now in use
    assert not add("c", 100, 200)   # its room (the start of the ring) holds "a", in use
    c.release("a")
    assert add("c", 100, 200)       # pushes out "a"
    assert c.get("a") is None and c.get("b") is not None and c.get("c") is not None
    c.release("b")
    c.release("c")
    assert c.bytes <= 4096
    assert c.reserve("huge", 10000, 10000) is None
