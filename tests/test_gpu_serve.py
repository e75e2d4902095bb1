"""Serving with continuous batching: requests arriving over time are grouped into micro-batches
on several streams; every request's count is the same as when its graph is counted alone (and as
the oracle's), batches hold several requests, and several batches are in flight."""
import pytest

from paper_2112_10913_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


def test_results_same_alone_and_in_the_mix(gpu, oracle_lib):
    from paper_2112_10913_gb300.serve import Request, ServeConfig, ServeEngine, poisson_arrivals, summarize

    pool = gg.config4_batch(seed=5, count=36, n_range=(50, 2000))
    pool.append(gg.BatchItem(gg.config2_rmat(seed=5, scale=12, edge_factor=16), 5))
    pool.append(gg.BatchItem(gg.fig1(), 3))
    arrivals = poisson_arrivals(3000.0, len(pool), seed=5)
    reqs = [gg_req for gg_req in (Request(i, it.graph, it.k, arrival=float(a))
                                  for i, (it, a) in enumerate(zip(pool, arrivals)))]
    eng = ServeEngine(ServeConfig(slots=3, max_batch_requests=8))
    try:
        done = eng.run(reqs, timeout_s=300)
    finally:
        eng.close()
    for r in done:
        alone = gpu.DeviceGraph(r.graph).count(r.k)
        assert r.count == alone == oracle_lib.count_graph(r.graph, r.k), r.rid
    batches = {}
    for r in done:
        batches.setdefault(r.batch, []).append(r)
    assert len(batches) > 1 and max(len(b) for b in batches.values()) > 1
    s = summarize(done)
    assert s["requests"] == len(pool) and s["p99_ms"] >= s["p50_ms"] > 0


def test_admission_respects_the_memory_budget(gpu):
    from paper_2112_10913_gb300.serve import Request, ServeConfig, ServeEngine, footprint_bytes

    graphs = [gg.small_er(i, 800, 12.0) for i in range(6)]
    arcs = max(g.arcs for g in graphs)
    one = footprint_bytes(800, arcs)
    extra = footprint_bytes(1600, 2 * arcs) - one
    # a budget that admits one request at a time: micro-batches of one, served one after another
    eng = ServeEngine(ServeConfig(slots=3, max_batch_requests=8, hbm_budget_bytes=one + extra // 2))
    try:
        done = eng.run([Request(i, g, 4, arrival=0.0) for i, g in enumerate(graphs)], timeout_s=120)
    finally:
        eng.close()
    assert len({r.batch for r in done}) == len(graphs)
    assert all(r.count == gpu.DeviceGraph(r.graph).count(4) for r in done)


def test_heavy_lane_and_capped_launches(gpu, oracle_lib):
    """Requests above the arc threshold are served in the heavy lane (a stream of their own with
    counting launches capped at part of the SMs) and still give the counts of the graph alone."""
    import torch

    from paper_2112_10913_gb300.serve import Request, ServeConfig, ServeEngine

    big = gg.config2_rmat(seed=7, scale=13, edge_factor=16)
    pool = [gg.BatchItem(big, 5)] + gg.config4_batch(seed=9, count=12, n_range=(50, 1500))
    pool.append(gg.BatchItem(big, 4))
    reqs = [Request(i, it.graph, it.k, arrival=0.001 * i) for i, it in enumerate(pool)]
    eng = ServeEngine(ServeConfig(slots=2, max_batch_requests=4, heavy_arcs=big.arcs,
                                  heavy_sm_fraction=0.25))
    try:
        assert eng.heavy_max_blocks == max(1, int(torch.cuda.get_device_properties(0).multi_processor_count * 0.25))
        done = eng.run(reqs, timeout_s=300)
    finally:
        eng.close()
    heavy_batches = {r.batch for r in done if r.graph is big}
    light_batches = {r.batch for r in done if r.graph is not big}
    assert heavy_batches and not heavy_batches & light_batches
    for r in done:
        assert r.count == gpu.DeviceGraph(r.graph).count(r.k) == oracle_lib.count_graph(r.graph, r.k), r.rid


def test_block_cap_keeps_counts(gpu):
    """citron_count_opts.max_blocks caps the grid of every counting path; the counts stay exact."""
    g = gg.config2_rmat(seed=3, scale=14, edge_factor=16)
    dg = gpu.DeviceGraph(g)
    for k in (3, 5, 7):
        want = dg.count(k)
        # one block alone at k = 7 runs for minutes on the sorted-list path: capped at 7 and 40
        for cap in ((1, 7, 40) if k < 7 else (7, 40)):
            assert dg.count(k, max_blocks=cap) == want, (k, cap)
            assert dg.count(k, max_blocks=cap, small_max=8, bitmap_max=64) == want, (k, cap)


def test_repeat_queries_use_the_device_cache(gpu, oracle_lib):
    """A graph queried again (another k) is served from its DAG kept on the device: no upload, no
    ordering; the counts equal the graph counted alone.  The cache never exceeds its bytes."""
    from paper_2112_10913_gb300.serve import Request, ServeConfig, ServeEngine

    pool = gg.config4_batch(seed=21, count=10, n_range=(60, 1500))
    first = [Request(i, it.graph, 3, arrival=0.0) for i, it in enumerate(pool)]
    again = [Request(100 + i, it.graph, 3 + i % 4, arrival=0.05) for i, it in enumerate(pool)]
    eng = ServeEngine(ServeConfig(slots=2, max_batch_requests=4, cache_bytes=256 << 20))
    try:
        done1 = eng.run(first, timeout_s=120)
        done2 = eng.run(again, timeout_s=120)
    finally:
        eng.close()
    assert not any(r.cached for r in done1)
    assert all(r.cached for r in done2)
    assert eng.cache.hits == len(again) and eng.cache.bytes <= 256 << 20
    for r in done1 + done2:
        assert r.count == gpu.DeviceGraph(r.graph).count(r.k) == oracle_lib.count_graph(r.graph, r.k), r.rid
