"""Error paths on the GPU, with faults injected from the host (citron_set_faults): no kernel is
broken and nothing faults the GPU.

- a look-back tile that never publishes its prefix: the next tile's bounded wait runs out and the
  call returns CITRON_E_TIMEOUT, with no hang; the next call, without the fault, is exact;
- a block of the core ordering that never arrives at the first grid barrier: the other blocks'
  bounded wait runs out (CITRON_E_TIMEOUT), the next call is exact;
- device totals seeded near 2^64: a count that carries them past 2^64 - 1 reports
  CITRON_E_OVERFLOW (single count, no-allocation count, batched count through the workspace
  status), while a count that ends exactly at 2^64 - 1 does not.
"""
import ctypes

import numpy as np
import pytest

from paper_2112_10913_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu
U64_MAX = (1 << 64) - 1


@pytest.fixture
def faults(gpu):
    yield gpu.citron_set_faults
    gpu.citron_set_faults()  # always restore normal operation


def _status(exc):
    return exc.value.name


def test_lookback_stall_times_out_then_recovers(gpu, faults, oracle_lib):
    import torch

    g = gg.small_rmat(31, 20000, 24.0)
    # at least four look-back tiles in every look-back pass: the GenOrdering compaction (4096 arcs
    # per tile) and the row-offset scan of the relabelled DAG (4096 rows per tile)
    assert g.arcs > 4 * 4096 and g.n > 4 * 4096
    G = gpu.DeviceGraph(g, relabel=False)
    dag_off = torch.empty_like(G.dag_off)
    dag_cols = torch.empty_like(G.dag_cols)
    want_off, want_cols = oracle_lib.gen_ordering(g.off, g.cols, g.n)
    for relabel in (False, True):
        rank = None
        if relabel:
            rank = torch.empty(g.n, dtype=torch.int32, device="cuda")
            gpu.citron_order(g.n, G.off, rank, None, G.ws)
        faults(lookback_spin_limit=2000, lookback_stall_tile=1)
        with pytest.raises(gpu.CitronError) as e:
            gpu.citron_build_dag(g.n, G.off, G.cols, rank, dag_off, dag_cols, G.ws)
        assert _status(e) == "CITRON_E_TIMEOUT"
        faults()
        gpu.citron_build_dag(g.n, G.off, G.cols, rank, dag_off, dag_cols, G.ws)
        if relabel:
            want_off, want_cols = oracle_lib.dag_by_rank(g.off, g.cols, g.n,
                                                         rank.cpu().numpy().view(np.uint32), True)
        m = int(want_off[-1])
        assert np.array_equal(dag_off.cpu().numpy().view(np.uint64), want_off)
        assert np.array_equal(dag_cols.cpu().numpy().view(np.uint32)[:m], want_cols)


def test_core_barrier_absent_block_times_out_then_recovers(gpu, faults, oracle_lib):
    import torch

    g = gg.small_rmat(32, 5000, 16.0)
    assert g.n > 3 * 1024  # the cooperative kernel runs at least three blocks
    G = gpu.DeviceGraph(g)
    rank = torch.empty(g.n, dtype=torch.int32, device="cuda")
    faults(barrier_wait_ns=2_000_000, barrier_absent_block=1)
    with pytest.raises(gpu.CitronError) as e:
        gpu.citron_core_order(g.n, G.off, G.cols, rank, None, G.ws)
    assert _status(e) == "CITRON_E_TIMEOUT"
    faults()
    level, rounds = gpu.citron_core_order(g.n, G.off, G.cols, rank, None, G.ws)
    want_rank, want_level, want_rounds = oracle_lib.core_rank_rounds(g.off, g.cols, g.n)
    assert (level, rounds) == (want_level, want_rounds)
    assert np.array_equal(rank.cpu().numpy().view(np.uint32), want_rank)


def test_seeded_total_overflows(gpu, faults):
    g = gg.config1_er_planted()
    G = gpu.DeviceGraph(g)
    k3 = G.count(3)
    assert k3 > 10
    # a total that ends exactly at 2^64 - 1 is still exact
    faults(count_seed=U64_MAX - k3)
    assert G.count(3) == U64_MAX
    # one more clique than fits: overflow, on every counting entry point
    faults(count_seed=U64_MAX - k3 + 1)
    with pytest.raises(gpu.CitronError) as e:
        G.count(3)
    assert _status(e) == "CITRON_E_OVERFLOW"
    with pytest.raises(gpu.CitronError) as e:
        G.count(3, small_max=8, bitmap_max=64)  # bitmap and sorted-list paths
    assert _status(e) == "CITRON_E_OVERFLOW"
    with pytest.raises(gpu.CitronError) as e:
        gpu.citron_count_noalloc(G.n, G.dag_off, G.dag_cols, 3)
    assert _status(e) == "CITRON_E_OVERFLOW"
    faults()
    assert G.count(3) == k3  # the error word was cleared and the next count is exact


def test_batched_overflow_reported_through_the_workspace(gpu, faults):
    from paper_2112_10913_gb300.batch import BatchCounter

    items = gg.config4_batch(seed=11, count=6, n_range=(200, 600))
    graphs, ks = [it.graph for it in items], [3] * len(items)
    bc = BatchCounter(graphs, ks)
    bc.launch()
    want = bc.result()
    assert min(want) > 0
    faults(count_seed=U64_MAX)  # any clique at all wraps the seeded per-graph totals
    bc.launch()
    with pytest.raises(gpu.CitronError) as e:
        bc.result()
    assert _status(e) == "CITRON_E_OVERFLOW"
    faults()
    bc.launch()
    assert bc.result() == want


def test_count_time_budget(gpu):
    """A count given a time budget stops taking work once the budget has run out and reports
    CITRON_E_BUDGET; the next count, with a budget it meets, is exact."""
    g = gg.config2_rmat(seed=9, scale=18, edge_factor=16)
    G = gpu.DeviceGraph(g)
    want = G.count(6)
    with pytest.raises(gpu.CitronError) as e:
        G.count(6, budget_ms=1)
    assert _status(e) == "CITRON_E_BUDGET"
    assert G.count(6, budget_ms=600000) == want
    assert G.count(6) == want
