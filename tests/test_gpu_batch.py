"""Batched counting (many graphs, each with its own k, one capturable launch sequence): every
per-graph count equals the oracle's and the one-launch-per-graph GPU path's, and CUDA-graph
replays give the same counts again."""
import numpy as np
import pytest

import oracle
from paper_2112_10913_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch_items():
    # the distribution of the 4,096-graph batch, with smaller graphs so the oracle is quick
    items = gg.config4_batch(seed=4, count=48, n_range=(50, 2500))
    # every k of the method, including the trivial ones and a graph with no edges
    items[0].k, items[1].k, items[2].k = 1, 2, 8
    items.append(gg.BatchItem(gg.csr_from_edges(7, [], []), 3))
    items.append(gg.BatchItem(gg.fig1(), 4))
    return items


def test_batch_matches_oracle_and_single_graph_path(gpu, oracle_lib, batch_items):
    from paper_2112_10913_gb300.batch import BatchCounter

    bc = BatchCounter([it.graph for it in batch_items], [it.k for it in batch_items])
    bc.launch()
    got = bc.result()
    want = [oracle_lib.count_graph(it.graph, it.k) for it in batch_items]
    assert got == want
    single = [gpu.DeviceGraph(it.graph).count(it.k) for it in batch_items]
    assert got == single


def test_batch_graph_replay(gpu, batch_items):
    from paper_2112_10913_gb300.batch import BatchCounter

    bc = BatchCounter([it.graph for it in batch_items], [it.k for it in batch_items])
    bc.launch()
    ref = bc.result()
    bc.capture()
    for _ in range(2):
        bc.counts.zero_()
        bc.replay()
        assert bc.result() == ref


def test_autotuner_keeps_counts(gpu, batch_items, tmp_path):
    from paper_2112_10913_gb300.batch import BatchCounter, tune

    bc = BatchCounter([it.graph for it in batch_items], [it.k for it in batch_items])
    bc.launch()
    ref = bc.result()
    cache = tmp_path / "tune.json"
    first = tune(bc, cache=cache, key="batch48")
    assert "ms" in first and cache.exists()
    bc.launch()
    assert bc.result() == ref
    again = tune(bc, cache=cache, key="batch48")
    assert again.get("cached") is True


def test_grouped_ordering_concatenates_the_graphs_dags(gpu, oracle_lib, batch_items):
    """citron_order_grouped ranks the union's vertices by (graph, degree, id); the DAG relabelled
    with that rank is the concatenation of every graph's own relabelled DAG (the oracle's degree
    ordering and DAG of the graph alone), ranks shifted by the graph's first position."""
    import torch

    from paper_2112_10913_gb300.batch import union_csr

    graphs = [it.graph for it in batch_items]
    u, group = union_csr(graphs)
    dev = torch.device("cuda")
    off = torch.from_numpy(u.off.view(np.int64)).to(dev)
    cols = torch.from_numpy(u.cols.view(np.int32)).to(dev)
    grp = torch.from_numpy(group.view(np.int32)).to(dev)
    ws = gpu.alloc_workspace(u.n, u.arcs, 0, device=dev)
    rank = torch.empty(u.n, dtype=torch.int32, device=dev)
    gpu.citron_order_grouped(u.n, off, grp, len(graphs), rank, None, ws)
    deg = np.diff(u.off).astype(np.int64)
    want_rank = np.empty(u.n, dtype=np.uint32)
    want_rank[np.lexsort((np.arange(u.n), deg, group))] = np.arange(u.n, dtype=np.uint32)
    assert np.array_equal(rank.cpu().numpy().view(np.uint32), want_rank)
    dag_off = torch.empty(u.n + 1, dtype=torch.int64, device=dev)
    dag_cols = torch.empty(max(1, u.arcs // 2), dtype=torch.int32, device=dev)
    gpu.citron_build_dag(u.n, off, cols, rank, dag_off, dag_cols, ws)
    got_off = dag_off.cpu().numpy().view(np.uint64)
    got_cols = dag_cols.cpu().numpy().view(np.uint32)
    vbase = abase = 0
    for g in graphs:
        r = oracle_lib.degree_rank(g.off, g.n)
        o, c = oracle_lib.dag_by_rank(g.off, g.cols, g.n, r, relabel=True)
        assert np.array_equal(got_off[vbase: vbase + g.n + 1] - np.uint64(abase), o)
        assert np.array_equal(got_cols[abase: abase + c.size], c + np.uint32(vbase))
        vbase += g.n
        abase += c.size
