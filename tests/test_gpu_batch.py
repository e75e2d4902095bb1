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
