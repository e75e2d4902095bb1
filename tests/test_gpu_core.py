"""Core ordering on the GPU (citron_core_order, Algorithm OrdCore in synchronous rounds): the rank,
the degeneracy and the number of rounds equal the oracle's round-based restatement; the DAG of
that rank has the degeneracy as its maximum out-degree; counts do not depend on the ordering."""
import numpy as np
import pytest
import torch

from paper_2112_10913_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


def _graph(n, edges):
    u = np.array([a for a, _ in edges], dtype=np.uint32)
    v = np.array([b for _, b in edges], dtype=np.uint32)
    return gg.csr_from_edges(n, u, v)


GRAPHS = {
    "fig1": gg.fig1,
    "path7": lambda: _graph(7, [(i, i + 1) for i in range(6)]),
    "star": lambda: _graph(40, [(0, i) for i in range(1, 40)]),
    "lollipop": lambda: _graph(6, [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3), (3, 4), (4, 5)]),
    "k20": lambda: gg.complete(20),
    "isolated": lambda: _graph(50, [(3, 4), (4, 5), (10, 11)]),
    "edgeless": lambda: _graph(9, []),
    "long_path": lambda: _graph(3001, [(i, i + 1) for i in range(3000)]),
    "c1": gg.config1_er_planted,
    "er": lambda: gg.small_er(11, 20000, 24.0),
    "rmat": lambda: gg.small_rmat(12, 50000, 30.0),
    "rmat16": lambda: gg.config2_rmat(seed=6, scale=16, edge_factor=16),
    "turan": lambda: gg.complete_multipartite([30, 20, 10, 5]),
}


def _core(gpu, g):
    dev = torch.device("cuda")
    off = torch.from_numpy(g.off.view(np.int64)).to(dev)
    cols = torch.from_numpy(g.cols.view(np.int32)).to(dev) if g.arcs else torch.zeros(1, dtype=torch.int32, device=dev)
    ws = gpu.alloc_workspace(g.n, g.arcs, 1, device=dev)
    rank = torch.empty(max(1, g.n), dtype=torch.int32, device=dev)
    perm = torch.empty(max(1, g.n), dtype=torch.int32, device=dev)
    level, rounds = gpu.citron_core_order(g.n, off, cols[: g.arcs] if g.arcs else cols[:0], rank, perm, ws)
    return rank.cpu().numpy().view(np.uint32)[: g.n], perm.cpu().numpy().view(np.uint32)[: g.n], level, rounds


@pytest.mark.parametrize("name", list(GRAPHS))
def test_rank_equals_oracle_rounds(gpu, oracle_lib, name):
    g = GRAPHS[name]()
    rank, perm, level, rounds = _core(gpu, g)
    want, wlevel, wrounds = oracle_lib.core_rank_rounds(g.off, g.cols, g.n)
    assert np.array_equal(rank, want), name
    assert np.array_equal(perm[rank], np.arange(g.n, dtype=np.uint32))
    assert (level, rounds) == (wlevel, wrounds)


@pytest.mark.parametrize("name", ["fig1", "c1", "rmat", "turan", "rmat16"])
def test_core_dag_degeneracy_and_counts(gpu, oracle_lib, name):
    g = GRAPHS[name]()
    core = gpu.DeviceGraph(g, ordering="core")
    deg = gpu.DeviceGraph(g)
    assert core.max_outdeg == core.degeneracy <= deg.max_outdeg
    off, cols = core.dag_numpy()
    rank, _, _ = oracle_lib.core_rank_rounds(g.off, g.cols, g.n)
    woff, wcols = oracle_lib.dag_by_rank(g.off, g.cols, g.n, rank, relabel=True)
    assert np.array_equal(off, woff) and np.array_equal(cols, wcols)
    for k in range(3, 8):
        assert core.count(k) == deg.count(k), k
    if g.n <= 5000:
        for k in (3, 4, 5):
            assert core.count(k) == oracle_lib.count_graph(g, k)
