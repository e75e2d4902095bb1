"""Seeded generators: deterministic, and every CSR satisfies the input contract
(symmetric, sorted, no loops, no duplicates)."""
import numpy as np
import pytest

import oracle
from paper_2112_10913_gb300 import graphgen as gg


def check_csr(g):
    assert g.off.dtype == np.uint64 and g.cols.dtype == np.uint32
    assert g.off[0] == 0 and g.off[-1] == g.cols.size and g.cols.size % 2 == 0
    assert oracle.validate(g.off, g.cols, g.n) == 0


def test_splitmix_reference_values():
    # SplitMix64 with state 0: the first outputs of the published generator
    z = gg._mix(np.array([0x9E3779B97F4A7C15], dtype=np.uint64))
    assert int(z[0]) == 0xE220A8397B1DCDAF


def test_draws_deterministic_and_counter_based():
    a = gg.draws_u64(5, 3, 1000)
    b = gg.draws_u64(5, 3, 600, start=400)
    assert np.array_equal(a[400:], b)
    assert not np.array_equal(a, gg.draws_u64(5, 4, 1000))
    u = gg.uniform(1, 1, 100000)
    assert 0.49 < u.mean() < 0.51 and u.min() >= 0 and u.max() < 1


@pytest.mark.parametrize("make", [gg.fig1, lambda: gg.complete(10), lambda: gg.turan(11, 4),
                                  lambda: gg.cocktail_party(4), lambda: gg.config1_er_planted(),
                                  lambda: gg.small_rmat(3, 5000, 20.0), lambda: gg.small_er(4, 3000, 30.0),
                                  lambda: gg.random_small(1, 14, 0.5)])
def test_csr_contract(make):
    check_csr(make())


def test_config1_shape():
    g = gg.config1_er_planted()
    assert g.n == 2000
    assert 19000 < g.m < 21500  # ER(2000, 20/1999): ~20,000 edges, plus <= 66 planted
    h = gg.config1_er_planted()
    assert np.array_equal(g.cols, h.cols)


def test_rmat_small_scale_shape():
    g = gg.config2_rmat(seed=2, scale=12, edge_factor=16)
    check_csr(g)
    deg = g.degrees()
    assert g.n == 4096 and deg.max() > 20 * deg.mean()  # heavy-tailed


def test_chung_lu_small_shape():
    g = gg.config3_chung_lu(seed=3, n=20000, cliques=3, clique_range=(10, 12))
    check_csr(g)
    w = gg.chung_lu_weights(20000, 2.1, 30.0, 20000.0)
    assert abs(w.mean() - 30.0) < 1e-6
    assert g.degrees().max() > 10 * g.degrees().mean()


def test_batch_items():
    items = gg.config4_batch(seed=4, count=6, n_range=(50, 400))
    for it in items:
        check_csr(it.graph)
        assert 3 <= it.k <= 7 and 50 <= it.graph.n <= 400


def test_parallel_batch_equals_serial():
    a = gg.config4_batch(seed=9, count=6, n_range=(50, 300))
    b = gg.config4_batch_parallel(seed=9, count=6, n_range=(50, 300), workers=2)
    for x, y in zip(a, b):
        assert x.k == y.k and np.array_equal(x.graph.off, y.graph.off) and np.array_equal(x.graph.cols, y.graph.cols)


def test_union_csr_for_batching():
    """The batch's union CSR: every graph's rows shifted by the vertices before it, the group map
    names each vertex's graph, the CSR contract holds, and (disjoint-union additivity) the
    oracle's count of the union is the sum of the graphs' counts for every k."""
    import oracle
    from paper_2112_10913_gb300.batch import union_csr

    graphs = [gg.fig1(), gg.csr_from_edges(3, [], []), gg.complete(6), gg.small_er(5, 200, 8.0)]
    u, group = union_csr(graphs)
    assert u.n == sum(g.n for g in graphs) and u.arcs == sum(g.arcs for g in graphs)
    assert oracle.validate(u.off, u.cols, u.n) == 0
    base = 0
    for i, g in enumerate(graphs):
        assert np.all(group[base: base + g.n] == i)
        for v in range(g.n):
            row = u.cols[u.off[base + v]: u.off[base + v + 1]]
            assert np.array_equal(row, g.cols[g.off[v]: g.off[v + 1]] + base)
        base += g.n
    for k in (1, 2, 3, 4, 5):
        assert oracle.count_graph(u, k) == sum(oracle.count_graph(g, k) for g in graphs)
