"""Parity of the CUDA path (called through the C ABI) with the oracle: bit-exact ranks, DAG CSR
bytes and uint64 counts, on seeded inputs that span several tiles with ragged tails, on every
counting path (warp-register, shared-memory bitmap, sorted list), and on the edge cases."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2112_10913_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


def dag_equal(G, off, cols):
    goff, gcols = G.dag_numpy()
    assert np.array_equal(goff, off), "DAG offsets differ"
    assert np.array_equal(gcols, cols), "DAG columns differ"


SMALL_GRAPHS = {
    "fig1": gg.fig1,
    "K33": lambda: gg.complete(33),
    "T(40,6)": lambda: gg.turan(40, 6),
    "CP(12)": lambda: gg.cocktail_party(12),
    "er2000+K12": gg.config1_er_planted,
    "rmat-n6000": lambda: gg.small_rmat(21, 6000, 24.0),
    "er-n9000": lambda: gg.small_er(22, 9000, 18.0),
    "rmat-n50000": lambda: gg.small_rmat(23, 50000, 30.0),
    # degree ~2 and ~1.5: a tile of arcs spans thousands of rows (and many rows are empty)
    "path-n30000": lambda: gg.csr_from_edges(30000, np.arange(29999, dtype=np.uint32),
                                             np.arange(1, 30000, dtype=np.uint32)),
    "er-n20000-sparse": lambda: gg.small_er(24, 20000, 1.5),
}


@pytest.fixture(scope="module")
def graphs():
    return {k: f() for k, f in SMALL_GRAPHS.items()}


@pytest.mark.parametrize("name", list(SMALL_GRAPHS))
def test_rank_is_degree_order(gpu, oracle_lib, graphs, name):
    g = graphs[name]
    G = gpu.DeviceGraph(g, relabel=True)
    assert np.array_equal(G.rank.cpu().numpy().view(np.uint32), oracle_lib.degree_rank(g.off, g.n))


@pytest.mark.parametrize("name", list(SMALL_GRAPHS))
def test_gen_ordering_dag_bytes(gpu, oracle_lib, graphs, name):
    g = graphs[name]
    G = gpu.DeviceGraph(g, relabel=False)
    off, cols = oracle_lib.gen_ordering(g.off, g.cols, g.n)
    dag_equal(G, off, cols)
    assert G.max_outdeg == int(np.diff(off).max())


@pytest.mark.parametrize("name", list(SMALL_GRAPHS))
def test_relabelled_dag_bytes(gpu, oracle_lib, graphs, name):
    g = graphs[name]
    G = gpu.DeviceGraph(g, relabel=True)
    rank = oracle_lib.degree_rank(g.off, g.n)
    off, cols = oracle_lib.dag_by_rank(g.off, g.cols, g.n, rank, relabel=True)
    dag_equal(G, off, cols)
    assert G.max_outdeg == int(np.diff(off).max())


@pytest.mark.parametrize("which", ["random", "identity", "core"])
def test_dag_of_any_rank(gpu, oracle_lib, graphs, which):
    g = graphs["rmat-n6000"]
    if which == "random":
        rank = gg.permutation(5, 5, g.n).argsort().astype(np.uint32)
    elif which == "identity":
        rank = np.arange(g.n, dtype=np.uint32)
    else:
        rank = oracle_lib.core_rank(g.off, g.cols, g.n)
    G = gpu.DeviceGraph(g, rank=rank)
    off, cols = oracle_lib.dag_by_rank(g.off, g.cols, g.n, rank, relabel=True)
    dag_equal(G, off, cols)
    # the count does not depend on the ordering
    ref = oracle_lib.count_graph(g, 4)
    assert G.count(4) == ref


def test_relabelled_rows_of_every_sort_length(gpu, oracle_lib):
    """Rows of every length class of the relabelled fill: sorted by one lane (<= 32 entries), by a
    warp (33..1024) and by a block (> 1024).  K_1100 in degree order has one row of each length
    0..1099; a random order of the same graph gives rows of unsorted ranks of every length."""
    g = gg.complete(1100)
    for rank in (oracle_lib.degree_rank(g.off, g.n), gg.permutation(7, 7, g.n).argsort().astype(np.uint32)):
        G = gpu.DeviceGraph(g, rank=rank)
        off, cols = oracle_lib.dag_by_rank(g.off, g.cols, g.n, rank, relabel=True)
        dag_equal(G, off, cols)
        assert G.max_outdeg == 1099


PATHS = {
    "default": {},
    "bitmap-only": dict(small_max=1, bitmap_max=1024),
    "small+list": dict(small_max=32, bitmap_max=32),
    "list-only": dict(small_max=1, bitmap_max=1),
    "narrow-cta": dict(warps_per_cta=2),
    # every bitmap-path root is split into units taken from a shared cursor; 3 blocks, so that
    # blocks that find the root queue empty help with roots still in progress
    "split-steal": dict(small_max=1, split_min=2, max_blocks=3),
}


@pytest.mark.parametrize("path", list(PATHS))
@pytest.mark.parametrize("name", ["fig1", "K33", "T(40,6)", "CP(12)", "er2000+K12", "rmat-n6000", "er-n9000"])
@pytest.mark.parametrize("relabel", [True, False])
def test_counts_match_oracle(gpu, oracle_lib, graphs, path, name, relabel):
    g = graphs[name]
    G = gpu.DeviceGraph(g, relabel=relabel)
    off, cols = G.dag_numpy()
    for k in range(1, 8):
        want = oracle_lib.count(off, cols, g.n, k)
        assert G.count(k, **PATHS[path]) == want, (k, path)


@pytest.mark.parametrize("path", ["default", "list-only", "split-steal"])
def test_per_root_counts(gpu, oracle_lib, graphs, path):
    g = graphs["rmat-n50000"]
    G = gpu.DeviceGraph(g, relabel=True)
    off, cols = G.dag_numpy()
    roots = np.arange(g.n, dtype=np.uint32)
    for k in (3, 4, 5):
        pr = torch.zeros(g.n, dtype=torch.int64, device="cuda")
        tot = G.count(k, per_root=pr, **PATHS[path])
        want_tot, want = oracle_lib.count_roots(off, cols, g.n, k, roots, per_root=True)
        got = pr.cpu().numpy().view(np.uint64)
        assert tot == want_tot
        assert np.array_equal(got, want), np.nonzero(got != want)[0][:10]


@pytest.mark.parametrize("path", list(PATHS))
def test_per_arc_counts(gpu, oracle_lib, graphs, path):
    """The debug per-arc output equals the oracle's per-edge counts arc by arc on every counting
    path (the count of each edge task: k-cliques whose first two vertices are the arc's ends),
    and sums to the total; k < 3 is refused."""
    for name in ("K33", "er2000+K12", "rmat-n6000"):
        g = graphs[name]
        G = gpu.DeviceGraph(g)
        off, cols = G.dag_numpy()
        for k in (3, 4, 5, 6):
            c, pa = G.count_per_arc(k, **PATHS[path])
            want = oracle_lib.count_per_edge(off, cols, g.n, k)
            assert np.array_equal(pa, want), (name, k, path)
            assert c == int(want.sum()) == G.count(k), (name, k, path)
    with pytest.raises(gpu.CitronError):
        gpu.DeviceGraph(graphs["fig1"]).count_per_arc(2)


def test_closed_forms(gpu):
    # (n, k) pairs whose enumeration stays small: C(n, k-1) leaf sets at most ~1e9
    for n in (1, 2, 5, 32, 33, 64, 200):
        G = gpu.DeviceGraph(gg.complete(n))
        for k in range(1, min(n + 2, 11)):
            if math.comb(n, k - 1) > 1e9:
                break
            assert G.count(k) == math.comb(n, k), (n, k)
    G = gpu.DeviceGraph(gg.cocktail_party(14))
    for k in range(1, 13):
        assert G.count(k) == math.comb(14, k) * 2 ** k
    parts = [9, 7, 7, 5, 3, 1]
    G = gpu.DeviceGraph(gg.complete_multipartite(parts))
    for k in range(1, 8):
        coef = [1]
        for s in parts:
            coef = [a + s * b for a, b in zip(coef + [0], [0] + coef)]
        assert G.count(k) == (coef[k] if k < len(coef) else 0)


def test_list_path_beyond_bitmap_capacity(gpu):
    # K_1100: out-degrees 0..1099 under any ordering; roots above 1024 take the sorted-list path
    G = gpu.DeviceGraph(gg.complete(1100))
    assert G.max_outdeg == 1099
    assert G.count(3) == math.comb(1100, 3)


def test_triangles_trace_config1(gpu):
    import scipy.sparse as sp

    g = gg.config1_er_planted()
    rows = np.repeat(np.arange(g.n), np.diff(g.off).astype(np.int64))
    a = sp.csr_matrix((np.ones(g.cols.size), (rows, g.cols.astype(np.int64))), shape=(g.n, g.n))
    assert gpu.DeviceGraph(g).count(3) == int(round((a @ a).multiply(a).sum() / 6))


def test_edge_cases(gpu, oracle_lib):
    # the empty graph: every entry point accepts n = 0
    g = gg.csr_from_edges(0, [], [])
    for relabel in (True, False):
        G = gpu.DeviceGraph(g, relabel=relabel)
        assert [G.count(k) for k in (1, 2, 3, 5)] == [0, 0, 0, 0]
    assert gpu.DeviceGraph(g, ordering="core").count(3) == 0
    assert gpu.DeviceGraph(g).list(3).shape[0] == 0
    # isolated vertices only
    g = gg.csr_from_edges(10, [], [])
    G = gpu.DeviceGraph(g)
    assert [G.count(k) for k in (1, 2, 3, 4)] == [10, 0, 0, 0]
    # one edge among many isolated vertices, ragged sizes
    g = gg.csr_from_edges(4099, [7], [4000])
    for relabel in (True, False):
        G = gpu.DeviceGraph(g, relabel=relabel)
        assert [G.count(k) for k in (1, 2, 3)] == [4099, 1, 0]
    # k above max out-degree + 1 is zero; k = 12 (largest supported) on K_14
    G = gpu.DeviceGraph(gg.complete(14))
    assert G.count(12) == math.comb(14, 12)
    g = gg.small_er(30, 3000, 3.0)
    G = gpu.DeviceGraph(g)
    assert G.max_outdeg + 2 <= 12
    for k in range(G.max_outdeg + 2, 13):
        assert G.count(k) == 0


def test_invalid_arguments(gpu):
    G = gpu.DeviceGraph(gg.fig1())
    with pytest.raises(gpu.CitronError) as e:
        G.count(0)
    assert e.value.name == "CITRON_E_INVALID"
    for k in (13, 15):
        with pytest.raises(gpu.CitronError) as e:
            G.count(k)
        assert e.value.name == "CITRON_E_UNSUPPORTED"


def test_validate_on_device(gpu, oracle_lib):
    g = gg.fig1()
    ws = gpu.alloc_workspace(g.n, g.cols.size)

    def run(cols):
        off_t = torch.from_numpy(g.off.view(np.int64)).cuda()
        cols_t = torch.from_numpy(cols.view(np.int32)).cuda()
        return gpu.citron_validate(g.n, off_t, cols_t, ws)

    assert run(g.cols.copy()) == 0
    for pos, val, want in [(0, 0, 4), (2, 6, 5), (2, 9, 2)]:
        bad = g.cols.copy()
        bad[pos] = val
        assert run(bad) == oracle_lib.validate(g.off, bad, g.n) == want
    bad = g.cols.copy()
    bad[0], bad[1] = bad[1], bad[0]
    assert run(bad) == 3


def test_host_pipeline(gpu, oracle_lib, graphs):
    g = graphs["rmat-n50000"]
    buf = torch.empty(gpu.citron_host_buffer_bytes(g.n, g.cols.size), dtype=torch.uint8, device="cuda")
    ws = gpu.alloc_workspace(g.n, g.cols.size, 2048)
    ks = [1, 2, 3, 4, 5, 6]
    got = gpu.citron_count_host(g.n, g.off, g.cols, ks, buf, ws)
    assert got == [oracle_lib.count_graph(g, k) for k in ks]


def test_dense_random_exercises_every_compact_width(gpu, oracle_lib):
    """A dense random graph (n = 300, p = 0.7, DAG max out-degree 190): candidate sets of every
    compact size class occur (1-4 word rows, packed 5- and 6-word rows at R = 3); counts equal
    the oracle's, and the cocktail-party closed form holds on a 200-vertex instance."""
    g = gg.random_small(21, 300, 0.7)
    G = gpu.DeviceGraph(g)
    assert G.max_outdeg > 160
    for k in (4, 5, 6):
        assert G.count(k) == oracle_lib.count_graph(g, k), k
    G = gpu.DeviceGraph(gg.cocktail_party(100))
    for k in (4, 5):
        assert G.count(k) == math.comb(100, k) * 2 ** k


def test_heavy_edge_splitting_and_stealing(gpu, oracle_lib):
    """Heavy roots split into edge sub-tasks (u, a_t, b) (rows above 128 members, k >= 6) and
    stolen by blocks whose root queue is empty: dense random graphs and a graph of planted
    40-cliques give the oracle's counts and per-root counts for every split threshold and block
    count, and the balance timers report a span that contains the tail."""
    dense = gg.random_small(31, 260, 0.75)
    planted = gg.config1_er_planted(seed=5, n=3000, avg_deg=12.0, clique=40)
    for g in (dense, planted):
        G = gpu.DeviceGraph(g)
        off, cols = G.dag_numpy()
        roots = np.arange(g.n, dtype=np.uint32)
        for k in (4, 5, 6, 7):
            want_tot, want = oracle_lib.count_roots(off, cols, g.n, k, roots, per_root=True)
            assert want_tot == oracle_lib.count_graph(g, k)
            for split_min, blocks in ((2, 2), (2, 7), (150, 4), (1, 0)):
                pr = torch.zeros(g.n, dtype=torch.int64, device="cuda")
                got, o = gpu.citron_count_ex(g.n, G.dag_off, G.dag_cols, k, G.ws, G.max_outdeg, pr,
                                             small_max=1, split_min=split_min, max_blocks=blocks,
                                             balance=True)
                assert got == want_tot, (k, split_min, blocks)
                assert np.array_equal(pr.cpu().numpy().view(np.uint64), want), (k, split_min, blocks)
                span, tail = o.busy_ms[0], o.busy_ms[1]
                assert 0.0 <= tail <= span
