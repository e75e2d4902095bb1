"""Parity at full size: the R-MAT scale-20 workload (2^20 vertices, edge factor 16) and the
Chung-Lu workload (4M vertices, exponent 2.1, 50 planted cliques of 20-40 vertices), in the
launch configuration the bench times: DAG bytes against the oracle, the exact triangle count, and
per-root counts for k = 4..6 on a seeded sample of roots the oracle can finish one by one."""
import numpy as np
import pytest
import torch

import oracle
from paper_2112_10913_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rmat20():
    return gg.config2_rmat()


@pytest.fixture(scope="module")
def dev(gpu, rmat20):
    return gpu.DeviceGraph(rmat20, relabel=True)


def test_dag_bytes_full(gpu, oracle_lib, rmat20, dev):
    g = rmat20
    rank = oracle_lib.degree_rank(g.off, g.n)
    assert np.array_equal(dev.rank.cpu().numpy().view(np.uint32), rank)
    off, cols = oracle_lib.dag_by_rank(g.off, g.cols, g.n, rank, relabel=True)
    goff, gcols = dev.dag_numpy()
    assert np.array_equal(goff, off) and np.array_equal(gcols, cols)
    G0 = gpu.DeviceGraph(g, relabel=False)
    off0, cols0 = oracle_lib.gen_ordering(g.off, g.cols, g.n)
    goff0, gcols0 = G0.dag_numpy()
    assert np.array_equal(goff0, off0) and np.array_equal(gcols0, cols0)


def test_core_order_full(gpu, oracle_lib, rmat20, dev):
    """Core ordering at full size: rank, degeneracy and rounds equal the oracle's; the core DAG's
    maximum out-degree is the degeneracy, below the degree ordering's; counts agree."""
    g = rmat20
    core = gpu.DeviceGraph(g, ordering="core")
    want, level, rounds = oracle_lib.core_rank_rounds(g.off, g.cols, g.n)
    assert np.array_equal(core.rank.cpu().numpy().view(np.uint32), want)
    assert (core.degeneracy, core.rounds) == (level, rounds)
    assert core.max_outdeg == level < dev.max_outdeg
    for k in (3, 4, 5):
        assert core.count(k) == dev.count(k)


def test_triangles_full(oracle_lib, dev):
    off, cols = dev.dag_numpy()
    assert dev.count(3) == oracle_lib.count(off, cols, dev.n, 3)


@pytest.mark.parametrize("k", [4, 5, 6])
def test_sampled_roots(oracle_lib, dev, k):
    off, cols = dev.dag_numpy()
    n = dev.n
    pr = torch.zeros(n, dtype=torch.int64, device="cuda")
    total = dev.count(k, per_root=pr)
    got = pr.cpu().numpy().view(np.uint64)
    assert int(got.sum(dtype=np.uint64)) == total
    outdeg = np.diff(off).astype(np.int64)
    # seeded sample: 2000 roots of the warp path, 1500 of the bitmap path (out-degree > 32)
    light = np.nonzero((outdeg >= k - 1) & (outdeg <= 32))[0]
    heavy = np.nonzero(outdeg > 32)[0]
    pick = np.concatenate([light[gg.permutation(k, 1, light.size)[:2000]],
                           heavy[gg.permutation(k, 2, heavy.size)[:1500]]])
    # keep roots the oracle can finish quickly (bounded work), at most 3e9 cliques in all
    pick = pick[got[pick] <= 5e7]
    pick = pick[np.cumsum(got[pick].astype(np.float64)) <= 3e9]
    assert pick.size > 1000
    _, want = oracle_lib.count_roots(off, cols, n, k, pick.astype(np.uint32), per_root=True)
    assert np.array_equal(got[pick], want)


# ---- Chung-Lu power law, n = 4M, avg degree 30, capped at 20,000, plus 50 planted cliques ----

@pytest.fixture(scope="module")
def chunglu():
    return gg.config3_chung_lu()


@pytest.fixture(scope="module")
def dev3(gpu, chunglu):
    return gpu.DeviceGraph(chunglu, relabel=True)


def test_chunglu_dag_and_triangles(gpu, oracle_lib, chunglu, dev3):
    g = chunglu
    rank = oracle_lib.degree_rank(g.off, g.n)
    assert np.array_equal(dev3.rank.cpu().numpy().view(np.uint32), rank)
    off, cols = oracle_lib.dag_by_rank(g.off, g.cols, g.n, rank, relabel=True)
    goff, gcols = dev3.dag_numpy()
    assert np.array_equal(goff, off) and np.array_equal(gcols, cols)
    assert dev3.count(3) == oracle_lib.count(off, cols, g.n, 3)


@pytest.mark.parametrize("k", [5, 6])
def test_chunglu_sampled_roots(oracle_lib, chunglu, dev3, k):
    import math

    off, cols = dev3.dag_numpy()
    n = dev3.n
    pr = torch.zeros(n, dtype=torch.int64, device="cuda")
    total = dev3.count(k, per_root=pr)
    got = pr.cpu().numpy().view(np.uint64)
    assert int(got.sum(dtype=np.uint64)) == total
    # every planted clique of size s contributes C(s, k) k-cliques on its own
    assert total >= max(math.comb(s, k) for s in chunglu.meta["planted"])
    outdeg = np.diff(off).astype(np.int64)
    light = np.nonzero((outdeg >= k - 1) & (outdeg <= 32))[0]
    heavy = np.nonzero(outdeg > 32)[0]
    pick = np.concatenate([light[gg.permutation(k, 3, light.size)[:2000]],
                           heavy[gg.permutation(k, 4, heavy.size)[:1500]]])
    pick = pick[got[pick] <= 5e7]
    pick = pick[np.cumsum(got[pick].astype(np.float64)) <= 3e9]
    assert pick.size > 1000
    _, want = oracle_lib.count_roots(off, cols, n, k, pick.astype(np.uint32), per_root=True)
    assert np.array_equal(got[pick], want)


# ---- the 4,096-graph batch at full size -----------------------------------------------------

def test_full_batch_sampled_graphs(gpu, oracle_lib):
    """The whole 4,096-graph batch (n log-uniform in [50, 50000], ER/R-MAT, k in 3..7), counted in
    one batched launch sequence; a seeded sample of 40 graphs that the oracle finishes quickly
    (count <= 1e8, n <= 20000) must match the oracle, and every batched count must match the
    graph's own launch sequence on a second seeded sample."""
    from paper_2112_10913_gb300.batch import BatchCounter

    items = gg.config4_batch_parallel(seed=4, count=4096)
    bc = BatchCounter([it.graph for it in items], [it.k for it in items])
    bc.launch()
    got = bc.result()
    order = gg.permutation(4, 9, len(items))
    picked = [int(i) for i in order if got[int(i)] <= 1e8 and items[int(i)].graph.n <= 20000][:40]
    assert len(picked) == 40
    for i in picked:
        assert got[i] == oracle_lib.count_graph(items[i].graph, items[i].k), i
    for i in [int(i) for i in order[-64:]]:
        assert got[i] == gpu.DeviceGraph(items[i].graph).count(items[i].k), i
