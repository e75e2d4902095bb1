"""Parity at full size, in the launch configuration the bench times: the R-MAT scale-20 workload
(2^20 vertices, edge factor 16) and the Chung-Lu workload (4M vertices, exponent 2.1, 50 planted
cliques of 20-40 vertices).

- DAG bytes against the oracle's own pipeline (degree ordering, Algorithm GenOrdering, the
  relabelled DAG);
- whole-graph totals against the oracle where it finishes: R-MAT K3, K4 and (slow) K5, Chung-Lu
  K3 and K4;
- per-root counts on a sample of roots stratified by out-degree (every out-degree band, seeded)
  plus the heaviest bitmap-path roots, chosen from the DAG alone, never from the GPU's output;
  the oracle's per-root values come from the oracle's own DAG (byte-equal to the GPU's, pinned
  above);
- where the oracle cannot finish (R-MAT k = 6, 7; Chung-Lu k = 5, 6): the GPU's totals on the
  degree-ordered and on the core-ordered DAG agree (the count does not depend on the ordering,
  Sec. II).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2112_10913_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu

# out-degree bands of the stratified sample: the warp-register path (<= 32), then the bitmap
# path in doubling bands
BANDS = [(0, 8), (8, 16), (16, 32), (32, 64), (64, 128), (128, 256), (256, 512), (512, 1024)]


def stratified_roots(off, k, per_band, seed, max_outdeg=None, heaviest=0):
    """Roots that can hold a k-clique (out-degree >= k-1): up to per_band seeded roots from every
    out-degree band, optionally only below max_outdeg, plus the `heaviest` roots of the bitmap path
    (largest out-degree first).  Depends on the DAG only."""
    outdeg = np.diff(off).astype(np.int64)
    pick = []
    for b, (lo, hi) in enumerate(BANDS):
        lo = max(lo, k - 2)
        if max_outdeg is not None:
            hi = min(hi, max_outdeg)
        ids = np.nonzero((outdeg > lo) & (outdeg <= hi))[0]
        pick.append(ids[gg.permutation(seed, 10 + b, ids.size)[:per_band]])
    if heaviest:
        mid = np.nonzero((outdeg > 32) & (outdeg <= 1024))[0]
        pick.append(mid[np.argsort(-outdeg[mid], kind="stable")[:heaviest]])
    return np.unique(np.concatenate(pick)).astype(np.uint32)


def check_roots(gpu_dev, oracle_dag, k, roots):
    off, cols = oracle_dag
    n = gpu_dev.n
    pr = torch.zeros(n, dtype=torch.int64, device="cuda")
    total = gpu_dev.count(k, per_root=pr)
    got = pr.cpu().numpy().view(np.uint64)
    assert int(got.sum(dtype=np.uint64)) == total
    shuffled = roots[gg.permutation(k, 99, roots.size)]  # any order: values go to their own slot
    _, want = oracle.count_roots(off, cols, n, k, shuffled, per_root=True)
    assert np.array_equal(got[shuffled], want)
    return total


# ---- R-MAT scale 20, edge factor 16 ------------------------------------------------------------

@pytest.fixture(scope="module")
def rmat20():
    return gg.config2_rmat()


@pytest.fixture(scope="module")
def rmat20_oracle_dag(oracle_lib, rmat20):
    g = rmat20
    rank = oracle_lib.degree_rank(g.off, g.n)
    return oracle_lib.dag_by_rank(g.off, g.cols, g.n, rank, relabel=True)


@pytest.fixture(scope="module")
def dev(gpu, rmat20):
    return gpu.DeviceGraph(rmat20, relabel=True)


@pytest.fixture(scope="module")
def core_dev(gpu, rmat20):
    return gpu.DeviceGraph(rmat20, ordering="core")


def test_dag_bytes_full(gpu, oracle_lib, rmat20, rmat20_oracle_dag, dev):
    g = rmat20
    rank = oracle_lib.degree_rank(g.off, g.n)
    assert np.array_equal(dev.rank.cpu().numpy().view(np.uint32), rank)
    off, cols = rmat20_oracle_dag
    goff, gcols = dev.dag_numpy()
    assert np.array_equal(goff, off) and np.array_equal(gcols, cols)
    G0 = gpu.DeviceGraph(g, relabel=False)
    off0, cols0 = oracle_lib.gen_ordering(g.off, g.cols, g.n)
    goff0, gcols0 = G0.dag_numpy()
    assert np.array_equal(goff0, off0) and np.array_equal(gcols0, cols0)


def test_core_order_full(gpu, oracle_lib, rmat20, dev, core_dev):
    """Core ordering at full size: rank, degeneracy and rounds equal the oracle's; the core DAG's
    maximum out-degree is the degeneracy, below the degree ordering's; counts agree."""
    g = rmat20
    want, level, rounds = oracle_lib.core_rank_rounds(g.off, g.cols, g.n)
    assert np.array_equal(core_dev.rank.cpu().numpy().view(np.uint32), want)
    assert (core_dev.degeneracy, core_dev.rounds) == (level, rounds)
    assert core_dev.max_outdeg == level < dev.max_outdeg
    for k in (3, 4, 5):
        assert core_dev.count(k) == dev.count(k)


@pytest.mark.parametrize("k", [3, 4])
def test_total_full(oracle_lib, rmat20_oracle_dag, dev, k):
    off, cols = rmat20_oracle_dag
    assert dev.count(k) == oracle_lib.count(off, cols, dev.n, k)


@pytest.mark.slow
def test_k5_total_full(oracle_lib, rmat20_oracle_dag, dev):
    """The oracle's whole K5 of R-MAT 20 (minutes of CPU work on the host's cores)."""
    off, cols = rmat20_oracle_dag
    assert dev.count(5) == oracle_lib.count(off, cols, dev.n, 5)


@pytest.mark.parametrize("k,per_band,max_outdeg,heaviest", [(4, 400, None, 200), (5, 300, None, 200),
                                                            (6, 300, 64, 0)])
def test_sampled_roots(rmat20_oracle_dag, dev, k, per_band, max_outdeg, heaviest):
    off, _ = rmat20_oracle_dag
    roots = stratified_roots(off, k, per_band, seed=k, max_outdeg=max_outdeg, heaviest=heaviest)
    assert roots.size > 1000
    check_roots(dev, rmat20_oracle_dag, k, roots)


@pytest.mark.parametrize("k", [6, 7])
def test_ordering_invariance_full(dev, core_dev, k):
    """Beyond the oracle's reach: the degree-ordered and the core-ordered DAG give the same total."""
    assert dev.count(k) == core_dev.count(k)


# ---- Chung-Lu power law, n = 4M, avg degree 30, capped at 20,000, plus 50 planted cliques ----

@pytest.fixture(scope="module")
def chunglu():
    return gg.config3_chung_lu()


@pytest.fixture(scope="module")
def chunglu_oracle_dag(oracle_lib, chunglu):
    g = chunglu
    rank = oracle_lib.degree_rank(g.off, g.n)
    return oracle_lib.dag_by_rank(g.off, g.cols, g.n, rank, relabel=True)


@pytest.fixture(scope="module")
def dev3(gpu, chunglu):
    return gpu.DeviceGraph(chunglu, relabel=True)


def test_chunglu_dag_and_totals(gpu, oracle_lib, chunglu, chunglu_oracle_dag, dev3):
    g = chunglu
    rank = oracle_lib.degree_rank(g.off, g.n)
    assert np.array_equal(dev3.rank.cpu().numpy().view(np.uint32), rank)
    off, cols = chunglu_oracle_dag
    goff, gcols = dev3.dag_numpy()
    assert np.array_equal(goff, off) and np.array_equal(gcols, cols)
    for k in (3, 4):
        assert dev3.count(k) == oracle_lib.count(off, cols, g.n, k)


@pytest.mark.parametrize("k,per_band,max_outdeg,heaviest", [(5, 300, None, 100), (6, 300, 64, 0)])
def test_chunglu_sampled_roots(chunglu, chunglu_oracle_dag, dev3, k, per_band, max_outdeg, heaviest):
    import math

    off, _ = chunglu_oracle_dag
    roots = stratified_roots(off, k, per_band, seed=10 + k, max_outdeg=max_outdeg, heaviest=heaviest)
    assert roots.size > 1000
    total = check_roots(dev3, chunglu_oracle_dag, k, roots)
    # every planted clique of size s contributes C(s, k) k-cliques on its own
    assert total >= max(math.comb(s, k) for s in chunglu.meta["planted"])


@pytest.fixture(scope="module")
def core3(gpu, chunglu):
    return gpu.DeviceGraph(chunglu, ordering="core")


@pytest.mark.parametrize("k", [5, 6])
def test_chunglu_ordering_invariance(dev3, core3, k):
    assert core3.max_outdeg <= dev3.max_outdeg
    assert dev3.count(k) == core3.count(k)


# ---- the 4,096-graph batch at full size -----------------------------------------------------

def test_full_batch_sampled_graphs(gpu, oracle_lib):
    """The whole 4,096-graph batch (n log-uniform in [50, 50000], ER/R-MAT, k in 3..7), counted in
    one batched launch sequence.  A seeded sample of 40 graphs chosen from the inputs alone (at
    most 20,000 vertices; k <= 5 or average degree <= 24, which bounds the oracle's work) must
    match the oracle's own pipeline, and every batched count must match the graph's own launch
    sequence on a second seeded sample."""
    from paper_2112_10913_gb300.batch import BatchCounter

    items = gg.config4_batch_parallel(seed=4, count=4096)
    bc = BatchCounter([it.graph for it in items], [it.k for it in items])
    bc.launch()
    got = bc.result()
    order = gg.permutation(4, 9, len(items))
    def cheap(it):
        return it.graph.n <= 20000 and (it.k <= 5 or it.graph.arcs <= 24 * it.graph.n)

    picked = [int(i) for i in order if cheap(items[int(i)])][:40]
    assert len(picked) == 40
    for i in picked:
        assert got[i] == oracle_lib.count_graph(items[i].graph, items[i].k), i
    for i in [int(i) for i in order[-64:]]:
        assert got[i] == gpu.DeviceGraph(items[i].graph).count(items[i].k), i
