"""Pins of the oracle against facts that do not come from the oracle itself.

- the Fig. 1 worked example (DAG arrows, the induced subgraph of vertex 0, c(G) = 3), read from
  tests/golden/fig1.txt;
- brute-force enumeration of all k-subsets (the plain definition of a k-clique, Sec. II);
- closed forms: C(n,k) on K_n, elementary symmetric polynomials of the part sizes on complete
  multipartite (Turan) graphs, C(r,k) 2^k on cocktail-party graphs;
- k = 3 against trace(A^3)/6 from a sparse matrix product;
- invariants: the count does not depend on the ordering (degree, identity, random, core), on
  vertex renaming, on relabelling the DAG to ranks; disjoint unions add;
- the core ordering's DAG has the smallest possible maximum out-degree (the degeneracy, found by
  brute force over vertex subsets), never above the degree ordering's.
"""
import itertools
import math

import numpy as np
import pytest
import scipy.sparse as sp

from paper_2112_10913_gb300 import graphgen as gg

GOLDEN = __import__("pathlib").Path(__file__).resolve().parent / "golden"


def read_golden(name):
    sections, cur = {}, None
    for line in (GOLDEN / name).read_text().splitlines():
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("["):
            cur = line.strip("[]")
            sections[cur] = []
        else:
            sections[cur].append([int(x) for x in line.split()])
    return sections


def adjacency_sets(g):
    return [set(g.cols[g.off[u]: g.off[u + 1]].tolist()) for u in range(g.n)]


def brute_count(g, k):
    """Number of k-subsets of V whose members are pairwise adjacent."""
    adj = adjacency_sets(g)
    if k == 0:
        return 1
    total = 0
    for s in itertools.combinations(range(g.n), k):
        if all(b in adj[a] for a, b in itertools.combinations(s, 2)):
            total += 1
    return total


def elementary_symmetric(parts, k):
    """e_k(parts) from the coefficients of prod(1 + s x)."""
    coef = [1]
    for s in parts:
        nxt = coef + [0]
        for i in range(len(coef)):
            nxt[i + 1] += coef[i] * s
        coef = nxt
    return coef[k] if k < len(coef) else 0


def dag_lists(off, cols, n):
    return [sorted(cols[off[u]: off[u + 1]].tolist()) for u in range(n)]


# -- Fig. 1 ------------------------------------------------------------------------------------


def test_fig1_graph_is_the_printed_one(oracle_lib):
    gold = read_golden("fig1.txt")
    g = gg.fig1()
    edges = {tuple(sorted(e)) for e in gold["edges"]}
    u, v = gg.edges_of(g)
    assert edges == set(zip(u.tolist(), v.tolist()))
    assert oracle_lib.validate(g.off, g.cols, g.n) == 0


def test_fig1_dag_is_the_printed_dag(oracle_lib):
    gold = read_golden("fig1.txt")
    g = gg.fig1()
    off, cols = oracle_lib.gen_ordering(g.off, g.cols, g.n)
    got = {(u, v) for u in range(g.n) for v in cols[off[u]: off[u + 1]].tolist()}
    assert got == {tuple(a) for a in gold["dag"]}
    # rows come out sorted (the DAG the paper keeps sorted, Sec. V-B)
    for u in range(g.n):
        row = cols[off[u]: off[u + 1]]
        assert np.all(np.diff(row.astype(np.int64)) > 0)


def test_fig1_induced_subgraph_of_vertex0(oracle_lib):
    gold = read_golden("fig1.txt")
    g = gg.fig1()
    off, cols = oracle_lib.gen_ordering(g.off, g.cols, g.n)
    verts = cols[off[0]: off[1]].tolist()
    assert verts == gold["induced0_vertices"][0]
    arcs = {(a, b) for a in verts for b in cols[off[a]: off[a + 1]].tolist() if b in verts}
    assert arcs == {tuple(a) for a in gold["induced0_arcs"]}


def test_fig1_core_value(oracle_lib):
    gold = read_golden("fig1.txt")
    g = gg.fig1()
    rank = oracle_lib.core_rank(g.off, g.cols, g.n)
    off, _ = oracle_lib.dag_by_rank(g.off, g.cols, g.n, rank, relabel=False)
    assert int(np.diff(off).max()) == gold["core_value"][0][0]


def test_fig1_counts_equal_brute_force(oracle_lib):
    g = gg.fig1()
    got = [oracle_lib.count_graph(g, k) for k in range(1, 7)]
    assert got == [brute_count(g, k) for k in range(1, 7)]
    assert got[:5] == [7, 11, 5, 1, 0]


# -- brute force on random small graphs ---------------------------------------------------------


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("n,p", [(9, 0.5), (12, 0.7), (15, 0.85), (16, 0.35)])
def test_brute_force(oracle_lib, seed, n, p):
    g = gg.random_small(seed * 100 + n, n, p)
    for k in range(1, n + 2):
        want = brute_count(g, k)
        assert oracle_lib.count_graph(g, k, threads=2) == want, (k, want)
        if want == 0 and k > 3:
            break


# -- closed forms --------------------------------------------------------------------------------


@pytest.mark.parametrize("n", [1, 2, 3, 7, 20, 40])
def test_complete_graph(oracle_lib, n):
    g = gg.complete(n)
    for k in range(1, min(n + 2, 12)):
        assert oracle_lib.count_graph(g, k) == math.comb(n, k)


@pytest.mark.parametrize("parts", [[4, 3, 3], [5, 5, 5, 5], [1, 2, 3, 4, 5], [7, 1], [3] * 8])
def test_complete_multipartite(oracle_lib, parts):
    g = gg.complete_multipartite(parts)
    for k in range(1, len(parts) + 2):
        assert oracle_lib.count_graph(g, k) == elementary_symmetric(parts, k)


def test_turan_10_3(oracle_lib):
    g = gg.turan(10, 3)  # parts 4, 3, 3
    assert [oracle_lib.count_graph(g, k) for k in (2, 3, 4)] == [33, 36, 0]


@pytest.mark.parametrize("r", [2, 5, 9])
def test_cocktail_party(oracle_lib, r):
    g = gg.cocktail_party(r)
    for k in range(1, r + 2):
        assert oracle_lib.count_graph(g, k) == math.comb(r, k) * 2 ** k


# -- k = 3 by linear algebra -----------------------------------------------------------------------


def trace_a3_over_6(g):
    rows = np.repeat(np.arange(g.n), np.diff(g.off).astype(np.int64))
    a = sp.csr_matrix((np.ones(g.cols.size, dtype=np.float64), (rows, g.cols.astype(np.int64))),
                      shape=(g.n, g.n))
    return int(round((a @ a).multiply(a).sum() / 6))


@pytest.mark.parametrize("make", [lambda: gg.config1_er_planted(),
                                  lambda: gg.small_rmat(5, 3000, 24.0),
                                  lambda: gg.small_er(6, 4000, 40.0)])
def test_triangles_trace(oracle_lib, make):
    g = make()
    assert oracle_lib.count_graph(g, 3) == trace_a3_over_6(g)


# -- invariants ------------------------------------------------------------------------------------


def orderings(oracle_lib, g):
    yield "degree", oracle_lib.degree_rank(g.off, g.n)
    yield "identity", np.arange(g.n, dtype=np.uint32)
    yield "random", np.argsort(gg.draws_u64(77, 1, g.n)).astype(np.uint32).argsort().astype(np.uint32)
    yield "core", oracle_lib.core_rank(g.off, g.cols, g.n)
    yield "core_rounds", oracle_lib.core_rank_rounds(g.off, g.cols, g.n)[0]


@pytest.mark.parametrize("make", [lambda: gg.config1_er_planted(), lambda: gg.small_rmat(9, 1500, 30.0),
                                  lambda: gg.complete_multipartite([6, 5, 4, 3, 2])])
def test_ordering_invariance(oracle_lib, make):
    g = make()
    ref = {k: oracle_lib.count_graph(g, k) for k in range(3, 7)}
    for name, rank in orderings(oracle_lib, g):
        assert sorted(rank.tolist()) == list(range(g.n)), name
        for relabel in (False, True):
            off, cols = oracle_lib.dag_by_rank(g.off, g.cols, g.n, rank, relabel)
            assert off[-1] == g.m
            for k, want in ref.items():
                assert oracle_lib.count(off, cols, g.n, k) == want, (name, relabel, k)


def test_degree_rank_gives_gen_ordering_dag(oracle_lib):
    g = gg.small_rmat(3, 2000, 20.0)
    rank = oracle_lib.degree_rank(g.off, g.n)
    deg = g.degrees()
    order = np.argsort(rank)
    # rank sorts by (degree, id)
    keys = list(zip(deg[order].tolist(), order.tolist()))
    assert keys == sorted(keys)
    a = oracle_lib.gen_ordering(g.off, g.cols, g.n)
    b = oracle_lib.dag_by_rank(g.off, g.cols, g.n, rank, relabel=False)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_vertex_renaming_invariance(oracle_lib):
    g = gg.config1_er_planted()
    h = gg.relabel(g, gg.permutation(11, 3, g.n))
    for k in (3, 4, 5, 6):
        assert oracle_lib.count_graph(g, k) == oracle_lib.count_graph(h, k)


def test_disjoint_union_adds(oracle_lib):
    parts = [gg.complete(9), gg.cocktail_party(5), gg.small_er(3, 300, 12.0), gg.fig1()]
    u = gg.disjoint_union(parts)
    for k in (1, 2, 3, 4, 5):
        assert oracle_lib.count_graph(u, k) == sum(oracle_lib.count_graph(p, k) for p in parts)


def test_planted_clique_lower_bound(oracle_lib):
    g = gg.config1_er_planted()
    for k in (3, 4, 5, 6):
        assert oracle_lib.count_graph(g, k) >= math.comb(12, k)


def test_k_beyond_max_outdegree_is_zero(oracle_lib):
    g = gg.small_rmat(4, 800, 16.0)
    off, cols = oracle_lib.gen_ordering(g.off, g.cols, g.n)
    mx = int(np.diff(off).max())
    assert oracle_lib.count(off, cols, g.n, mx + 2) == 0


def test_per_root_and_per_edge_sum_to_total(oracle_lib):
    g = gg.config1_er_planted()
    off, cols = oracle_lib.gen_ordering(g.off, g.cols, g.n)
    for k in (3, 4, 5):
        tot = oracle_lib.count(off, cols, g.n, k)
        pe = oracle_lib.count_per_edge(off, cols, g.n, k)
        s, pr = oracle_lib.count_roots(off, cols, g.n, k, np.arange(g.n), per_root=True)
        assert int(pe.sum()) == tot == s == int(pr.sum())


def brute_first_two(g, k, key):
    """For every k-clique (brute force over k-subsets), its first and second vertex when the
    vertices are ordered by key (smaller first): the root that counts it (Sec. II, every clique is
    counted once at its first vertex in the DAG order) and the edge task (root, second) that
    reaches it in the edge-parallel form."""
    adj = adjacency_sets(g)
    out = []
    for s in itertools.combinations(range(g.n), k):
        if all(b in adj[a] for a, b in itertools.combinations(s, 2)):
            o = sorted(s, key=key)
            out.append((o[0], o[1] if k > 1 else None))
    return out


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
@pytest.mark.parametrize("relabel", [False, True])
def test_per_root_and_per_edge_values_equal_brute_force(oracle_lib, seed, relabel):
    """Every per-root value (for a shuffled subset of roots) and every per-edge value equals the
    number of brute-force k-cliques whose first vertex (first two vertices) in the DAG order it is.
    Two DAG layouts: Algorithm GenOrdering's (input ids, degree order) and a DAG relabelled to a
    seeded random order (row r = the vertex of rank r)."""
    rng = np.random.default_rng(100 + seed)
    n = 14 + seed
    g = gg.random_small(seed + 40, n, 0.55)
    deg = np.diff(g.off).astype(np.int64)
    if relabel:
        rank = rng.permutation(n).astype(np.uint32)
        off, cols = oracle_lib.dag_by_rank(g.off, g.cols, n, rank, relabel=True)
        key = lambda u: int(rank[u])
        name = lambda u: int(rank[u])  # DAG id of input vertex u
    else:
        off, cols = oracle_lib.gen_ordering(g.off, g.cols, n)
        key = lambda u: (int(deg[u]), u)
        name = lambda u: u
    roots = rng.permutation(n)[: n - 3].astype(np.uint32)  # shuffled, not all vertices
    for k in (3, 4, 5):
        firsts = brute_first_two(g, k, key)
        want_root = np.zeros(n, dtype=np.int64)
        want_edge = {}
        for a, b in firsts:
            want_root[name(a)] += 1
            want_edge[(name(a), name(b))] = want_edge.get((name(a), name(b)), 0) + 1
        tot, pr = oracle_lib.count_roots(off, cols, n, k, roots, per_root=True)
        assert [int(x) for x in pr] == [int(want_root[r]) for r in roots]
        assert tot == int(want_root[roots].sum())
        pe = oracle_lib.count_per_edge(off, cols, n, k)
        # the arc-subset form on a shuffled subset of arcs (including arcs of the last rows)
        sub = rng.permutation(int(off[-1]))[: max(1, int(off[-1]) // 2)].astype(np.uint64)
        sub_tot, pa = oracle_lib.count_arcs(off, cols, n, k, sub, per_arc=True)
        for u in range(n):
            for e in range(int(off[u]), int(off[u + 1])):
                assert int(pe[e]) == want_edge.pop((u, int(cols[e])), 0), (k, u, int(cols[e]))
        assert not want_edge  # every (root, second) pair is an arc of the DAG
        assert [int(x) for x in pa] == [int(pe[e]) for e in sub] and sub_tot == int(pe[sub].sum())


def degeneracy_brute(g):
    adj = adjacency_sets(g)
    best = 0
    for mask in range(1, 1 << g.n):
        s = [v for v in range(g.n) if mask >> v & 1]
        best = max(best, min(len(adj[v] & set(s)) for v in s))
    return best


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_core_order_minimises_max_outdegree(oracle_lib, seed):
    g = gg.random_small(seed, 12, 0.45)
    core = oracle_lib.core_rank(g.off, g.cols, g.n)
    off_c, _ = oracle_lib.dag_by_rank(g.off, g.cols, g.n, core, relabel=False)
    off_d, _ = oracle_lib.gen_ordering(g.off, g.cols, g.n)
    mc, md = int(np.diff(off_c).max()), int(np.diff(off_d).max())
    assert mc == degeneracy_brute(g)
    assert mc <= md


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5])
def test_core_rounds_order_reaches_the_degeneracy(oracle_lib, seed):
    g = gg.random_small(seed, 13, 0.4)
    rank, level, rounds = oracle_lib.core_rank_rounds(g.off, g.cols, g.n)
    assert sorted(rank.tolist()) == list(range(g.n))
    off, _ = oracle_lib.dag_by_rank(g.off, g.cols, g.n, rank, relabel=False)
    assert int(np.diff(off).max()) == level == degeneracy_brute(g)
    assert 1 <= rounds <= g.n


def _graph(n, edges):
    u = np.array([a for a, _ in edges], dtype=np.uint32)
    v = np.array([b for _, b in edges], dtype=np.uint32)
    return gg.csr_from_edges(n, u, v)


# rounds worked out by hand from the definition (remove every vertex of remaining degree <= level
# together, level = max(level, smallest remaining degree), ties by id)
@pytest.mark.parametrize("name,n,edges,want_rank,want_level,want_rounds", [
    ("path7", 7, [(i, i + 1) for i in range(6)], [0, 2, 4, 6, 5, 3, 1], 1, 4),
    ("star5", 6, [(0, i) for i in range(1, 6)], [5, 0, 1, 2, 3, 4], 1, 2),
    ("cycle6", 6, [(i, (i + 1) % 6) for i in range(6)], [0, 1, 2, 3, 4, 5], 2, 1),
    ("k5", 5, [(i, j) for i in range(5) for j in range(i + 1, 5)], [0, 1, 2, 3, 4], 4, 1),
    ("lollipop", 6, [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3), (3, 4), (4, 5)],
     [2, 3, 4, 5, 1, 0], 3, 3),
])
def test_core_rounds_hand_examples(oracle_lib, name, n, edges, want_rank, want_level, want_rounds):
    g = _graph(n, edges)
    rank, level, rounds = oracle_lib.core_rank_rounds(g.off, g.cols, g.n)
    assert rank.tolist() == want_rank and level == want_level and rounds == want_rounds, name


def test_fig1_core_value_by_rounds(oracle_lib):
    gold = read_golden("fig1.txt")
    g = gg.fig1()
    rank, level, _ = oracle_lib.core_rank_rounds(g.off, g.cols, g.n)
    off, _ = oracle_lib.dag_by_rank(g.off, g.cols, g.n, rank, relabel=False)
    assert int(np.diff(off).max()) == level == gold["core_value"][0][0]


def test_gen_ordering_keeps_each_edge_once(oracle_lib):
    g = gg.small_rmat(8, 5000, 30.0)
    off, cols = oracle_lib.gen_ordering(g.off, g.cols, g.n)
    deg = g.degrees()
    rows = np.repeat(np.arange(g.n), np.diff(off).astype(np.int64))
    c = cols.astype(np.int64)
    assert off[-1] == g.m
    # orientation: lower degree first, lower id on ties (Sec. II / Algorithm GenOrdering)
    assert np.all((deg[rows] < deg[c]) | ((deg[rows] == deg[c]) & (rows < c)))
    eu, ev = gg.edges_of(g)
    a = set(zip(np.minimum(rows, c).tolist(), np.maximum(rows, c).tolist()))
    assert a == set(zip(eu.tolist(), ev.tolist()))


def test_validate_catches_defects(oracle_lib):
    g = gg.fig1()
    assert oracle_lib.validate(g.off, g.cols, g.n) == 0
    bad = g.cols.copy()
    bad[0], bad[1] = bad[1], bad[0]  # unsorted
    assert oracle_lib.validate(g.off, bad, g.n) == 3
    bad = g.cols.copy()
    bad[0] = 0  # self-loop at vertex 0
    assert oracle_lib.validate(g.off, bad, g.n) == 4
    bad = g.cols.copy()
    bad[2] = 6  # 0 -> 6 without 6 -> 0
    assert oracle_lib.validate(g.off, bad, g.n) == 5
    bad = g.cols.copy()
    bad[2] = 9
    assert oracle_lib.validate(g.off, bad, g.n) == 2


# -- listing (Sec. VIII: the counting recursion enumerates every clique once) ------------------


def brute_cliques(g, k):
    adj = adjacency_sets(g)
    return {frozenset(s) for s in itertools.combinations(range(g.n), k)
            if all(b in adj[a] for a, b in itertools.combinations(s, 2))}


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("relabel", [False, True])
def test_listing_is_the_set_of_all_cliques(oracle_lib, seed, relabel):
    g = gg.random_small(seed, 14, 0.6)
    rank = oracle_lib.degree_rank(g.off, g.n)
    off, cols = oracle_lib.dag_by_rank(g.off, g.cols, g.n, rank, relabel)
    inv = np.argsort(rank) if relabel else np.arange(g.n)
    for k in range(1, 8):
        rows = oracle_lib.list_cliques(off, cols, g.n, k)
        got = [frozenset(inv[r].tolist()) for r in rows]
        assert len(got) == len(set(got)) == brute_count(g, k)
        assert set(got) == brute_cliques(g, k)
        # each row follows DAG arcs: every later vertex is an out-neighbour of every earlier one
        for r in rows[:200]:
            for i in range(k):
                for j in range(i + 1, k):
                    assert r[j] in cols[off[r[i]]: off[r[i] + 1]]


def test_listing_fig1_and_capacity(oracle_lib):
    g = gg.fig1()
    off, cols = oracle_lib.gen_ordering(g.off, g.cols, g.n)
    tri = oracle_lib.list_cliques(off, cols, g.n, 3)
    assert {frozenset(r.tolist()) for r in tri} == brute_cliques(g, 3) and len(tri) == 5
    assert [set(r.tolist()) for r in oracle_lib.list_cliques(off, cols, g.n, 4)] == [{0, 1, 3, 4}]
    part = oracle_lib.list_cliques(off, cols, g.n, 3, capacity=2)
    assert part.tolist() == tri[:2].tolist()
