"""The pins are strong enough: plant plausible mistakes in a COPY of the oracle (a flipped
comparison, a dropped element, an off-by-one, a transposed operand), compile each mutant on the
CPU and check that at least one pin fails for it.  The oracle source itself is never changed."""
import ctypes
import itertools
import math
import subprocess
from pathlib import Path

import numpy as np
import pytest

import oracle
from paper_2112_10913_gb300 import graphgen as gg

SRC = Path(oracle.__file__).resolve().parent / "citron_oracle.c"

# (name, original text, mutated text); every original must occur exactly once.
MUTANTS = [
    ("degree-direction", "return du < dv || (du == dv && u < v);", "return du > dv || (du == dv && u < v);"),
    ("tie-break", "return du < dv || (du == dv && u < v);", "return du < dv || (du == dv && u > v);"),
    ("prune-off-by-one", "if (len < (uint32_t)r) return ORACLE_OK;", "if (len <= (uint32_t)r) return ORACLE_OK;"),
    ("leaf-size", "        *out = len;\n        return ORACLE_OK;", "        *out = len - (len > 1);\n        return ORACLE_OK;"),
    ("merge-compare", "if (a[i] < b[j]) i++;", "if (a[i] <= b[j]) i++;"),
    ("penultimate-drop-last", "part = intersect(C, len, na, da, NULL);", "part = intersect(C, len, na, da ? da - 1 : 0, NULL);"),
    ("recursion-depth", "int st = cnt(g, next, len2, r - 1, levels + 1, &part);", "int st = cnt(g, next, len2, r - 2 > 0 ? r - 2 : 1, levels + 1, &part);"),
    ("root-level", "st = cnt(p->g, nu, du, p->k - 1, levels, &c);", "st = cnt(p->g, nu, du, p->k, levels, &c);"),
    ("fill-transposed", "if (degree_before(off, u, cols[e])) dag_cols[pos++] = cols[e];", "if (degree_before(off, cols[e], u)) dag_cols[pos++] = cols[e];"),
    ("rounds-level-falls", "if (least > level) level = least;", "level = least;"),
    ("rounds-stale-members", "                now[u] = 0;\n", ""),
    ("list-depth", "int depth = L->k - r; /* vertices already chosen */", "int depth = L->k - r - (r > 2);"),
    ("per-root-slot", "if (p->per_root) p->per_root[t] = c;", "if (p->per_root) p->per_root[u % p->nroots] = c;"),
    ("per-edge-slot", "st = cnt(&g, levels[0], len, k - 2, levels + 1, &per_edge[e]);",
     "st = cnt(&g, levels[0], len, k - 2, levels + 1, &per_edge[dag_off[u] + dag_off[u + 1] - 1 - e]);"),
    ("arc-row-search", "if (dag_off[mid] <= e) lo = mid;", "if (dag_off[mid] < e) lo = mid;"),
    ("prefix-sum", "for (uint32_t u = 0; u < n; u++) dag_off[u + 1] = dag_off[u] + count[u];", "for (uint32_t u = 0; u < n; u++) dag_off[u + 1] = dag_off[u] + count[u] - (count[u] > 2);"),
]


def build_mutant(tmp: Path, name: str, a: str, b: str) -> ctypes.CDLL:
    text = SRC.read_text()
    assert text.count(a) == 1, name
    src = tmp / f"m_{name}.c"
    src.write_text(text.replace(a, b))
    so = tmp / f"m_{name}.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-pthread", "-shared", "-fPIC", "-o", str(so), str(src)], check=True)
    return so


def pins_hold() -> bool:
    """A compact battery of the pins in test_oracle_pins (Fig. 1, closed forms, brute force)."""
    try:
        g = gg.fig1()
        off, cols = oracle.gen_ordering(g.off, g.cols, g.n)
        arcs = {(u, v) for u in range(g.n) for v in cols[off[u]: off[u + 1]].tolist()}
        if arcs != {(0, 1), (0, 3), (0, 4), (3, 1), (1, 4), (2, 1), (2, 5), (3, 4), (5, 4), (6, 4), (6, 5)}:
            return False
        if [oracle.count_graph(g, k, threads=1) for k in range(1, 6)] != [7, 11, 5, 1, 0]:
            return False
        for n in (6, 11):
            if [oracle.count_graph(gg.complete(n), k, threads=1) for k in range(1, n + 1)] != \
                    [math.comb(n, k) for k in range(1, n + 1)]:
                return False
        parts = [4, 3, 3, 2]
        g = gg.complete_multipartite(parts)
        if oracle.count_graph(g, 3, threads=1) != 4 * 3 * 3 + 4 * 3 * 2 + 4 * 3 * 2 + 3 * 3 * 2:
            return False
        # core ordering by rounds: a hand-worked example and the degeneracy on random graphs
        g = gg.csr_from_edges(6, np.array([0, 0, 0, 1, 1, 2, 3, 4], dtype=np.uint32),
                              np.array([1, 2, 3, 2, 3, 3, 4, 5], dtype=np.uint32))
        rank, level, rounds = oracle.core_rank_rounds(g.off, g.cols, g.n)
        if rank.tolist() != [2, 3, 4, 5, 1, 0] or level != 3 or rounds != 3:
            return False
        for seed in (1, 2, 3, 4, 5):
            g = gg.random_small(seed, 12, 0.4)
            rank, level, _ = oracle.core_rank_rounds(g.off, g.cols, g.n)
            off, _ = oracle.dag_by_rank(g.off, g.cols, g.n, rank, relabel=False)
            if not int(np.diff(off).max()) == level == degeneracy(g):
                return False
        # listing: every row a distinct clique, as many as the brute-force count
        g = gg.random_small(2, 12, 0.6)
        off, cols = oracle.gen_ordering(g.off, g.cols, g.n)
        adj = [set(g.cols[g.off[v]: g.off[v + 1]].tolist()) for v in range(g.n)]
        for k in (3, 4, 5):
            rows = [tuple(r.tolist()) for r in oracle.list_cliques(off, cols, g.n, k)]
            want = sum(1 for s in itertools.combinations(range(g.n), k)
                       if all(b in adj[a] for a, b in itertools.combinations(s, 2)))
            if len(rows) != want or len({frozenset(r) for r in rows}) != want:
                return False
            if any(b not in adj[a] for r in rows for a, b in itertools.combinations(r, 2)):
                return False
        # per-root values for a shuffled subset of roots, and per-edge values, against brute
        # force: cliques whose first (first two) vertices in the degree order they are
        g = gg.random_small(7, 13, 0.6)
        off, cols = oracle.gen_ordering(g.off, g.cols, g.n)
        adj = [set(g.cols[g.off[v]: g.off[v + 1]].tolist()) for v in range(g.n)]
        deg = np.diff(g.off)
        roots = np.array([5, 11, 0, 7, 2, 9, 12, 3], dtype=np.uint32)
        for k in (3, 4):
            want_root, want_edge = [0] * g.n, {}
            for s in itertools.combinations(range(g.n), k):
                if all(b in adj[a] for a, b in itertools.combinations(s, 2)):
                    o = sorted(s, key=lambda v: (int(deg[v]), v))
                    want_root[o[0]] += 1
                    want_edge[(o[0], o[1])] = want_edge.get((o[0], o[1]), 0) + 1
            _, pr = oracle.count_roots(off, cols, g.n, k, roots, threads=1, per_root=True)
            if [int(x) for x in pr] != [want_root[r] for r in roots]:
                return False
            pe = oracle.count_per_edge(off, cols, g.n, k)
            got_edge = {(u, int(cols[e])): int(pe[e]) for u in range(g.n)
                        for e in range(int(off[u]), int(off[u + 1])) if pe[e]}
            if got_edge != want_edge:
                return False
            # the arc-subset form on a shuffled subset of arcs (the CPU baseline's unit)
            sub = np.random.default_rng(3).permutation(int(off[-1]))[: int(off[-1]) // 2 + 1]
            tot, pa = oracle.count_arcs(off, cols, g.n, k, sub.astype(np.uint64), per_arc=True)
            arc_of = {e: (u, int(cols[e])) for u in range(g.n) for e in range(int(off[u]), int(off[u + 1]))}
            if [int(x) for x in pa] != [want_edge.get(arc_of[int(e)], 0) for e in sub]:
                return False
            if tot != sum(want_edge.get(arc_of[int(e)], 0) for e in sub):
                return False
        return True
    except Exception:
        return False


def degeneracy(g) -> int:
    """Largest minimum degree over all induced subgraphs (brute force, n <= 12)."""
    adj = [set(g.cols[g.off[v]: g.off[v + 1]].tolist()) for v in range(g.n)]
    best = 0
    for mask in range(1, 1 << g.n):
        s = {v for v in range(g.n) if mask >> v & 1}
        best = max(best, min(len(adj[v] & s) for v in s))
    return best


def test_unmutated_oracle_passes_battery():
    assert pins_hold()


@pytest.mark.parametrize("name,a,b", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, monkeypatch, name, a, b):
    so = build_mutant(tmp_path, name, a, b)
    saved = oracle._lib
    try:
        oracle._lib = None
        monkeypatch.setattr(oracle, "_LIB", so)
        monkeypatch.setattr(oracle, "build", lambda force=False: so)
        assert not pins_hold(), f"mutant {name} survived the pins"
    finally:
        oracle._lib = saved
