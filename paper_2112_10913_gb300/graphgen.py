"""Seeded synthetic input graphs (shared by the CUDA path, the oracle tests and the bench).

This module only *makes inputs*: random draws, edge lists and the undirected CSR that both sides
consume.  It holds none of the method's arithmetic (no ordering, no orientation, no counting).

Random numbers come from one counter-based generator, SplitMix64 (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): draw ``i`` of stream ``s`` under
seed ``x`` is ``mix(key(x, s) + (i + 1) * GAMMA)``.  Everything is vectorised numpy uint64
arithmetic, so the same seed gives the same graph on any machine and numpy version.

CSR convention (the paper's input, Sec. II and Sec. VI-B): undirected, symmetrised, unweighted,
no self-loops, no duplicate edges, neighbour lists sorted ascending; ``off`` is uint64[n+1],
``cols`` is uint32[2m] (every undirected edge appears as two arcs).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (vectorised, wraps mod 2^64)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> np.uint64:
    """Key of an independent stream: two SplitMix64 steps over (seed, stream)."""
    with np.errstate(over="ignore"):
        a = _mix(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64) + GAMMA)
        b = _mix(a ^ (np.uint64(stream & 0xFFFFFFFFFFFFFFFF) * _M2 + GAMMA))
    return np.uint64(b[0])


def draws_u64(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """``count`` raw 64-bit draws of stream ``stream`` beginning at counter ``start``."""
    key = stream_key(seed, stream)
    idx = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(key + idx * GAMMA)


def uniform(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of each draw."""
    return (draws_u64(seed, stream, count, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def below(seed: int, stream: int, count: int, bound: int, start: int = 0) -> np.ndarray:
    """Integers in [0, bound) by multiply-shift of the top 32 bits (bound < 2^32)."""
    assert 0 < bound < (1 << 32)
    hi = draws_u64(seed, stream, count, start) >> np.uint64(32)
    with np.errstate(over="ignore"):
        return ((hi * np.uint64(bound)) >> np.uint64(32)).astype(np.int64)


def splitmix_child(seed: int, i: int) -> int:
    """Per-item seed SplitMix64(seed, i) used for families of graphs (batches, request streams)."""
    return int(draws_u64(seed, 0x5EED, 1, start=i)[0])


def permutation(seed: int, stream: int, n: int) -> np.ndarray:
    """Seeded uniform random permutation of range(n) (argsort of 64-bit keys, stable on ties)."""
    return np.argsort(draws_u64(seed, stream, n), kind="stable").astype(np.int64)


# --------------------------------------------------------------------------------------------
# CSR container and construction


@dataclass
class Csr:
    """Undirected CSR: ``off`` uint64[n+1], ``cols`` uint32[2m], rows sorted, symmetric."""

    n: int
    off: np.ndarray
    cols: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def arcs(self) -> int:
        return int(self.off[-1])

    @property
    def m(self) -> int:
        """Number of undirected edges."""
        return self.arcs // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.off).astype(np.int64)

    def nbytes(self) -> int:
        return self.off.nbytes + self.cols.nbytes


def csr_from_edges(n: int, src, dst, name: str = "", meta: dict | None = None) -> Csr:
    """Symmetrise, drop self-loops, deduplicate and sort an edge list into a CSR."""
    if n >= (1 << 32) - 1:
        raise ValueError("vertex ids must fit uint32 with one value spare")
    src = np.asarray(src, dtype=np.uint64)
    dst = np.asarray(dst, dtype=np.uint64)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    nn = np.uint64(n)
    with np.errstate(over="ignore"):
        keys = np.concatenate([src * nn + dst, dst * nn + src])
    del src, dst, keep
    keys.sort()
    if keys.size:
        first = np.empty(keys.size, dtype=bool)
        first[0] = True
        np.not_equal(keys[1:], keys[:-1], out=first[1:])
        keys = keys[first]
    rows = (keys // nn).astype(np.int64)
    cols = (keys % nn).astype(np.uint32)
    del keys
    counts = np.bincount(rows, minlength=n)
    off = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(counts, out=off[1:])
    return Csr(n=n, off=off, cols=cols, name=name, meta=dict(meta or {}))


def edges_of(g: Csr) -> tuple[np.ndarray, np.ndarray]:
    """Undirected edge list (u < v) of a CSR."""
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.off).astype(np.int64))
    cols = g.cols.astype(np.int64)
    keep = rows < cols
    return rows[keep], cols[keep]


def relabel(g: Csr, perm: np.ndarray, name: str | None = None) -> Csr:
    """Rename vertex ``v`` to ``perm[v]`` (a permutation of range(n))."""
    u, v = edges_of(g)
    perm = np.asarray(perm, dtype=np.int64)
    return csr_from_edges(g.n, perm[u], perm[v], name=name or g.name + "+relabel", meta=g.meta)


def disjoint_union(graphs: list[Csr], name: str = "union") -> Csr:
    """Vertex-disjoint union; graph i's vertices are shifted by the sizes before it."""
    us, vs, base = [], [], 0
    for g in graphs:
        u, v = edges_of(g)
        us.append(u + base)
        vs.append(v + base)
        base += g.n
    return csr_from_edges(base, np.concatenate(us), np.concatenate(vs), name=name)


# --------------------------------------------------------------------------------------------
# Deterministic families with known clique counts


def fig1() -> Csr:
    """The 7-vertex, 11-edge example graph of Fig. 1 (Sec. II)."""
    e = [(0, 1), (0, 3), (0, 4), (1, 3), (1, 4), (1, 2), (2, 5), (3, 4), (4, 6), (4, 5), (5, 6)]
    u, v = zip(*e)
    return csr_from_edges(7, u, v, name="fig1")


def complete(n: int) -> Csr:
    """Complete graph K_n."""
    iu, ju = np.triu_indices(n, 1)
    return csr_from_edges(n, iu, ju, name=f"K{n}")


def complete_multipartite(parts: list[int]) -> Csr:
    """Complete multipartite graph: vertices in different parts are adjacent (Turan graphs)."""
    label = np.repeat(np.arange(len(parts)), parts)
    n = int(sum(parts))
    iu, ju = np.triu_indices(n, 1)
    keep = label[iu] != label[ju]
    return csr_from_edges(n, iu[keep], ju[keep], name="multipartite" + "-".join(map(str, parts)))


def turan(n: int, r: int) -> Csr:
    """Turan graph T(n, r): complete r-partite with part sizes as equal as possible."""
    parts = [n // r + (1 if i < n % r else 0) for i in range(r)]
    g = complete_multipartite(parts)
    g.name = f"T({n},{r})"
    return g


def cocktail_party(r: int) -> Csr:
    """Cocktail-party graph CP(r) = K_{2,2,...,2} with r parts."""
    g = complete_multipartite([2] * r)
    g.name = f"CP({r})"
    return g


# --------------------------------------------------------------------------------------------
# Random families shaped like the paper's sparse real-world inputs (Table I)


def erdos_renyi_gnp(n: int, p: float, seed: int, stream: int = 1) -> tuple[np.ndarray, np.ndarray]:
    """G(n, p) over all n(n-1)/2 pairs (for small n): pair i<j kept when its draw is < p."""
    iu, ju = np.triu_indices(n, 1)
    keep = uniform(seed, stream, iu.size) < p
    return iu[keep], ju[keep]


def erdos_renyi_gnm_draws(n: int, draws: int, seed: int, stream: int = 1):
    """``draws`` uniform endpoint pairs with replacement (loops and repeats removed later)."""
    u = below(seed, stream, draws, n)
    v = below(seed, stream + 1, draws, n)
    return u, v


def planted(n: int, size: int, seed: int, stream: int) -> tuple[np.ndarray, np.ndarray]:
    """All pairs of ``size`` distinct uniform vertices (a planted clique)."""
    verts = permutation(seed, stream, n)[:size]
    iu, ju = np.triu_indices(size, 1)
    return verts[iu], verts[ju]


def rmat_draws(scale: int, draws: int, abcd, seed: int, stream: int = 10):
    """R-MAT endpoint pairs: ``scale`` quadrant choices per edge with probabilities (a,b,c,d).

    Each 64-bit draw serves two levels: its high and low 32-bit halves are compared with the
    cumulative thresholds a, a+b, a+b+c scaled to 2^32."""
    a, b, c, _ = abcd
    t1, t2, t3 = (np.uint64(int(x * 2.0 ** 32)) for x in (a, a + b, a + b + c))
    src = np.zeros(draws, dtype=np.uint32)
    dst = np.zeros(draws, dtype=np.uint32)
    mask32 = np.uint64(0xFFFFFFFF)
    for pair in range((scale + 1) // 2):
        x = draws_u64(seed, stream + pair, draws)
        for half, level in ((x >> np.uint64(32), 2 * pair), (x & mask32, 2 * pair + 1)):
            if level >= scale:
                break
            half = half.astype(np.uint32)
            shift = np.uint32(scale - 1 - level)
            down = half >= np.uint32(t2)  # quadrants c and d
            right = (half >= np.uint32(t1)) != down
            right ^= half >= np.uint32(t3)  # quadrants b and d
            src |= down.astype(np.uint32) << shift
            dst |= right.astype(np.uint32) << shift
    src = src.astype(np.int64)
    dst = dst.astype(np.int64)
    return src, dst


def chung_lu_weights(n: int, beta: float, mean_deg: float, cap: float) -> np.ndarray:
    """w_i proportional to (i+1)^(-1/(beta-1)), scaled so mean(min(w, cap)) = mean_deg, capped."""
    base = np.arange(1, n + 1, dtype=np.float64) ** (-1.0 / (beta - 1.0))
    lo, hi = 0.0, 1.0
    while np.minimum(base * hi, cap).mean() < mean_deg:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if np.minimum(base * mid, cap).mean() < mean_deg:
            lo = mid
        else:
            hi = mid
    return np.minimum(base * hi, cap)


def chung_lu_draws(w: np.ndarray, draws: int, seed: int, stream: int = 30):
    """Endpoint pairs, each endpoint drawn with probability proportional to its weight."""
    cum = np.cumsum(w)
    total = cum[-1]
    out = []
    for s in (stream, stream + 1):
        x = uniform(seed, s, draws) * total
        idx = np.searchsorted(cum, x, side="right")
        np.minimum(idx, w.size - 1, out=idx)
        out.append(idx.astype(np.int64))
    return out[0], out[1]


# --------------------------------------------------------------------------------------------
# The five workloads (sizes of the paper-shaped configurations)


def config1_er_planted(seed: int = 1, n: int = 2000, avg_deg: float = 20.0, clique: int = 12) -> Csr:
    """ER G(n, p=avg_deg/(n-1)) plus one planted K_clique on distinct uniform vertices."""
    u, v = erdos_renyi_gnp(n, avg_deg / (n - 1), seed, stream=1)
    pu, pv = planted(n, clique, seed, stream=2)
    return csr_from_edges(n, np.concatenate([u, pu]), np.concatenate([v, pv]),
                          name=f"er{n}+K{clique}", meta=dict(seed=seed, planted=[clique]))


def config2_rmat(seed: int = 2, scale: int = 20, edge_factor: int = 16,
                 abcd=(0.57, 0.19, 0.19, 0.05)) -> Csr:
    """R-MAT scale/edge factor, no noise, seeded vertex-id permutation, dedup, symmetrised."""
    n = 1 << scale
    src, dst = rmat_draws(scale, edge_factor * n, abcd, seed)
    perm = permutation(seed, 99, n)
    return csr_from_edges(n, perm[src], perm[dst], name=f"rmat{scale}-ef{edge_factor}",
                          meta=dict(seed=seed, scale=scale, edge_factor=edge_factor))


def config3_chung_lu(seed: int = 3, n: int = 4_000_000, beta: float = 2.1, mean_deg: float = 30.0,
                     cap: float = 20_000.0, cliques: int = 50, clique_range=(20, 40)) -> Csr:
    """Chung-Lu power law (fast endpoint-pair model) plus planted cliques, seeded permutation."""
    w = chung_lu_weights(n, beta, mean_deg, cap)
    draws = int(n * mean_deg / 2)
    u, v = chung_lu_draws(w, draws, seed)
    sizes = clique_range[0] + below(seed, 40, cliques, clique_range[1] - clique_range[0] + 1)
    us, vs = [u], [v]
    for i, s in enumerate(sizes):
        pu, pv = planted(n, int(s), seed, stream=1000 + i)
        us.append(pu)
        vs.append(pv)
    perm = permutation(seed, 99, n)
    u = perm[np.concatenate(us)]
    v = perm[np.concatenate(vs)]
    return csr_from_edges(n, u, v, name=f"chunglu{n}-b{beta}",
                          meta=dict(seed=seed, planted=[int(s) for s in sizes]))


def small_rmat(seed: int, n: int, avg_deg: float, abcd=(0.57, 0.19, 0.19, 0.05)) -> Csr:
    """R-MAT at scale ceil(log2 n) with endpoints >= n rejected, redrawn until the target count."""
    scale = max(1, math.ceil(math.log2(max(n, 2))))
    target = int(round(n * avg_deg / 2))
    us, vs, have, stream = [], [], 0, 10
    while have < target:
        want = max(64, int((target - have) * 1.3))
        s, d = rmat_draws(scale, want, abcd, seed, stream=stream)
        keep = (s < n) & (d < n)
        us.append(s[keep])
        vs.append(d[keep])
        have += int(keep.sum())
        stream += scale
    u = np.concatenate(us)[:target]
    v = np.concatenate(vs)[:target]
    perm = permutation(seed, 99, n)
    return csr_from_edges(n, perm[u], perm[v], name=f"rmat-n{n}", meta=dict(seed=seed))


def small_er(seed: int, n: int, avg_deg: float) -> Csr:
    """Sparse ER by uniform endpoint-pair draws (n * avg_deg / 2 draws, loops/repeats removed)."""
    u, v = erdos_renyi_gnm_draws(n, int(round(n * avg_deg / 2)), seed)
    return csr_from_edges(n, u, v, name=f"er-n{n}", meta=dict(seed=seed))


@dataclass
class BatchItem:
    graph: Csr
    k: int


def config4_batch(seed: int = 4, count: int = 4096, n_range=(50, 50_000), deg_range=(8.0, 64.0),
                  k_range=(3, 7)) -> list[BatchItem]:
    """Many small graphs: n log-uniform, ER/R-MAT half and half, avg degree and k uniform."""
    return [_batch_item((seed, i, n_range, deg_range, k_range)) for i in range(count)]


def _batch_item(args):
    seed, i, n_range, deg_range, k_range = args
    s = splitmix_child(seed, i)
    ln = math.log(n_range[0]) + uniform(s, 1, 1)[0] * (math.log(n_range[1]) - math.log(n_range[0]))
    n = int(round(math.exp(ln)))
    deg = deg_range[0] + uniform(s, 2, 1)[0] * (deg_range[1] - deg_range[0])
    deg = min(deg, n - 1)
    k = int(k_range[0] + below(s, 3, 1, k_range[1] - k_range[0] + 1)[0])
    g = small_er(s, n, deg) if below(s, 4, 1, 2)[0] == 0 else small_rmat(s, n, deg)
    return BatchItem(g, k)


def config4_batch_parallel(seed: int = 4, count: int = 4096, n_range=(50, 50_000),
                           deg_range=(8.0, 64.0), k_range=(3, 7), workers: int | None = None):
    """config4_batch with the graphs generated by a pool of processes (spawned, so it is safe
    to call at any time); the result is identical to config4_batch."""
    import multiprocessing as mp
    import os

    workers = workers or max(1, min(32, len(os.sched_getaffinity(0))))
    args = [(seed, i, n_range, deg_range, k_range) for i in range(count)]
    if workers == 1:
        return [_batch_item(a) for a in args]
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_batch_item, args, chunksize=8)


def random_small(seed: int, n: int, p: float) -> Csr:
    """G(n, p) for brute-force checks on tiny graphs."""
    u, v = erdos_renyi_gnp(n, p, seed, stream=7)
    return csr_from_edges(n, u, v, name=f"gnp{n}-{p}")
