"""Python handle on the oracle (plain C, built with gcc, loaded with ctypes).

TEST INFRASTRUCTURE ONLY.  The oracle is the slow, obviously correct CPU restatement of the
paper's method that the CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package; the product path never does.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "citron_oracle.c"
_LIB = _HERE / "libcitron_oracle.so"

ERRORS = {
    0: "ok",
    1: "bad offsets",
    2: "vertex id out of range",
    3: "row unsorted or duplicate",
    4: "self-loop",
    5: "asymmetric",
    6: "uint64 overflow",
    7: "out of memory",
    8: "bad argument",
}


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> Path:
    """Compile the oracle into a shared library next to its source."""
    if force or not _LIB.exists() or _LIB.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB.with_suffix(f".{os.getpid()}.tmp")
        subprocess.run(["gcc", "-O2", "-std=c11", "-pthread", "-shared", "-fPIC", "-o", str(tmp),
                        str(_SRC)], check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(str(_LIB))
        p = ctypes.c_void_p
        u32, i32, u64 = ctypes.c_uint32, ctypes.c_int, ctypes.c_uint64
        L.oracle_validate.argtypes = [u32, p, p]
        L.oracle_validate.restype = i32
        L.oracle_degree_rank.argtypes = [u32, p, p]
        L.oracle_degree_rank.restype = None
        L.oracle_gen_ordering.argtypes = [u32, p, p, p, p]
        L.oracle_gen_ordering.restype = None
        L.oracle_dag_by_rank.argtypes = [u32, p, p, p, i32, p, p]
        L.oracle_dag_by_rank.restype = None
        L.oracle_core_rank.argtypes = [u32, p, p, p]
        L.oracle_core_rank.restype = None
        L.oracle_list.argtypes = [u32, p, p, i32, p, u64, p]
        L.oracle_list.restype = i32
        L.oracle_core_rank_rounds.argtypes = [u32, p, p, p, p, p]
        L.oracle_core_rank_rounds.restype = None
        L.oracle_count.argtypes = [u32, p, p, i32, i32, p]
        L.oracle_count.restype = i32
        L.oracle_count_roots.argtypes = [u32, p, p, i32, p, u64, i32, p, p]
        L.oracle_count_roots.restype = i32
        L.oracle_count_per_edge.argtypes = [u32, p, p, i32, p]
        L.oracle_count_per_edge.restype = i32
        L.oracle_count_arcs.argtypes = [u32, p, p, i32, p, u64, p, p]
        L.oracle_count_arcs.restype = i32
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a.size else ctypes.c_void_p(0)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _check(st: int):
    if st:
        raise OracleError(ERRORS.get(st, f"error {st}"))


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)))


def validate(off, cols, n: int) -> int:
    off, cols = _c(off, np.uint64), _c(cols, np.uint32)
    return int(lib().oracle_validate(n, _ptr(off), _ptr(cols)))


def degree_rank(off, n: int) -> np.ndarray:
    off = _c(off, np.uint64)
    rank = np.zeros(n, dtype=np.uint32)
    lib().oracle_degree_rank(n, _ptr(off), _ptr(rank))
    return rank


def core_rank(off, cols, n: int) -> np.ndarray:
    off, cols = _c(off, np.uint64), _c(cols, np.uint32)
    rank = np.zeros(n, dtype=np.uint32)
    lib().oracle_core_rank(n, _ptr(off), _ptr(cols), _ptr(rank))
    return rank


def core_rank_rounds(off, cols, n: int):
    """Core ordering by synchronous peeling rounds: (rank, degeneracy, rounds)."""
    off, cols = _c(off, np.uint64), _c(cols, np.uint32)
    rank = np.zeros(n, dtype=np.uint32)
    level, rounds = ctypes.c_uint32(0), ctypes.c_uint32(0)
    lib().oracle_core_rank_rounds(n, _ptr(off), _ptr(cols), _ptr(rank), ctypes.byref(level),
                                  ctypes.byref(rounds))
    return rank, int(level.value), int(rounds.value)


def gen_ordering(off, cols, n: int):
    """DAG of the degree ordering in the input's vertex ids (Algorithm GenOrdering)."""
    off, cols = _c(off, np.uint64), _c(cols, np.uint32)
    dag_off = np.zeros(n + 1, dtype=np.uint64)
    dag_cols = np.zeros(max(1, cols.size // 2), dtype=np.uint32)
    lib().oracle_gen_ordering(n, _ptr(off), _ptr(cols), _ptr(dag_off), _ptr(dag_cols))
    return dag_off, dag_cols[: int(dag_off[-1])]


def dag_by_rank(off, cols, n: int, rank, relabel: bool):
    off, cols, rank = _c(off, np.uint64), _c(cols, np.uint32), _c(rank, np.uint32)
    dag_off = np.zeros(n + 1, dtype=np.uint64)
    dag_cols = np.zeros(max(1, cols.size // 2), dtype=np.uint32)
    lib().oracle_dag_by_rank(n, _ptr(off), _ptr(cols), _ptr(rank), int(relabel), _ptr(dag_off),
                             _ptr(dag_cols))
    return dag_off, dag_cols[: int(dag_off[-1])]


def count(dag_off, dag_cols, n: int, k: int, threads: int | None = None) -> int:
    dag_off, dag_cols = _c(dag_off, np.uint64), _c(dag_cols, np.uint32)
    out = np.zeros(1, dtype=np.uint64)
    _check(lib().oracle_count(n, _ptr(dag_off), _ptr(dag_cols), k, threads or default_threads(),
                              _ptr(out)))
    return int(out[0])


def count_roots(dag_off, dag_cols, n: int, k: int, roots, threads: int | None = None,
                per_root: bool = False):
    dag_off, dag_cols, roots = _c(dag_off, np.uint64), _c(dag_cols, np.uint32), _c(roots, np.uint32)
    out = np.zeros(1, dtype=np.uint64)
    pr = np.zeros(max(1, roots.size), dtype=np.uint64)
    _check(lib().oracle_count_roots(n, _ptr(dag_off), _ptr(dag_cols), k, _ptr(roots), roots.size,
                                    threads or default_threads(), _ptr(pr), _ptr(out)))
    return (int(out[0]), pr[: roots.size]) if per_root else int(out[0])


def list_cliques(dag_off, dag_cols, n: int, k: int, capacity: int | None = None) -> np.ndarray:
    """Every k-clique as a row of k DAG ids in recursion order (root first); shape (K_k, k)."""
    dag_off, dag_cols = _c(dag_off, np.uint64), _c(dag_cols, np.uint32)
    total = ctypes.c_uint64(0)
    if capacity is None:
        _check(lib().oracle_list(n, _ptr(dag_off), _ptr(dag_cols), k, None, 0, ctypes.byref(total)))
        capacity = int(total.value)
    out = np.zeros((max(1, capacity), k), dtype=np.uint32)
    _check(lib().oracle_list(n, _ptr(dag_off), _ptr(dag_cols), k, _ptr(out), capacity,
                             ctypes.byref(total)))
    return out[: min(capacity, int(total.value))]


def count_per_edge(dag_off, dag_cols, n: int, k: int) -> np.ndarray:
    dag_off, dag_cols = _c(dag_off, np.uint64), _c(dag_cols, np.uint32)
    out = np.zeros(max(1, dag_cols.size), dtype=np.uint64)
    _check(lib().oracle_count_per_edge(n, _ptr(dag_off), _ptr(dag_cols), k, _ptr(out)))
    return out[: dag_cols.size]


def count_arcs(dag_off, dag_cols, n: int, k: int, arcs, per_arc: bool = False):
    """Edge tasks of the listed DAG arc indices (k >= 3), on one thread: their total and, with
    per_arc, the count of each (the entries of count_per_edge at those arcs)."""
    dag_off, dag_cols, arcs = _c(dag_off, np.uint64), _c(dag_cols, np.uint32), _c(arcs, np.uint64)
    out = np.zeros(1, dtype=np.uint64)
    pa = np.zeros(max(1, arcs.size), dtype=np.uint64)
    _check(lib().oracle_count_arcs(n, _ptr(dag_off), _ptr(dag_cols), k, _ptr(arcs), arcs.size, _ptr(pa),
                                   _ptr(out)))
    return (int(out[0]), pa[: arcs.size]) if per_arc else int(out[0])


def count_graph(g, k: int, threads: int | None = None) -> int:
    """K_k of a CSR graph by the paper's pipeline: degree ordering -> GenOrdering DAG -> Counting."""
    if k == 1:
        return g.n
    dag_off, dag_cols = gen_ordering(g.off, g.cols, g.n)
    return count(dag_off, dag_cols, g.n, k, threads)
