"""GB300 (sm_103a) k-clique counter: the ordering-based method of arXiv 2112.10913 (CITRON).

The compute lives in ``libcitron.so`` (hand-written CUDA, C ABI declared in ``include/citron.h``).
This module is the thin Python binding: it marshals torch tensors (device memory) and CUDA
stream handles into the C calls of the same names and turns status codes into exceptions.
It has no CPU fallback: without the built library every call raises.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import numpy as np

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "libcitron.so"
MAX_K = 12

STATUS = {
    0: "CITRON_OK",
    1: "CITRON_E_INVALID",
    2: "CITRON_E_WORKSPACE",
    3: "CITRON_E_CUDA",
    4: "CITRON_E_OVERFLOW",
    5: "CITRON_E_TIMEOUT",
    6: "CITRON_E_UNSUPPORTED",
    7: "CITRON_E_BUDGET",
}

# Every function the C ABI exports (checked against include/citron.h by the tests).
EXPORTS = (
    "citron_status_str",
    "citron_last_cuda_error",
    "citron_version",
    "citron_workspace_bytes",
    "citron_validate",
    "citron_order",
    "citron_order_grouped",
    "citron_core_order",
    "citron_build_dag",
    "citron_count",
    "citron_count_ex",
    "citron_list",
    "citron_kernel_launches",
    "citron_host_buffer_bytes",
    "citron_count_host",
    "citron_count_noalloc",
    "citron_count_batch",
    "citron_workspace_status",
    "citron_dag_append",
    "citron_set_faults",
    "citron_probe_word_ops",
)

COUNT_TIME_KERNELS = 1
COUNT_WORK = 2
COUNT_BALANCE = 4


class CountOpts(ctypes.Structure):
    """Mirror of citron_count_opts (include/citron.h)."""

    _fields_ = [
        ("small_max", ctypes.c_uint32),
        ("bitmap_max", ctypes.c_uint32),
        ("warps_per_cta", ctypes.c_uint32),
        ("flags", ctypes.c_uint32),
        ("compact_max", ctypes.c_uint32),
        ("max_blocks", ctypes.c_uint32),
        ("d_per_root", ctypes.c_void_p),
        ("work_ops", ctypes.c_uint64),
        ("kernel_ms", ctypes.c_float * 3),
        ("split_min", ctypes.c_uint32),
        ("busy_ms", ctypes.c_float * 2),
        ("budget_ms", ctypes.c_uint32),
        ("d_per_arc", ctypes.c_void_p),
    ]


class Faults(ctypes.Structure):
    """Mirror of citron_faults (include/citron.h): fault injection for error-path tests."""

    _fields_ = [
        ("lookback_spin_limit", ctypes.c_uint32),
        ("lookback_stall_tile", ctypes.c_uint32),
        ("barrier_wait_ns", ctypes.c_uint64),
        ("barrier_absent_block", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32),
        ("count_seed", ctypes.c_uint64),
    ]


class CitronError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        self.name = STATUS.get(code, f"status {code}")
        detail = ""
        if self.name == "CITRON_E_CUDA" and _lib is not None:
            detail = f" ({_lib.citron_last_cuda_error().decode()})"
        super().__init__(f"{where}: {self.name}{detail}")


_lib = None


def lib() -> ctypes.CDLL:
    """Load libcitron.so (built by ``paper_2112_10913_gb300.build``); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not LIB_PATH.exists():
        raise RuntimeError(f"{LIB_PATH} is not built: run paper_2112_10913_gb300.build.build() "
                           "(needs nvcc); there is no fallback implementation")
    L = ctypes.CDLL(str(LIB_PATH))
    vp, u32, u64, sz, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_size_t, ctypes.c_int
    L.citron_status_str.argtypes = [i32]
    L.citron_status_str.restype = ctypes.c_char_p
    L.citron_last_cuda_error.argtypes = []
    L.citron_last_cuda_error.restype = ctypes.c_char_p
    L.citron_version.argtypes = []
    L.citron_version.restype = i32
    L.citron_workspace_bytes.argtypes = [u32, u64, u32]
    L.citron_workspace_bytes.restype = sz
    L.citron_validate.argtypes = [u32, u64, vp, vp, vp, vp, sz, vp]
    L.citron_validate.restype = i32
    L.citron_order.argtypes = [u32, vp, vp, vp, vp, sz, vp]
    L.citron_order.restype = i32
    L.citron_order_grouped.argtypes = [u32, vp, vp, u32, vp, vp, vp, sz, vp]
    L.citron_order_grouped.restype = i32
    L.citron_core_order.argtypes = [u32, u64, vp, vp, vp, vp, vp, vp, vp, sz, vp]
    L.citron_core_order.restype = i32
    L.citron_build_dag.argtypes = [u32, u64, vp, vp, vp, vp, vp, vp, vp, sz, vp]
    L.citron_build_dag.restype = i32
    L.citron_count.argtypes = [u32, vp, vp, u32, u32, vp, vp, vp, sz, vp]
    L.citron_count.restype = i32
    L.citron_count_ex.argtypes = [u32, vp, vp, u32, u32, vp, vp, vp, sz, vp]
    L.citron_count_ex.restype = i32
    L.citron_list.argtypes = [u32, vp, vp, u32, vp, vp, u64, vp, vp, sz, vp]
    L.citron_list.restype = i32
    L.citron_kernel_launches.argtypes = []
    L.citron_kernel_launches.restype = u64
    L.citron_host_buffer_bytes.argtypes = [u32, u64]
    L.citron_host_buffer_bytes.restype = sz
    L.citron_count_host.argtypes = [u32, u64, vp, vp, vp, u32, vp, vp, sz, vp, sz, vp]
    L.citron_count_host.restype = i32
    L.citron_count_noalloc.argtypes = [u32, vp, vp, u32, vp, vp]
    L.citron_count_noalloc.restype = i32
    L.citron_count_batch.argtypes = [u32, vp, vp, vp, vp, vp, u32, u32, u32, vp, vp, vp, sz, vp]
    L.citron_count_batch.restype = i32
    L.citron_workspace_status.argtypes = [vp, vp]
    L.citron_workspace_status.restype = i32
    L.citron_dag_append.argtypes = [u32, vp, vp, u32, vp, vp, u32, u64, vp]
    L.citron_dag_append.restype = i32
    L.citron_set_faults.argtypes = [vp]
    L.citron_set_faults.restype = i32
    L.citron_probe_word_ops.argtypes = [u32, u32, vp, vp, vp]
    L.citron_probe_word_ops.restype = i32
    _lib = L
    return L


def _check(code: int, where: str):
    if code != 0:
        raise CitronError(code, where)


def _dptr(t) -> ctypes.c_void_p:
    """Device pointer of a CUDA tensor (None -> NULL)."""
    if t is None:
        return ctypes.c_void_p(0)
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream))


def _nbytes(t) -> int:
    return t.numel() * t.element_size()


# ---------------------------------------------------------------------------------------------
# Entry points (same names as the C ABI)


def citron_workspace_bytes(n: int, arcs: int, max_outdeg: int = 0) -> int:
    return int(lib().citron_workspace_bytes(n, arcs, max_outdeg))


def alloc_workspace(n: int, arcs: int, max_outdeg: int = 0, device="cuda"):
    """Zero-initialised device workspace (uint8 tensor, 256-byte aligned)."""
    import torch

    ws = torch.zeros(citron_workspace_bytes(n, arcs, max_outdeg) + 256, dtype=torch.uint8, device=device)
    pad = (-ws.data_ptr()) % 256
    return ws[pad: pad + ws.numel() - 256]


def citron_validate(n: int, off, cols, ws, stream=None) -> int:
    """0 when the CSR satisfies the input contract, else the smallest defect code (1..5)."""
    bad = ctypes.c_uint32(0)
    code = lib().citron_validate(n, int(cols.numel()), _dptr(off), _dptr(cols),
                                 ctypes.byref(bad), _dptr(ws), _nbytes(ws), _stream(stream))
    if code not in (0, 1):
        _check(code, "citron_validate")
    return int(bad.value)


def citron_order(n: int, off, rank, perm=None, ws=None, stream=None):
    _check(lib().citron_order(n, _dptr(off), _dptr(rank), _dptr(perm), _dptr(ws), _nbytes(ws),
                              _stream(stream)), "citron_order")


def citron_order_grouped(n: int, off, group, ngroups: int, rank, perm=None, ws=None, stream=None):
    """Degree ordering of a disjoint union of graphs, graph by graph: (group, degree, id)."""
    _check(lib().citron_order_grouped(n, _dptr(off), _dptr(group), ngroups, _dptr(rank), _dptr(perm),
                                      _dptr(ws), _nbytes(ws), _stream(stream)), "citron_order_grouped")


def citron_core_order(n: int, off, cols, rank, perm=None, ws=None, stream=None) -> tuple[int, int]:
    """Core ordering by synchronous peeling rounds; returns (degeneracy, rounds)."""
    level, rounds = ctypes.c_uint32(0), ctypes.c_uint32(0)
    _check(lib().citron_core_order(n, int(cols.numel()), _dptr(off), _dptr(cols), _dptr(rank),
                                   _dptr(perm), ctypes.byref(level), ctypes.byref(rounds),
                                   _dptr(ws), _nbytes(ws), _stream(stream)), "citron_core_order")
    return int(level.value), int(rounds.value)


def citron_build_dag(n: int, off, cols, rank, dag_off, dag_cols, ws, stream=None,
                     want_max_outdeg: bool = True):
    mx = ctypes.c_uint32(0)
    _check(lib().citron_build_dag(n, int(cols.numel()), _dptr(off), _dptr(cols), _dptr(rank),
                                  _dptr(dag_off), _dptr(dag_cols),
                                  ctypes.byref(mx) if want_max_outdeg else ctypes.c_void_p(0),
                                  _dptr(ws), _nbytes(ws), _stream(stream)), "citron_build_dag")
    return int(mx.value) if want_max_outdeg else None


def citron_count(n: int, dag_off, dag_cols, k: int, ws, max_outdeg: int = 0, per_root=None,
                 stream=None) -> int:
    out = ctypes.c_uint64(0)
    _check(lib().citron_count(n, _dptr(dag_off), _dptr(dag_cols), k, max_outdeg, ctypes.byref(out),
                              _dptr(per_root), _dptr(ws), _nbytes(ws), _stream(stream)),
           f"citron_count(k={k})")
    return int(out.value)


def citron_count_ex(n: int, dag_off, dag_cols, k: int, ws, max_outdeg: int = 0, per_root=None,
                    stream=None, small_max: int = 0, bitmap_max: int = 0, warps_per_cta: int = 0,
                    time_kernels: bool = False, count_work: bool = False, compact_max: int = 0,
                    max_blocks: int = 0, split_min: int = 0, balance: bool = False,
                    budget_ms: int = 0, per_arc=None):
    """Returns (count, CountOpts) -- the options carry work_ops, kernel_ms and busy_ms on return.
    per_arc: optional device uint64 array of one entry per DAG arc (3 <= k <= 8), filled with
    each edge task's count (debug mode); count_work also needs k <= 8."""
    o = CountOpts(small_max, bitmap_max, warps_per_cta,
                  (COUNT_TIME_KERNELS if time_kernels else 0) | (COUNT_WORK if count_work else 0)
                  | (COUNT_BALANCE if balance else 0),
                  compact_max, max_blocks, _dptr(per_root).value, 0)
    o.split_min = split_min
    o.budget_ms = budget_ms
    o.d_per_arc = _dptr(per_arc).value
    out = ctypes.c_uint64(0)
    _check(lib().citron_count_ex(n, _dptr(dag_off), _dptr(dag_cols), k, max_outdeg, ctypes.byref(o),
                                 ctypes.byref(out), _dptr(ws), _nbytes(ws), _stream(stream)),
           f"citron_count_ex(k={k})")
    return int(out.value), o


def citron_count_noalloc(n: int, dag_off, dag_cols, k: int, stream=None) -> int:
    """citron_count without a workspace (fixed device scratch; n <= 65536)."""
    out = ctypes.c_uint64(0)
    _check(lib().citron_count_noalloc(n, _dptr(dag_off), _dptr(dag_cols), k, ctypes.byref(out),
                                      _stream(stream)), f"citron_count_noalloc(k={k})")
    return int(out.value)


def citron_count_batch(n: int, dag_off, dag_cols, rank, group_of_vertex, group_k, ngroups: int,
                       kmask: int, max_outdeg: int, counts, ws, stream=None, opts: "CountOpts" = None):
    """Asynchronous batched count (see include/citron.h); counts[g] receives graph g's count."""
    _check(lib().citron_count_batch(n, _dptr(dag_off), _dptr(dag_cols), _dptr(rank),
                                    _dptr(group_of_vertex), _dptr(group_k), ngroups, kmask,
                                    max_outdeg, ctypes.byref(opts) if opts is not None else None,
                                    _dptr(counts), _dptr(ws), _nbytes(ws), _stream(stream)),
           "citron_count_batch")


def citron_set_faults(lookback_spin_limit: int = 0, lookback_stall_tile: int | None = None,
                      barrier_wait_ns: int = 0, barrier_absent_block: int | None = None,
                      count_seed: int = 0):
    """Inject faults for error-path tests (tile / block indices are 0-based here; None: none).
    Call with no arguments to restore normal operation."""
    f = Faults(lookback_spin_limit, 0 if lookback_stall_tile is None else lookback_stall_tile + 1,
               barrier_wait_ns, 0 if barrier_absent_block is None else barrier_absent_block + 1, 0,
               count_seed)
    clear = not any((lookback_spin_limit, lookback_stall_tile is not None, barrier_wait_ns,
                     barrier_absent_block is not None, count_seed))
    _check(lib().citron_set_faults(None if clear else ctypes.byref(f)), "citron_set_faults")


def citron_probe_word_ops(blocks_per_sm: int = 2, iters: int = 200000, stream=None) -> tuple[float, float]:
    """Measured peak of 32-bit word operations (AND + POPC + add) per second, and its kernel ms."""
    ops, ms = ctypes.c_double(0), ctypes.c_float(0)
    _check(lib().citron_probe_word_ops(blocks_per_sm, iters, ctypes.byref(ops), ctypes.byref(ms),
                                       _stream(stream)), "citron_probe_word_ops")
    return float(ops.value), float(ms.value)


def citron_dag_append(n: int, src_off, src_cols, src_row: int, dst_off, dst_cols, dst_row: int,
                      dst_arc: int, stream=None):
    """Copy the DAG rows src_row.. (src_off: their n+1 offsets) to rows dst_row.., arcs from
    dst_arc, offsets re-based and column ids shifted (asynchronous)."""
    _check(lib().citron_dag_append(n, _dptr(src_off), _dptr(src_cols), src_row, _dptr(dst_off),
                                   _dptr(dst_cols), dst_row, dst_arc, _stream(stream)),
           "citron_dag_append")


def citron_workspace_status(ws, stream=None):
    _check(lib().citron_workspace_status(_dptr(ws), _stream(stream)), "citron_workspace_status")


def citron_list(n: int, dag_off, dag_cols, k: int, ws, out=None, capacity: int | None = None,
                id_map=None, stream=None) -> int:
    """Write the k-cliques as rows of `out` (a CUDA int32 tensor of shape (capacity, k)); returns
    the number of k-cliques (only min(total, capacity) rows are written)."""
    total = ctypes.c_uint64(0)
    if capacity is None:
        capacity = 0 if out is None else int(out.shape[0])
    _check(lib().citron_list(n, _dptr(dag_off), _dptr(dag_cols), k, _dptr(id_map), _dptr(out),
                             capacity, ctypes.byref(total), _dptr(ws), _nbytes(ws), _stream(stream)),
           "citron_list")
    return int(total.value)


def citron_kernel_launches() -> int:
    return int(lib().citron_kernel_launches())


def citron_host_buffer_bytes(n: int, arcs: int) -> int:
    return int(lib().citron_host_buffer_bytes(n, arcs))


def citron_count_host(n: int, off: np.ndarray, cols: np.ndarray, ks, d_buf, ws, stream=None) -> list[int]:
    """Whole path from host CSR arrays (pinned numpy views or torch CPU tensors)."""
    ks_arr = np.ascontiguousarray(np.asarray(ks, dtype=np.uint32))
    out = np.zeros(len(ks_arr), dtype=np.uint64)
    _check(lib().citron_count_host(n, int(cols.shape[0]), ctypes.c_void_p(_host_ptr(off)),
                                   ctypes.c_void_p(_host_ptr(cols)), ctypes.c_void_p(ks_arr.ctypes.data),
                                   len(ks_arr), ctypes.c_void_p(out.ctypes.data), _dptr(d_buf),
                                   _nbytes(d_buf), _dptr(ws), _nbytes(ws), _stream(stream)),
           "citron_count_host")
    return [int(x) for x in out]


def _host_ptr(a) -> int:
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    return a.data_ptr()


# ---------------------------------------------------------------------------------------------
# Convenience: one graph resident on the device


class DeviceGraph:
    """A CSR graph uploaded once, with its degree ordering and DAG built on the device.

    ``relabel=True`` (default) builds the DAG in rank space from citron_order's ranks;
    ``relabel=False`` builds the paper's GenOrdering DAG in the input's vertex ids;
    ``ordering="core"`` ranks by citron_core_order instead (relabelled DAG).
    """

    def __init__(self, g, relabel: bool = True, device="cuda", stream=None, rank=None,
                 ordering: str = "degree"):
        import torch

        self.n = g.n
        self.arcs = int(g.cols.shape[0])
        dev = torch.device(device)
        self.off = torch.from_numpy(np.ascontiguousarray(g.off).view(np.int64)).to(dev)
        self.cols = torch.from_numpy(np.ascontiguousarray(g.cols).view(np.int32)).to(dev)
        self.ws = alloc_workspace(self.n, self.arcs, 1, device=dev)
        self.rank = None
        self.degeneracy = self.rounds = None
        if ordering not in ("degree", "core"):
            raise ValueError("ordering is 'degree' or 'core'")
        if rank is not None:
            self.rank = torch.as_tensor(np.asarray(rank, dtype=np.uint32).view(np.int32), device=dev)
        elif ordering == "core":
            self.rank = torch.empty(max(1, self.n), dtype=torch.int32, device=dev)
            self.degeneracy, self.rounds = citron_core_order(self.n, self.off, self.cols, self.rank,
                                                             None, self.ws, stream)
        elif relabel:
            self.rank = torch.empty(max(1, self.n), dtype=torch.int32, device=dev)
            citron_order(self.n, self.off, self.rank, None, self.ws, stream)
        self.dag_off = torch.empty(self.n + 1, dtype=torch.int64, device=dev)
        self.dag_cols = torch.empty(max(1, self.arcs // 2), dtype=torch.int32, device=dev)
        self.max_outdeg = citron_build_dag(self.n, self.off, self.cols, self.rank, self.dag_off,
                                           self.dag_cols, self.ws, stream)
        need = citron_workspace_bytes(self.n, self.arcs, self.max_outdeg)
        if need > _nbytes(self.ws):
            self.ws = alloc_workspace(self.n, self.arcs, self.max_outdeg, device=dev)

    def count(self, k: int, per_root=None, stream=None, **tuned) -> int:
        if tuned:
            return citron_count_ex(self.n, self.dag_off, self.dag_cols, k, self.ws, self.max_outdeg,
                                   per_root, stream, **tuned)[0]
        return citron_count(self.n, self.dag_off, self.dag_cols, k, self.ws, self.max_outdeg,
                            per_root, stream)

    def count_per_arc(self, k: int, stream=None, **tuned) -> tuple[int, np.ndarray]:
        """(K_k, per-arc counts): for every DAG arc e = (u, v), the k-cliques whose first two
        vertices in the DAG order are u, v (k >= 3; a debug mode of citron_count_ex)."""
        import torch

        arcs = int(self.dag_off[-1].item())
        pa = torch.empty(max(1, arcs), dtype=torch.int64, device=self.dag_off.device)
        c, _ = citron_count_ex(self.n, self.dag_off, self.dag_cols, k, self.ws, self.max_outdeg,
                               stream=stream, per_arc=pa, **tuned)
        return c, pa[:arcs].cpu().numpy().view(np.uint64)

    def list(self, k: int, input_ids: bool = True, stream=None) -> np.ndarray:
        """Every k-clique as a row of k vertex ids (input ids by default), shape (K_k, k)."""
        import torch

        total = citron_list(self.n, self.dag_off, self.dag_cols, k, self.ws, None, 0, None, stream)
        out = torch.empty((max(1, total), k), dtype=torch.int32, device=self.dag_off.device)
        id_map = None
        if input_ids and self.rank is not None:
            id_map = torch.empty_like(self.rank)
            id_map[self.rank[: self.n].long()] = torch.arange(self.n, dtype=torch.int32,
                                                              device=self.rank.device)
        got = citron_list(self.n, self.dag_off, self.dag_cols, k, self.ws, out, total, id_map, stream)
        if got != total:
            raise RuntimeError("clique count changed between the sizing and the listing call")
        return out[:total].cpu().numpy().view(np.uint32)

    def dag_numpy(self):
        off = self.dag_off.cpu().numpy().view(np.uint64)
        cols = self.dag_cols.cpu().numpy().view(np.uint32)[: int(off[-1])]
        return off, cols
