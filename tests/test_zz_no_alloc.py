"""citron_count_noalloc -- the counting entry point for callers that cannot allocate device
memory (for example a host framework that owns the device heap and forbids allocation after
start-up, or a plain C caller with no allocator).  It must give the same exact counts as
citron_count, which uses a caller-allocated workspace, on two calls in a row (its fixed scratch
keeps the previous call's contents and must be cleared by each call), leave the free device
memory unchanged, and reject what does not fit its fixed scratch.  This file is collected last on
purpose."""
import ctypes
import math

import numpy as np
import pytest

from paper_2112_10913_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


def _call(L, G, k, stream):
    out = ctypes.c_uint64(0)
    st = L.citron_count_noalloc(G.n, ctypes.c_void_p(G.dag_off.data_ptr()),
                                ctypes.c_void_p(G.dag_cols.data_ptr()), k, ctypes.byref(out), stream)
    return st, int(out.value)


def _stream():
    import torch

    return ctypes.c_void_p(int(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("make", [gg.config1_er_planted, lambda: gg.small_rmat(21, 6000, 24.0),
                                  lambda: gg.complete(40)])
def test_noalloc_equals_workspace_entry_point(gpu, make):
    L = gpu.lib()
    stream = _stream()
    for relabel in (True, False):
        G = gpu.DeviceGraph(make(), relabel=relabel)
        for k in range(1, 8):
            want = G.count(k)
            for _ in range(2):  # two calls in a row through the C ABI
                st, got = _call(L, G, k, stream)
                assert st == 0, gpu.STATUS.get(st)
                assert got == want, (k, got, want)


def test_noalloc_sorted_list_path_and_no_allocation(gpu):
    """K_1100: the first 75 roots have out-degree above 1024 and take the sorted-list path inside
    the fixed scratch; the triangle count is C(1100, 3).  Free device memory is the same before
    and after a call."""
    import torch

    L = gpu.lib()
    stream = _stream()
    G = gpu.DeviceGraph(gg.complete(1100))
    assert G.max_outdeg == 1099
    for k in (3,):
        want = G.count(k)
        assert want == math.comb(1100, k)
        _call(L, G, k, stream)  # warm-up: module load and the scratch address look-up
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(2):
            st, got = _call(L, G, k, stream)
            assert st == 0, gpu.STATUS.get(st)
            assert got == want, (k, got, want)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_sizes_beyond_its_maximum(gpu):
    L = gpu.lib()
    g = gg.csr_from_edges(70000, [1, 2], [3, 4])
    G = gpu.DeviceGraph(g)
    st, _ = _call(L, G, 3, _stream())
    assert gpu.STATUS[st] == "CITRON_E_UNSUPPORTED"


def test_noalloc_reports_scratch_too_small(gpu):
    """A root of out-degree 8000 at k = 12 needs 4 warps x 8000 x 9 words of sorted-list scratch
    (1.15 MB), more than the fixed array holds: CITRON_E_WORKSPACE, and the next call still works."""
    import torch

    L = gpu.lib()
    n = 8001
    off = np.zeros(n + 1, dtype=np.uint64)
    off[1:] = 8000  # vertex 0 -> 1..8000, no other arc: a valid DAG with sorted rows
    cols = np.arange(1, n, dtype=np.uint32)
    dag_off = torch.from_numpy(off.view(np.int64)).cuda()
    dag_cols = torch.from_numpy(cols.view(np.int32)).cuda()
    out = ctypes.c_uint64(0)
    st = L.citron_count_noalloc(n, ctypes.c_void_p(dag_off.data_ptr()), ctypes.c_void_p(dag_cols.data_ptr()),
                                12, ctypes.byref(out), _stream())
    assert gpu.STATUS[st] == "CITRON_E_WORKSPACE"
    st = L.citron_count_noalloc(n, ctypes.c_void_p(dag_off.data_ptr()), ctypes.c_void_p(dag_cols.data_ptr()),
                                3, ctypes.byref(out), _stream())
    assert st == 0 and out.value == 0
