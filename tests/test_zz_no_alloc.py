"""citron_count_noalloc -- the counting entry point for callers that cannot allocate device
memory (for example code inside a CUDA-graph capture, or a host framework that forbids device
allocation after start-up).  It must give the same exact counts as citron_count, which uses a
caller-allocated workspace, on two calls in a row (its fixed scratch keeps the previous call's
contents and must be cleared by each call).  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_2112_10913_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


def _call(L, G, k, stream):
    out = ctypes.c_uint64(0)
    st = L.citron_count_noalloc(G.n, ctypes.c_void_p(G.dag_off.data_ptr()),
                                ctypes.c_void_p(G.dag_cols.data_ptr()), k, ctypes.byref(out), stream)
    return st, int(out.value)


@pytest.mark.parametrize("make", [gg.config1_er_planted, lambda: gg.small_rmat(21, 6000, 24.0),
                                  lambda: gg.complete(40)])
def test_noalloc_equals_workspace_entry_point(gpu, make):
    import torch

    L = gpu.lib()
    stream = ctypes.c_void_p(int(torch.cuda.current_stream().cuda_stream))
    for relabel in (True, False):
        G = gpu.DeviceGraph(make(), relabel=relabel)
        for k in range(1, 8):
            want = G.count(k)
            for _ in range(2):  # two calls in a row through the C ABI
                st, got = _call(L, G, k, stream)
                assert st == 0, gpu.STATUS.get(st)
                assert got == want, (k, got, want)


def test_noalloc_rejects_sizes_beyond_its_maximum(gpu):
    import torch

    L = gpu.lib()
    g = gg.csr_from_edges(70000, [1, 2], [3, 4])
    G = gpu.DeviceGraph(g)
    stream = ctypes.c_void_p(int(torch.cuda.current_stream().cuda_stream))
    st, _ = _call(L, G, 3, stream)
    assert gpu.STATUS[st] == "CITRON_E_UNSUPPORTED"
