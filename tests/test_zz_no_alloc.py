"""mfd_knn_static: kNN stencils for callers that cannot allocate device memory.

Some callers must not call cudaMalloc (their host application owns all device
memory through its own pool, or forbids allocation once running). For them the
library offers one entry point that takes caller-owned device arrays and keeps
its scratch in a static device array. This test calls it through the C ABI on
two calls in a row (different node sets, so the second call reuses scratch the
first one left behind) and checks that its stencils equal, entry for entry,
those of the allocating entry point (mfd_stencils_build + mfd_stencils_read).
The file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
M = pytest.importorskip("paper_2508_18205_gb300")


def _static_knn(ns, n):
    dev = torch.device("cuda", 0)
    xyz = torch.from_numpy(np.ascontiguousarray(ns.xyz)).to(dev)
    out = torch.full((ns.n, n), -1, dtype=torch.int32, device=dev)
    per = np.ascontiguousarray(ns.period, dtype=np.float64)
    stream = torch.cuda.current_stream(dev).cuda_stream
    st = M.lib().mfd_knn_static(ns.dim, ns.n, C.c_void_p(xyz.data_ptr()), ns.n, C.c_void_p(xyz.data_ptr()),
                                per.ctypes.data_as(C.c_void_p), n, C.c_void_p(out.data_ptr()),
                                C.c_void_p(stream))
    M._ck(st)
    torch.cuda.synchronize(dev)
    return out.cpu().numpy().astype(np.int64)


def _allocating_knn(ctx, ns, n):
    nd = M.Nodes(ctx, ns.xyz, ns.period)
    return M.Stencils(nd, nd, n).read()


def test_static_knn_matches_allocating_entry_point_twice():
    ctx = M.Ctx(0)
    first = W.periodic_box((70, 50), 0.25, 61)      # periodic, 3500 nodes
    second = W.pec_box((23, 19, 11), 0.25, 62)      # 3D PEC box, 4807 nodes
    a = _static_knn(first, 31)
    b = _static_knn(second, 40)
    assert np.array_equal(a, _allocating_knn(ctx, first, 31))
    assert np.array_equal(b, _allocating_knn(ctx, second, 40))


def test_static_knn_rejects_oversized_source_sets():
    ns = 3_000_000
    with pytest.raises(M.MfdError, match="static scratch"):
        dev = torch.device("cuda", 0)
        xyz = torch.zeros((ns, 2), dtype=torch.float64, device=dev)
        xyz[:, 0] = torch.arange(ns, device=dev, dtype=torch.float64)
        out = torch.empty((1, 4), dtype=torch.int32, device=dev)
        per = np.zeros(2)
        M._ck(M.lib().mfd_knn_static(2, 1, C.c_void_p(xyz.data_ptr()), ns, C.c_void_p(xyz.data_ptr()),
                                     per.ctypes.data_as(C.c_void_p), 4, C.c_void_p(out.data_ptr()), None))
