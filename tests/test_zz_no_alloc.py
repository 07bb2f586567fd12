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


def _static_knn(ns, n, centres=None, period=True, check_free=False):
    """The static-scratch kNN of the centres (default: the source set itself)
    among the nodes of ns; with check_free, the free device memory reported by
    the driver is the same before and after the call."""
    dev = torch.device("cuda", 0)
    xs = torch.from_numpy(np.ascontiguousarray(ns.xyz)).to(dev)
    xc = xs if centres is None else torch.from_numpy(np.ascontiguousarray(centres)).to(dev)
    nc = xc.shape[0]
    out = torch.full((nc, n), -1, dtype=torch.int32, device=dev)
    per = np.ascontiguousarray(ns.period, dtype=np.float64)
    stream = torch.cuda.current_stream(dev).cuda_stream
    torch.cuda.synchronize(dev)
    free0 = torch.cuda.mem_get_info(dev)[0]
    st = M.lib().mfd_knn_static(ns.dim, nc, C.c_void_p(xc.data_ptr()), ns.n, C.c_void_p(xs.data_ptr()),
                                per.ctypes.data_as(C.c_void_p) if period else None, n,
                                C.c_void_p(out.data_ptr()), C.c_void_p(stream))
    M._ck(st)
    torch.cuda.synchronize(dev)
    if check_free:
        assert torch.cuda.mem_get_info(dev)[0] == free0
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


def test_static_knn_allocates_nothing_and_covers_separate_centres_and_no_period():
    """After a first call has loaded the kernels, a call leaves the free device
    memory unchanged; centres other than the sources (a staggered set), and a
    non-periodic set passed with period = NULL, give the allocating entry
    point's stencils."""
    ctx = M.Ctx(0)
    e = W.periodic_box((40, 40), 0.25, 63)
    h = W.periodic_box((40, 40), 0.25, 64, offset=(0.5, 0.5))
    _static_knn(e, 30)  # loads the kernels
    got = _static_knn(e, 30, centres=h.xyz, check_free=True)
    ne, nh = M.Nodes(ctx, e.xyz, e.period), M.Nodes(ctx, h.xyz, h.period)
    assert np.array_equal(got, M.Stencils(nh, ne, 30).read())
    box = W.pec_box((30, 26), 0.25, 65)
    got = _static_knn(box, 12, period=False, check_free=True)
    assert np.array_equal(got, _allocating_knn(ctx, box, 12))


def test_static_knn_rejects_periodic_coordinates_outside_the_period():
    ns = W.periodic_box((20, 20), 0.25, 66)
    bad = W.NodeSet(xyz=ns.xyz + np.array([20.0, 0.0]), pec=ns.pec, period=ns.period, box_lo=ns.box_lo,
                    box_hi=ns.box_hi)
    with pytest.raises(M.MfdError, match="period"):
        _static_knn(bad, 12)


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
