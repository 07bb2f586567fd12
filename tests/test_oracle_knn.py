"""Pins of the oracle's stencil selection (Sec. 4.1, Eq. 11: the n nodes closest to x_c).

The oracle's brute force is pinned against an independent numpy ordering
(lexsort on squared distance, then node id), and the oracle's cell list is
pinned against its brute force, on regular grids (many exact distance ties),
jittered grids, periodic boxes and cross-set (staggered) queries.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W


def numpy_knn(centres, sources, period, n):
    out = np.empty((len(centres), n), dtype=np.int64)
    ids = np.arange(len(sources))
    for c, x in enumerate(centres):
        d = sources - x
        for a in range(d.shape[1]):
            if period[a] > 0:
                p = period[a]
                d[:, a] = np.where(d[:, a] > 0.5 * p, d[:, a] - p,
                                   np.where(d[:, a] < -0.5 * p, d[:, a] + p, d[:, a]))
        d2 = np.zeros(len(sources))
        for a in range(d.shape[1]):
            d2 = d2 + d[:, a] * d[:, a]
        out[c] = np.lexsort((ids, d2))[:n]
    return out


@pytest.mark.parametrize("kind", ["grid2", "jit2", "per2", "jit3", "per3", "grid3"])
def test_brute_matches_numpy(kind):
    if kind == "grid2":
        ns = W.pec_box((9, 7), 0.0, 1)
    elif kind == "jit2":
        ns = W.pec_box((9, 8), 0.25, 2)
    elif kind == "per2":
        ns = W.periodic_box((8, 8), 0.25, 3)
    elif kind == "jit3":
        ns = W.pec_box((5, 5, 4), 0.25, 4)
    elif kind == "per3":
        ns = W.periodic_box((5, 5, 5), 0.25, 5)
    else:
        ns = W.pec_box((4, 5, 4), 0.0, 6)
    n = 13 if ns.dim == 2 else 20
    a = O.knn_brute(ns.xyz, ns.xyz, ns.period, n)
    b = numpy_knn(ns.xyz, ns.xyz, ns.period, n)
    assert np.array_equal(a, b)
    # the centre itself comes first (distance 0, no other node at distance 0)
    assert np.array_equal(a[:, 0], np.arange(ns.n))


def test_cross_set_brute_matches_numpy():
    e = W.periodic_box((10, 10), 0.25, 7)
    h = W.periodic_box((10, 10), 0.25, 8, offset=(0.5, 0.5))
    a = O.knn_brute(h.xyz, e.xyz, e.period, 12)
    b = numpy_knn(h.xyz, e.xyz, e.period, 12)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("shape,jit,periodic,n", [
    ((64, 64), 0.0, False, 31),
    ((64, 64), 0.25, False, 31),
    ((64, 64), 0.25, True, 57),
    ((64, 64), 0.0, True, 12),
    ((16, 16, 16), 0.25, False, 71),
    ((16, 16, 16), 0.25, True, 40),
])
def test_cells_match_brute(shape, jit, periodic, n):
    ns = (W.periodic_box(shape, jit, 11) if periodic else W.pec_box(shape, jit, 11))
    a = O.knn_cells(ns.xyz, ns.xyz, ns.period, n)
    b = O.knn_brute(ns.xyz, ns.xyz, ns.period, n)
    assert np.array_equal(a, b)


def test_cells_cross_set_match_brute():
    e = W.periodic_box((48, 48), 0.25, 12)
    h = W.periodic_box((48, 48), 0.25, 13, offset=(0.5, 0.5))
    a = O.knn_cells(h.xyz, e.xyz, e.period, 30)
    b = O.knn_brute(h.xyz, e.xyz, e.period, 30)
    assert np.array_equal(a, b)


def test_regular_grid_plus_stencil():
    """On a unit grid the 5 nearest nodes are the centre and its 4 axis neighbours."""
    ns = W.periodic_box((6, 6), 0.0, 1)
    idx = O.knn_brute(ns.xyz, ns.xyz, ns.period, 5)
    i = 2 * 6 + 3  # node (3, 2)
    got = {tuple(ns.xyz[j]) for j in idx[i]}
    assert got == {(3, 2), (2, 2), (4, 2), (3, 1), (3, 3)}
    # ties (four neighbours at distance 1) are broken by node id
    assert list(idx[i][1:]) == sorted(idx[i][1:])
