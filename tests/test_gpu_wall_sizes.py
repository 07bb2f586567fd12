"""Per-centre stencil sizes (mfd_weights_compute_sized) against the oracle.

* weights: every row within 1e-8 of the oracle's weights at that centre's own
  size (max-norm per row), zero past it.
* steps: a periodic 3D box with mixed curl sizes (40, 41, 43, 44: whole and
  partial chunks, slices with different chunk counts) and the PEC cube with
  images and a 44-node curl layer next to the walls, FP64 within 1e-10 and
  FP32 within 1e-5 relative L2 of the oracle.
* the corner of the 100^3 PEC cube where 40-node image stencils grow: on the
  GPU too the 40-node scheme grows and the 44-node wall layer does not.
* layouts that take one size per operator refuse sized weights.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_2508_18205_gb300")

N_CURL, N_WALL, ALPHA = 40, 44, 2


def _pec(ctx, box):
    nd = M.Nodes(ctx, box.xyz, box.period)
    nd.set_mirror(7, box.box_hi)
    return nd


def test_sized_weights_match_the_oracle():
    ctx = M.Ctx(0)
    box = W.periodic_box((9, 8, 10), 0.25, 61)
    sizes = np.random.default_rng(62).choice([40, 41, 43, 44], box.n).astype(np.int32)
    nd = M.Nodes(ctx, box.xyz, box.period)
    st = M.Stencils(nd, nd, 71)
    gw = M.Weights(st, sizes, 3, 3, M.MFD_OP_GRAD).read()
    ids = O.knn(box.xyz, box.xyz, box.period, 71)
    rw = O.weights_sized(box.xyz, box.xyz, box.period, ids, sizes, 3, 3, O.OP_GRAD)
    assert gw.shape == rw.shape == (3, box.n, 44)
    scale = np.max(np.abs(rw), axis=2, keepdims=True)
    assert np.max(np.abs(gw - rw) / scale) <= 1e-8
    for c in range(box.n):
        assert not np.any(gw[:, c, sizes[c]:])


@pytest.mark.parametrize("prec,tol", [(M.MFD_FP64, 1e-10), (M.MFD_FP32, 1e-5)])
def test_mixed_sizes_periodic_box_matches_the_oracle(prec, tol):
    ctx = M.Ctx(0)
    dt, eps0, mu0, c0, eta0 = W.units(0.5)
    box = W.periodic_box((10, 9, 11), 0.25, 63)
    sizes = np.random.default_rng(64).choice([40, 41, 43, 44], box.n).astype(np.int32)
    nd = M.Nodes(ctx, box.xyz, box.period)
    st = M.Stencils(nd, nd, 71)
    cw = M.Weights(st, sizes, 3, 3, M.MFD_OP_GRAD)
    hw = M.Weights(st, 71, 5, 4, M.MFD_OP_LAP_POW, ALPHA)
    sim = M.Sim(ctx, 3, prec, dt, eps0, mu0, -1e-3, cw, hw, compensated=prec == M.MFD_FP32)
    eps = W.eps_r_uniform(box.n, 65, 1.0, 3.0)
    sim.set_materials(eps, None)
    rng = np.random.default_rng(66)
    E0, H0 = 0.3 * rng.standard_normal((3, box.n)), 0.3 * rng.standard_normal((3, box.n))
    for comp in range(3):
        sim.set_field(comp, E0[comp])
        sim.set_field(3 + comp, H0[comp])
    sim.step(50)
    got = np.concatenate([sim.get_field(c) for c in range(6)])
    prob, _ = O.max3d_collocated(box, N_CURL, 3, 3, ALPHA, dt, eps0, mu0, -1e-3, eps_r=eps, n_per=sizes)
    E1, H1, _, _ = O.run_3d(prob, E0, H0, 50)
    ref = np.concatenate([E1.ravel(), H1.ravel()])
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)
    u = sim.energy()
    assert np.isfinite(u) and u > 0


@pytest.mark.parametrize("prec,tol", [(M.MFD_FP64, 1e-10), (M.MFD_FP32, 1e-5)])
def test_pec_cube_with_a_wall_layer_matches_the_oracle(prec, tol):
    ctx = M.Ctx(0)
    dt, eps0, mu0, c0, eta0 = W.units(0.5)
    cube = W.pec_box_cells((9, 10, 8), 0.25, 67)
    nd = _pec(ctx, cube)
    st = M.Stencils(nd, nd, 71)
    sizes = M.wall_layer_sizes(cube.xyz, cube.box_lo, cube.box_hi, N_CURL, N_WALL)
    assert np.array_equal(sizes, O.wall_sizes(cube, N_CURL, N_WALL))
    cw = M.Weights(st, sizes, 3, 3, M.MFD_OP_GRAD)
    hw = M.Weights(st, 71, 5, 4, M.MFD_OP_LAP_POW, ALPHA)
    sim = M.Sim(ctx, 3, prec, dt, eps0, mu0, -1e-3, cw, hw, compensated=prec == M.MFD_FP32)
    eps = W.eps_r_smooth_3d(cube.xyz, cube.box_hi, 68, grid=32)
    sim.set_materials(eps, None)
    rng = np.random.default_rng(69)
    E0, H0 = 0.3 * rng.standard_normal((3, cube.n)), 0.3 * rng.standard_normal((3, cube.n))
    for comp in range(3):
        sim.set_field(comp, E0[comp])
        sim.set_field(3 + comp, H0[comp])
    sim.step(60)
    got = np.concatenate([sim.get_field(c) for c in range(6)])
    E1, H1, _ = O.run_3d_images(cube, N_CURL, 3, 3, ALPHA, dt, eps0, mu0, -1e-3, E0, H0, 60, eps_r=eps,
                                n_wall=N_WALL)
    ref = np.concatenate([E1.ravel(), H1.ravel()])
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)


def test_the_wall_layer_removes_the_growing_corner_mode_on_the_gpu():
    ctx = M.Ctx(0)
    dt, eps0, mu0, c0, eta0 = W.units(0.5)
    full = W.pec_box_cells((100, 100, 100), 0.25, 3)
    lo, size = np.array([26, 60, 0]), np.array([12, 12, 8])
    cell = np.floor(full.xyz).astype(np.int64)
    sel = np.all((cell >= lo) & (cell < lo + size), axis=1)
    xyz = full.xyz[sel] - lo
    nd = M.Nodes(ctx, xyz, np.zeros(3))
    nd.set_mirror(7, size.astype(float))
    st = M.Stencils(nd, nd, 71)
    hw = M.Weights(st, 71, 5, 4, M.MFD_OP_LAP_POW, ALPHA)
    rng = np.random.default_rng(1)
    E0, H0 = rng.standard_normal((3, len(xyz))), rng.standard_normal((3, len(xyz)))
    growth = []
    for sizes in (N_CURL, M.wall_layer_sizes(xyz, np.zeros(3), size, N_CURL, N_WALL)):
        cw = M.Weights(st, sizes, 3, 3, M.MFD_OP_GRAD)
        sim = M.Sim(ctx, 3, M.MFD_FP64, dt, eps0, mu0, -1e-3, cw, hw)
        for comp in range(3):
            sim.set_field(comp, E0[comp])
            sim.set_field(3 + comp, H0[comp])
        u0 = sim.energy()
        sim.step(300)
        growth.append(sim.energy() / u0)
    assert growth[0] > 1e3
    assert growth[1] <= 1.0


def test_sized_weights_are_refused_where_one_size_is_expected():
    ctx = M.Ctx(0)
    dt, eps0, mu0, c0, eta0 = W.units(0.5)
    sq = W.pec_box((16, 16), 0.25, 70)
    nd = M.Nodes(ctx, sq.xyz, sq.period)
    st = M.Stencils(nd, nd, 31)
    sizes = np.where(sq.pec == 1, 14, 12).astype(np.int32)
    cw = M.Weights(st, sizes, 3, 2, M.MFD_OP_GRAD)
    hw = M.Weights(st, 31, 5, 4, M.MFD_OP_LAP_POW, 2)
    with pytest.raises(M.MfdError):  # the 2D layouts take one curl size
        M.Sim(ctx, 2, M.MFD_FP32, dt, eps0, mu0, -4e-3, cw, hw)
    with pytest.raises(M.MfdError):  # the batch too
        M.Batch(ctx, [(cw, M.Weights(st, 31, 5, 4, M.MFD_OP_LAP_POW, 2), dt, eps0, mu0, -4e-3)], nrhs=4)
    box = W.periodic_box((8, 8, 8), 0.25, 71)
    nd3 = M.Nodes(ctx, box.xyz, box.period)
    st3 = M.Stencils(nd3, nd3, 71)
    cw3 = M.Weights(st3, 40, 3, 3, M.MFD_OP_GRAD)
    hv_sized = M.Weights(st3, np.full(box.n, 71, np.int32) - (np.arange(box.n) % 2), 5, 4, M.MFD_OP_LAP_POW, 2)
    with pytest.raises(M.MfdError):  # hyperviscosity weights take one size
        M.Sim(ctx, 3, M.MFD_FP32, dt, eps0, mu0, -1e-3, cw3, hv_sized)
    with pytest.raises(M.MfdError):  # a size beyond the stencils
        M.Weights(st3, np.full(box.n, 72, np.int32), 3, 3, M.MFD_OP_GRAD)
    with pytest.raises(ValueError):
        M.Weights(st3, np.full(box.n - 1, 40, np.int32), 3, 3, M.MFD_OP_GRAD)
