"""PEC walls by images on the GPU (mfd_nodes_set_mirror) against the oracle,
which computes the same on the doubled periodic box (oracle.mirror_doubled).

* kNN: the stencils of every node of a 2D and a 3D PEC box among the nodes and
  their mirror images equal the oracle's on the doubled box, entry for entry
  (node id and reflection code), ties included.
* weights: within 1e-8 of the oracle's (max-norm per stencil), GRAD and Delta^alpha.
* steps: the TM11 cavity with sources and probes (2D) and the TM110 cube with
  eps_r (3D), FP64 within 1e-10 and FP32 within 1e-5 relative L2 of the oracle.
* calls that do not support images refuse them (staggered layout, batch, gradient).
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_2508_18205_gb300")


def _mirror_nodes(ctx, box):
    nd = M.Nodes(ctx, box.xyz, box.period)
    nd.set_mirror((1 << box.dim) - 1, box.box_hi)
    return nd


def _oracle_rows(box, n):
    dbl, orig, code = O.mirror_doubled(box)
    ids = O.knn(box.xyz, dbl.xyz, dbl.period, n)
    return dbl, ids, orig[ids] + (code[ids] << 32)


@pytest.mark.parametrize("shape,n", [((20, 17), 31), ((12, 12), 12), ((8, 9, 7), 71), ((7, 7, 7), 40)])
def test_image_stencils_and_weights_match_the_oracle(shape, n):
    ctx = M.Ctx(0)
    box = W.pec_box_cells(shape, 0.25, 41)
    nd = _mirror_nodes(ctx, box)
    st = M.Stencils(nd, nd, n)
    dbl, ids, want = _oracle_rows(box, n)
    got = st.read()
    assert np.array_equal(got, want)
    assert np.any(want >> 32)  # images were taken
    d = box.dim
    for op, k, m, alpha, nu in ((M.MFD_OP_GRAD, 3, 2, 0, min(n, 12 if d == 2 else 40)),
                                (M.MFD_OP_LAP_POW, 5, 4, 2, 31 if d == 2 else 71)):
        if nu > n:
            continue
        gw = M.Weights(st, nu, k, m, op, alpha).read()
        rw = O.weights(box.xyz, dbl.xyz, dbl.period, ids, nu, k, m, op, alpha)
        scale = np.max(np.abs(rw), axis=2, keepdims=True)
        assert np.max(np.abs(gw - rw) / scale) <= 1e-8


@pytest.mark.parametrize("prec,tol", [(M.MFD_FP64, 1e-10), (M.MFD_FP32, 1e-5)])
def test_tm11_cavity_with_images_matches_the_oracle(prec, tol):
    ctx = M.Ctx(0)
    S, c = 0.5, 4e-3
    dt, eps0, mu0, c0, eta0 = W.units(S)
    box = W.pec_box_cells((30, 30), 0.25, 42)
    nd = _mirror_nodes(ctx, box)
    st = M.Stencils(nd, nd, 31)
    cw = M.Weights(st, 12, 3, 2, M.MFD_OP_GRAD)
    hw = M.Weights(st, 31, 5, 4, M.MFD_OP_LAP_POW, 2)
    sim = M.Sim(ctx, 2, prec, dt, eps0, mu0, -c, cw, hw, compensated=prec == M.MFD_FP32)
    eps = W.eps_r_uniform(box.n, 43)
    sim.set_materials(eps, None)
    ez, hx, hy = W.tm11_fields(box.xyz, 30.0, c0, mu0, 0.0, -0.5 * dt)
    src = W.ricker_sources(box, 3, 44, c0)
    probes = W.interior_nodes(box, 6, 45)
    for comp, f in ((M.MFD_EZ, ez), (M.MFD_HX, hx), (M.MFD_HY, hy)):
        sim.set_field(comp, f)
    sim.set_sources(src.node, src.amp, src.f0, src.t0)
    sim.set_probes(probes, 300)
    nsteps = 300
    sim.step(nsteps)
    got = np.concatenate([sim.get_field(cc) for cc in (M.MFD_EZ, M.MFD_HX, M.MFD_HY)])
    order = np.argsort(src.node)
    srt = W.Sources(node=src.node[order], rhs=src.rhs[order], amp=src.amp[order], f0=src.f0[order], t0=src.t0[order])
    e1, x1, y1, pr, _ = O.run_tmz_images(box, 12, 3, 2, 2, dt, eps0, mu0, -c, ez, hx, hy, nsteps, eps_r=eps,
                                         sources=srt, probes=probes)
    ref = np.concatenate([e1, x1, y1])
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)
    gp = sim.read_probes()
    assert np.linalg.norm(gp - pr) <= tol * np.linalg.norm(pr)
    # the energy of Eq. 20 (the box's part) is computed with the image signs too
    u = sim.energy()
    assert np.isfinite(u) and u > 0


@pytest.mark.parametrize("prec,tol", [(M.MFD_FP64, 1e-10), (M.MFD_FP32, 1e-5)])
def test_tm110_cube_with_images_matches_the_oracle(prec, tol):
    ctx = M.Ctx(0)
    S, c = 0.5, 1e-3
    dt, eps0, mu0, c0, eta0 = W.units(S)
    cube = W.pec_box_cells((9, 10, 8), 0.25, 46)
    nd = _mirror_nodes(ctx, cube)
    st = M.Stencils(nd, nd, 71)
    cw = M.Weights(st, 40, 3, 3, M.MFD_OP_GRAD)
    hw = M.Weights(st, 71, 5, 4, M.MFD_OP_LAP_POW, 2)
    sim = M.Sim(ctx, 3, prec, dt, eps0, mu0, -c, cw, hw, compensated=prec == M.MFD_FP32)
    eps = W.eps_r_smooth_3d(cube.xyz, cube.box_hi, 47, grid=32)
    sim.set_materials(eps, None)
    rng = np.random.default_rng(48)
    E0 = 0.3 * rng.standard_normal((3, cube.n))
    H0 = 0.3 * rng.standard_normal((3, cube.n))
    for comp in range(3):
        sim.set_field(comp, E0[comp])
        sim.set_field(3 + comp, H0[comp])
    nsteps = 60
    sim.step(nsteps)
    got = np.concatenate([sim.get_field(cc) for cc in range(6)])
    E1, H1, _ = O.run_3d_images(cube, 40, 3, 3, 2, dt, eps0, mu0, -c, E0, H0, nsteps, eps_r=eps)
    ref = np.concatenate([E1.ravel(), H1.ravel()])
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)


def test_images_are_refused_where_unsupported():
    ctx = M.Ctx(0)
    dt, eps0, mu0, c0, eta0 = W.units(0.5)
    box = W.pec_box_cells((12, 12), 0.25, 49)
    nd = _mirror_nodes(ctx, box)
    st = M.Stencils(nd, nd, 31)
    cw = M.Weights(st, 12, 3, 2, M.MFD_OP_GRAD)
    hw = M.Weights(st, 31, 5, 4, M.MFD_OP_LAP_POW, 2)
    with pytest.raises(M.MfdError):
        M.Batch(ctx, [(cw, hw, dt, eps0, mu0, -4e-3)], nrhs=4)
    sim = M.Sim(ctx, 2, M.MFD_FP64, dt, eps0, mu0, -4e-3, cw, hw)
    sim.set_probes([50], 10)
    with pytest.raises(M.MfdError):
        sim.grad(5)
    plain = M.Nodes(ctx, box.xyz, box.period)
    with pytest.raises(M.MfdError):  # a cross-set stencil from a mirrored set
        M.Stencils(plain, nd, 12)
    with pytest.raises(M.MfdError):  # nodes outside the walls
        M.Nodes(ctx, box.xyz + 0.6, box.period).set_mirror(3, box.box_hi)
