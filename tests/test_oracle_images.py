"""Pins of the image treatment of PEC walls (a reading: the paper only uses
periodic boxes). A perfectly conducting wall acts as a mirror: the tangential
E and the normal H are odd under the reflection, the normal E and the
tangential H even. A stencil of a box node takes the n nearest among the nodes
and their mirror images (the doubled periodic box, oracle.mirror_doubled) and
gathers an image with the sign of the field's parity; only the box's nodes are
stepped (oracle.tmz_images / max3d_images, orc_run_tmz_img / orc_run_3d_img).

* The parity table equals the closed-form TM11 (2D) and TM110 (3D) cavity modes
  evaluated at the mirrored positions.
* The doubled box holds every node once (a wall node is its own image).
* On a regular grid with stencils of whole distance shells (mirror-symmetric
  stencils), the box stepped with images equals the doubled periodic box
  stepped by the plain periodic scheme with the parity-extended fields, on
  every box node: the signed gathers and the image positions of the weights
  are pinned to the periodic scheme.
* The TM11 cavity with image stencils converges to the exact mode as h -> 0,
  at about second order. The nodes sit at the cell centres, so none lies on a
  wall (a node on a mirror plane sees every neighbour and its image at one
  distance, and the stencil's n-th cut can split such pairs).
* The energy of the PEC square with images stays within 0.2 % over 3000 steps.
* 3D: the TM110 cube converges, and the PEC cube with image stencils keeps its
  energy bounded where one-sided wall stencils grow (Sec. 5.1 / App. A).
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


def test_parities_match_the_closed_form_modes():
    S = 0.4
    dt, eps0, mu0, c0, eta0 = W.units(S)
    box = W.pec_box((9, 7), 0.25, 1)
    dbl, orig, code = O.mirror_doubled(box)
    L = box.box_hi[0]
    f = W.tm11_fields(box.xyz, L, c0, mu0, 0.3, 0.7)
    # the mode on the doubled box: a square cavity of side L in x needs L equal in y
    box = W.pec_box((9, 9), 0.25, 1)
    dbl, orig, code = O.mirror_doubled(box)
    L = box.box_hi[0]
    f = W.tm11_fields(box.xyz, L, c0, mu0, 0.3, 0.7)
    g = W.tm11_fields(dbl.xyz, L, c0, mu0, 0.3, 0.7)
    for k, comp in enumerate(("ez", "hx", "hy")):
        assert np.allclose(g[k], f[k][orig] * O.image_sign_tmz(code, comp), atol=1e-13)
    cube = W.pec_box((6, 6, 6), 0.25, 2)
    dbl, orig, code = O.mirror_doubled(cube)
    L = cube.box_hi[0]
    # TM110 in 3D and its rotations (the mode constant along axis p)
    for p in range(3):
        perm = [a for a in range(3) if a != p] + [p]
        Ef, Hf = W.tm110_fields_3d(cube.xyz[:, perm], L, c0, mu0, 0.3, 0.7)
        Eg, Hg = W.tm110_fields_3d(dbl.xyz[:, perm], L, c0, mu0, 0.3, 0.7)
        inv = np.argsort(perm)
        Ef, Hf, Eg, Hg = ([v[i] for i in inv] for v in (Ef, Hf, Eg, Hg))
        for b in range(3):
            assert np.allclose(Eg[b], Ef[b][orig] * O.image_sign_3d(code, "e", b), atol=1e-13)
            assert np.allclose(Hg[b], Hf[b][orig] * O.image_sign_3d(code, "h", b), atol=1e-13)


def test_doubled_box_counts_every_node_once():
    for shape in ((7, 6), (5, 6, 4)):
        box = W.pec_box(shape, 0.25, 3)
        dbl, orig, code = O.mirror_doubled(box)
        assert dbl.n == int(np.prod([2 * (s - 1) for s in shape]))
        assert np.all(dbl.xyz >= 0) and np.all(dbl.xyz < dbl.period)
        # no two entries coincide
        key = np.round(dbl.xyz * 1e9).astype(np.int64)
        assert len(np.unique(key, axis=0)) == dbl.n
        assert np.all(code[:box.n] == 0) and np.array_equal(orig[:box.n], np.arange(box.n))


def test_regular_grid_whole_shells_equal_the_doubled_periodic_box_2d():
    S, c = 0.4, 2e-3
    dt, eps0, mu0, c0, eta0 = W.units(S)
    box = W.pec_box_cells((9, 8), 0.0, 1)
    n, nhv = 13, 25  # whole shells of the square lattice: 1 + 4 + 4 + 4 and + 8 + 4
    rng = np.random.default_rng(3)
    ez, hx, hy = rng.standard_normal((3, box.n))
    # a wall node is its own image: its odd components are 0 (tangential E, normal H)
    ez[box.pec == 1] = 0.0
    hx[(box.normal_axes & 1) == 1] = 0.0
    hy[(box.normal_axes & 2) == 2] = 0.0
    er = W.eps_r_uniform(box.n, 4)
    e1, x1, y1, _, _ = O.run_tmz_images(box, n, 3, 2, 2, dt, eps0, mu0, -c, ez, hx, hy, 12, eps_r=er,
                                        nh_override=nhv)
    dbl, orig, code = O.mirror_doubled(box)
    prob, _ = O.tmz_collocated(dbl, n, 3, 2, 2, dt, eps0, mu0, -c, eps_r=er[orig], nh_override=nhv)
    f = [v[orig] * O.image_sign_tmz(code, k) for v, k in ((ez, "ez"), (hx, "hx"), (hy, "hy"))]
    e2, x2, y2, _, _ = O.run_tmz(prob, *f, 12)
    for a, b in ((e1, e2), (x1, x2), (y1, y2)):
        assert np.allclose(a, b[:box.n], rtol=0, atol=1e-11)


def test_regular_grid_whole_shells_equal_the_doubled_periodic_box_3d():
    S, c = 0.3, 1e-3
    dt, eps0, mu0, c0, eta0 = W.units(S)
    cube = W.pec_box_cells((6, 5, 6), 0.0, 2)
    n, nhv = 19, 57  # whole shells of the cubic lattice: 1 + 6 + 12 and + 8 + 6 + 24
    rng = np.random.default_rng(5)
    E0 = rng.standard_normal((3, cube.n))
    H0 = rng.standard_normal((3, cube.n))
    m = cube.normal_axes
    for b in range(3):  # a wall node's odd components are 0 (tangential E, normal H)
        E0[b][(m & (7 & ~(1 << b))) != 0] = 0.0
        H0[b][(m & (1 << b)) != 0] = 0.0
    er = W.eps_r_uniform(cube.n, 6)
    E1, H1, _ = O.run_3d_images(cube, n, 3, 2, 2, dt, eps0, mu0, -c, E0, H0, 6, eps_r=er, nh_override=nhv)
    dbl, orig, code = O.mirror_doubled(cube)
    prob, _ = O.max3d_collocated(dbl, n, 3, 2, 2, dt, eps0, mu0, -c, eps_r=er[orig], nh_override=nhv)
    Ed = np.stack([E0[b][orig] * O.image_sign_3d(code, "e", b) for b in range(3)])
    Hd = np.stack([H0[b][orig] * O.image_sign_3d(code, "h", b) for b in range(3)])
    E2, H2, _, _ = O.run_3d(prob, Ed, Hd, 6)
    assert np.allclose(E1, E2[:, :cube.n], rtol=0, atol=1e-11)
    assert np.allclose(H1, H2[:, :cube.n], rtol=0, atol=1e-11)


def _tm11_image_error(nx, c=4e-3, S=0.5):
    dt, eps0, mu0, c0, eta0 = W.units(S)
    box = W.pec_box_cells((nx, nx), 0.25, 1)
    L = float(nx)
    steps = int(round(4.2 * nx))
    ez, hx, hy = W.tm11_fields(box.xyz, L, c0, mu0, 0.0, -0.5 * dt)
    e1, x1, y1, _, _ = O.run_tmz_images(box, 12, 3, 2, 2, dt, eps0, mu0, -c, ez, hx, hy, steps)
    T = steps * dt
    ea, xa, ya = W.tm11_fields(box.xyz, L, c0, mu0, T, T - 0.5 * dt)
    return np.linalg.norm(np.r_[e1 - ea, x1 - xa, y1 - ya]) / np.linalg.norm(np.r_[ea, xa, ya])


def test_tm11_cavity_with_images_converges():
    e1, e2, e3 = _tm11_image_error(20), _tm11_image_error(40), _tm11_image_error(80)
    assert e1 > e2 > e3
    assert math.log2(e1 / e3) / 2 > 1.5  # about second order
    assert e3 < 1e-3


def test_pec_square_with_images_conserves_energy():
    S, c = 0.5, 4e-3
    dt, eps0, mu0, c0, eta0 = W.units(S)
    box = W.pec_box_cells((40, 40), 0.25, 7)
    ez, hx, hy = W.tm11_fields(box.xyz, 40.0, c0, mu0, 0.0, -0.5 * dt)
    _, _, _, _, en = O.run_tmz_images(box, 12, 3, 2, 2, dt, eps0, mu0, -c, ez, hx, hy, 3000, energy=True)
    u = en / en[0]
    assert np.all(np.abs(u - 1.0) < 2e-3), (u.min(), u.max())


def _tm110_image_error(nx, S=0.5, c=1e-3):
    dt, eps0, mu0, c0, eta0 = W.units(S)
    cube = W.pec_box_cells((nx, nx, nx), 0.25, 7)
    L = float(nx)
    steps = int(round(4 * L))  # the same time in units of L / c0
    E0, H0 = W.tm110_fields_3d(cube.xyz, L, c0, mu0, 0.0, -0.5 * dt)
    E1, H1, _ = O.run_3d_images(cube, 40, 3, 3, 2, dt, eps0, mu0, -c, np.array(E0), np.array(H0), steps)
    T = steps * dt
    Ea, Ha = W.tm110_fields_3d(cube.xyz, L, c0, mu0, T, T - 0.5 * dt)
    ref = np.r_[np.ravel(Ea), np.ravel(Ha)]
    return np.linalg.norm(np.r_[E1.ravel(), H1.ravel()] - ref) / np.linalg.norm(ref)


def test_3d_tm110_cavity_with_images_converges():
    e1, e2, e3 = _tm110_image_error(8), _tm110_image_error(12), _tm110_image_error(16)
    assert e1 > e2 > e3
    assert math.log(e1 / e3) / math.log(2) > 1.2
    assert e3 < 1e-2


def test_3d_pec_cube_with_images_is_stable_one_sided_walls_grow():
    S, c = 0.5, 1e-3
    dt, eps0, mu0, c0, eta0 = W.units(S)
    cube = W.pec_box_cells((10, 10, 10), 0.25, 7)
    E0, H0 = W.tm110_fields_3d(cube.xyz, 10.0, c0, mu0, 0.0, -0.5 * dt)
    _, _, en = O.run_3d_images(cube, 40, 3, 3, 2, dt, eps0, mu0, -c, np.array(E0), np.array(H0), 3000, energy=True)
    u = en / en[0]
    # bounded: the hyperviscosity only damps this 20 h mode
    assert np.all(u <= 1.0 + 1e-6) and u[-1] > 0.5
    walls = W.pec_box((10, 10, 10), 0.25, 7)
    prob, _ = O.max3d_collocated(walls, 40, 3, 3, 2, dt, eps0, mu0, -c)
    E0, H0 = W.tm110_fields_3d(walls.xyz, 9.0, c0, mu0, 0.0, -0.5 * dt)
    _, _, _, en2 = O.run_3d(prob, np.array(E0), np.array(H0), 200, energy=True)
    assert en2[-1] / en2[0] > 1e3


def _corner_of_the_100_cube():
    """The cells [26, 38) x [60, 72) x [0, 8) of the 100^3 PEC box of seed 3 as a
    PEC box of their own (its z = 0 face is the cube's wall): with 40-node
    curl stencils (r^3, degree 3) the layer at that wall holds a mode that
    grows by about e^0.05 per step under Delta^2 HV with c = 1e-3 (the 200^3
    and 100^3 cubes of the 3D workload grew from such places)."""
    full = W.pec_box_cells((100, 100, 100), 0.25, 3)
    lo, size = np.array([26, 60, 0]), np.array([12, 12, 8])
    cell = np.floor(full.xyz).astype(np.int64)
    sel = np.all((cell >= lo) & (cell < lo + size), axis=1)
    return W.NodeSet(xyz=full.xyz[sel] - lo, pec=np.zeros(int(sel.sum()), np.uint8), period=np.zeros(3),
                     box_lo=np.zeros(3), box_hi=size.astype(float), normal_axes=np.zeros(int(sel.sum()), np.uint8))


def test_wall_sized_stencils_are_the_plain_stencils_of_each_size():
    box = W.pec_box_cells((6, 7, 5), 0.25, 17)
    dt, eps0, mu0, c0, eta0 = W.units(0.5)
    p = O.max3d_images(box, 40, 3, 3, 2, dt, eps0, mu0, -1e-3, n_wall=44)
    sizes = O.wall_sizes(box, 40, 44)
    assert set(np.unique(sizes)) == {40, 44}
    dbl, ids, orig, code = O.image_stencils(box, 71)
    for n_use in (40, 44):
        sel = np.nonzero(sizes == n_use)[0]
        ref = O.weights(box.xyz[sel], dbl.xyz, dbl.period, ids[sel], n_use, 3, 3, O.OP_GRAD)
        assert np.array_equal(p.c.w[:, sel, :n_use], ref)
        assert not np.any(p.c.w[:, sel, n_use:])
        assert np.array_equal(p.c.idx[sel], orig[ids[sel, :44]])
    # every weight row still differentiates the monomials up to degree 3 exactly
    rel = dbl.xyz[ids[:, :44]] - box.xyz[:, None, :]
    rel -= dbl.period * np.round(rel / dbl.period)  # minimum image on the doubled box
    for e in O.monomials(3, 3):
        vals = np.prod(rel ** e[None, None, :], axis=2)
        for a in range(3):
            want = float(e[a] == 1 and e.sum() == 1)
            got = np.einsum("ij,ij->i", p.c.w[a], vals)
            assert np.max(np.abs(got - want)) < 1e-8


def test_a_larger_wall_layer_stencil_removes_the_growing_wall_mode():
    box = _corner_of_the_100_cube()
    dt, eps0, mu0, c0, eta0 = W.units(0.5)
    rng = np.random.default_rng(1)
    E0, H0 = rng.standard_normal((3, box.n)), rng.standard_normal((3, box.n))
    _, _, en40 = O.run_3d_images(box, 40, 3, 3, 2, dt, eps0, mu0, -1e-3, E0, H0, 300, energy=True)
    _, _, en44 = O.run_3d_images(box, 40, 3, 3, 2, dt, eps0, mu0, -1e-3, E0, H0, 300, energy=True, n_wall=44)
    assert en40[-1] / en40[0] > 1e3
    assert np.all(en44 / en44[0] <= 1.0 + 1e-6)
