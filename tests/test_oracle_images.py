"""Pins of the image treatment of PEC walls (a reading: the paper only uses
periodic boxes). A perfectly conducting wall acts as a mirror: the tangential
E and the normal H are odd under the reflection, the normal E and the
tangential H even, so a PEC box on [0, L] per axis is a periodic box of period
2 L holding fields of those parities, and stencils near a wall take the mirror
images of the nodes with signed values. The oracle computes this on the
doubled periodic box (mirror_doubled) with its pinned periodic stepper.

* The parity table equals the closed-form TM11 (2D) and TM110 (3D) cavity modes
  evaluated at the mirrored positions.
* The doubled box holds every node once (a wall node is its own image).
* The TM11 cavity with image stencils converges to the exact mode as h -> 0,
  at about second order. No component is held at a wall node: the symmetry of
  the extension is the boundary condition.
* 3D: the PEC cube with image stencils keeps its energy bounded (the same cube
  with one-sided wall stencils grows exponentially, Sec. 5.1 / App. A), and the
  TM110 mode of the cavity is followed.
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


def _tm11_image_error(nx, steps, c=4e-3, S=0.5):
    dt, eps0, mu0, c0, eta0 = W.units(S)
    box = W.pec_box((nx, nx), 0.25, 1)
    L = nx - 1
    ez, hx, hy = W.tm11_fields(box.xyz, L, c0, mu0, 0.0, -0.5 * dt)
    ez[box.pec == 1] = 0.0
    e1, x1, y1, _, _ = O.run_tmz_images(box, 12, 3, 2, 2, dt, eps0, mu0, -c, ez, hx, hy, steps)
    T = steps * dt
    ea, xa, ya = W.tm11_fields(box.xyz, L, c0, mu0, T, T - 0.5 * dt)
    return np.linalg.norm(np.r_[e1 - ea, x1 - xa, y1 - ya]) / np.linalg.norm(np.r_[ea, xa, ya])


def test_tm11_cavity_with_images_converges():
    e1 = _tm11_image_error(21, 84)
    e2 = _tm11_image_error(41, 168)
    e3 = _tm11_image_error(81, 336)
    assert e1 > e2 > e3
    assert math.log2(e1 / e3) / 2 > 1.5  # about second order (the one-sided closure is below that)
    assert e3 < 1e-3


def _tm110_image_error(nx, S=0.5, c=1e-3):
    dt, eps0, mu0, c0, eta0 = W.units(S)
    cube = W.pec_box((nx, nx, nx), 0.25, 7)
    L = nx - 1.0
    steps = int(round(4 * L))  # the same time in units of L / c0
    E0, H0 = W.tm110_fields_3d(cube.xyz, L, c0, mu0, 0.0, -0.5 * dt)
    E1, H1, _ = O.run_3d_images(cube, 40, 3, 3, 2, dt, eps0, mu0, -c, np.array(E0), np.array(H0), steps)
    T = steps * dt
    Ea, Ha = W.tm110_fields_3d(cube.xyz, L, c0, mu0, T, T - 0.5 * dt)
    ref = np.r_[np.ravel(Ea), np.ravel(Ha)]
    return np.linalg.norm(np.r_[E1.ravel(), H1.ravel()] - ref) / np.linalg.norm(ref)


def test_3d_tm110_cavity_with_images_converges():
    e1, e2, e3 = _tm110_image_error(9), _tm110_image_error(13), _tm110_image_error(17)
    assert e1 > e2 > e3
    assert math.log(e1 / e3) / math.log(16 / 8) > 1.2
    assert e3 < 1e-2


def test_3d_pec_cube_with_images_is_stable_one_sided_walls_grow():
    S, c = 0.5, 1e-3
    dt, eps0, mu0, c0, eta0 = W.units(S)
    cube = W.pec_box((10, 10, 10), 0.25, 7)
    E0, H0 = W.tm110_fields_3d(cube.xyz, 9.0, c0, mu0, 0.0, -0.5 * dt)
    _, _, en = O.run_3d_images(cube, 40, 3, 3, 2, dt, eps0, mu0, -c, np.array(E0), np.array(H0), 600, energy=True)
    u = en / en[0]
    assert np.all(u <= 1.0 + 1e-3) and u[-1] > 0.5  # bounded; the hyperviscosity damps this 18 h mode
    prob, _ = O.max3d_collocated(cube, 40, 3, 3, 2, dt, eps0, mu0, -c)
    _, _, _, en2 = O.run_3d(prob, np.array(E0), np.array(H0), 200, energy=True)
    assert en2[-1] / en2[0] > 1e3
