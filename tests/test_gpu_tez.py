"""TEz mode through the E/H duality (Sec. 2): the TMz kernels, created with
exchanged constants and fed (Hz, -Ex, -Ey), against TEz steppers written here
directly from the TEz equations
    dEx/dt = (1/eps) dHz/dy,  dEy/dt = -(1/eps) dHz/dx,
    dHz/dt = (1/mu) (dEx/dy - dEy/dx)
(E at half steps, Hz at whole steps, hyperviscosity gamma Delta^alpha on every
component as in Eq. 19), with the oracle's weights for the meshless step."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
M = pytest.importorskip("paper_2508_18205_gb300")


def test_tez_yee_by_duality():
    ctx = M.Ctx(0)
    nx, ny, S, steps = 48, 40, 0.5, 120
    dt, eps0, mu0, c0, eta0 = W.units(S)
    eps0, mu0 = 1.3 * eps0, mu0 / 1.3  # unequal constants: a swap would show
    rng = np.random.default_rng(8)
    hz, ex, ey = (rng.standard_normal((ny, nx)) for _ in range(3))
    e2, m2 = M.tez_constants(eps0, mu0)
    y = M.Yee(ctx, nx, ny, M.MFD_FP64, dt, 1.0, e2, m2)
    for name, v in (("Hz", hz), ("Ex", ex), ("Ey", ey)):
        M.tez_set(y, name, v)
    y.step(steps)
    # TEz Yee: Hz[j][i] at (i, j), Ex[j][i] at (i, j + 1/2), Ey[j][i] at (i + 1/2, j)
    for _ in range(steps):
        ex = ex + dt / eps0 * (np.roll(hz, -1, 0) - hz)
        ey = ey - dt / eps0 * (np.roll(hz, -1, 1) - hz)
        hz = hz + dt / mu0 * ((ex - np.roll(ex, 1, 0)) - (ey - np.roll(ey, 1, 1)))
    for name, want in (("Hz", hz), ("Ex", ex), ("Ey", ey)):
        got = M.tez_get(y, name)
        assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want)), name


def test_tez_meshless_by_duality():
    ctx = M.Ctx(0)
    S, c, steps = 0.5, 4e-3, 60
    dt, eps0, mu0, c0, eta0 = W.units(S)
    eps0, mu0 = 1.2 * eps0, mu0 / 1.2
    nodes = W.periodic_box((22, 18), 0.25, 61)
    mu_r = 1.0 + 0.5 * np.random.default_rng(3).random(nodes.n)
    gamma = -c  # alpha = 2
    prob, _ = O.tmz_collocated(nodes, 12, 3, 2, 2, dt, eps0, mu0, gamma)
    Dx, Dy, V = prob.hc.w[0], prob.hc.w[1], prob.hv.w[0]
    ic, iv = prob.hc.idx, prob.hv.idx
    rng = np.random.default_rng(4)
    hz, ex, ey = (rng.standard_normal(nodes.n) for _ in range(3))
    nd = M.Nodes(ctx, nodes.xyz, nodes.period)
    st = M.Stencils(nd, nd, 31)
    cw = M.Weights(st, 12, 3, 2, M.MFD_OP_GRAD)
    hw = M.Weights(st, 31, 5, 4, M.MFD_OP_LAP_POW, 2)
    e2, m2 = M.tez_constants(eps0, mu0)
    sim = M.Sim(ctx, 2, M.MFD_FP64, dt, e2, m2, gamma, cw, hw)
    sim.set_materials(mu_r, None)  # TMz eps_r = TEz mu_r
    for name, v in (("Hz", hz), ("Ex", ex), ("Ey", ey)):
        M.tez_set(sim, name, v)
    sim.step(steps)

    def ap(w, idx, f):
        return np.sum(w * f[idx], axis=1)

    for _ in range(steps):
        ex1 = ex + dt / eps0 * (ap(Dy, ic, hz) + gamma * ap(V, iv, ex))
        ey1 = ey + dt / eps0 * (-ap(Dx, ic, hz) + gamma * ap(V, iv, ey))
        hz = hz + dt / (mu0 * mu_r) * (ap(Dy, ic, ex1) - ap(Dx, ic, ey1) + gamma * ap(V, iv, hz))
        ex, ey = ex1, ey1
    got = np.concatenate([M.tez_get(sim, n) for n in ("Hz", "Ex", "Ey")])
    want = np.concatenate([hz, ex, ey])
    assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want)
