"""The headline workload's problem (staggered periodic pulse: n = 30 curl
stencils with PHS r^5 and degree-4 monomials, Delta^3 hyperviscosity on 57
nodes, Courant number 0.5) on a 160 x 160 + 160 x 160 sub-square, over the
whole 5000 steps of the configuration, against the FP64 oracle at every 100th
step (Eq. 19): FP32 with compensated sums and plain FP32 within 1e-5 relative
L2 of all fields together at every check and over the probe series; FP64
within 1e-10.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_2508_18205_gb300")
bench = pytest.importorskip("bench")


def test_pulse_5000_steps_against_oracle_every_100():
    ctx = M.Ctx(0)
    nx, steps, every = 160, 5000, 100
    g = bench.pulse_reduced_gpu(M, ctx, nx, steps, every)
    p = bench.PARAMS
    dt, eps0, mu0, c0, eta0 = W.units(p["S"])
    e, h = bench.node_sets(nx)
    prob = O.tmz_staggered(e, h, p["n"], p["k"], p["m"], p["alpha"], dt, eps0, mu0,
                           p["c"] * (-1) ** (p["alpha"] - 1))
    ref = list(bench.pulse_fields(e, h, nx, dt))
    probes = W.interior_nodes(e, 16, 24)
    rp = []
    for k in range(steps // every):
        o = O.run_tmz(prob, *ref, every, step0=k * every, probes=probes)
        ref = list(o[:3])
        rp.append(o[3])
        r = np.concatenate(ref)
        for tag, tol in (("fp32_compensated", 1e-5), ("fp32_plain", 1e-5), ("fp64", 1e-10)):
            got = g[tag]["snaps"][k]
            err = np.linalg.norm(got - r) / np.linalg.norm(r)
            assert err <= tol, (tag, (k + 1) * every, err)
    rp = np.concatenate(rp)
    for tag, tol in (("fp32_compensated", 1e-5), ("fp32_plain", 1e-5), ("fp64", 1e-10)):
        gp = g[tag]["probes"]
        assert gp.shape == rp.shape
        assert np.linalg.norm(gp - rp) <= tol * np.linalg.norm(rp), tag


def test_pec_cube_2000_steps_against_oracle_every_500():
    """The 3D workload's problem (PEC cube by images, 40-node curl stencils and
    44 in the wall layer, Delta^2 HV, eps_r field, TM110 fields, Courant
    number 0.5) on a 24^3 cube over the configuration's 2000 steps, against the
    FP64 oracle every 500 steps: FP32 (compensated) within 1e-5, FP64 within
    1e-10, every field; the oracle's energy stays within 1 % of its start."""
    ctx = M.Ctx(0)
    C = bench.CUBE
    S, c, n, k, m, alpha = (C[x] for x in ("S", "c", "n", "k", "m", "alpha"))
    dt, eps0, mu0, c0, eta0 = W.units(S)
    sim32, keep, nodes, er, E0, H0, _ = bench._pec_cube(M, ctx, 24)
    nd, st, cw, hw = keep
    sim64 = M.Sim(ctx, 3, M.MFD_FP64, dt, eps0, mu0, -c, cw, hw)
    sim64.set_materials(er, None)
    for comp, v in zip(range(6), (*E0, *H0)):
        sim64.set_field(comp, v)
    prob = O.max3d_images(nodes, n, k, m, alpha, dt, eps0, mu0, -c, eps_r=er, n_wall=C["n_wall"])
    RE, RH = E0, H0
    u = []
    for blk in range(4):
        RE, RH, _, en = O.run_3d(prob, RE, RH, 500, step0=500 * blk, energy=True)
        u.append(en)
        ref = np.concatenate([RE.ravel(), RH.ravel()])
        for sim, tol in ((sim32, 1e-5), (sim64, 1e-10)):
            sim.step(500)
            got = np.concatenate([sim.get_field(a) for a in range(6)])
            err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert err <= tol, (tol, 500 * (blk + 1), err)
    u = np.concatenate(u)
    assert np.all(np.abs(u / u[0] - 1.0) <= 1e-2)
