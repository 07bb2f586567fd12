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
