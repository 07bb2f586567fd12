"""Hyperviscosity search on the GPU: per right-hand-side coefficients and
energies of the batched kernel against independent oracle runs, and
mfd_hv_search against the oracle's search on the same problem."""
import math

import numpy as np
import pytest

import oracle as O
import oracle.hv_search as S
import workloads as W

pytestmark = pytest.mark.gpu
M = pytest.importorskip("paper_2508_18205_gb300")

COURANT = 1 / (10 * math.sqrt(2))  # Sec. 6
NX, N, PHS, POLY, ALPHA = 24, 30, 5, 4, 2


def _setup(ctx):
    dt, eps0, mu0, c0, eta0 = W.units(COURANT)
    nodes = W.periodic_box((NX, NX), 0.25, 41)
    nhv = 2 * math.comb(2 * ALPHA + 2, 2) + 1
    nd = M.Nodes(ctx, nodes.xyz, nodes.period)
    st = M.Stencils(nd, nd, max(N, nhv))
    cw = M.Weights(st, N, PHS, POLY, M.MFD_OP_GRAD)
    hw = M.Weights(st, nhv, 2 * ALPHA + 1, 2 * ALPHA, M.MFD_OP_LAP_POW, ALPHA)
    ez, hx, hy = W.gaussian_pulse(nodes.xyz, NX, NX / 2, 2.0, c0, eta0, dt, None)
    prob, _ = O.tmz_collocated(nodes, N, PHS, POLY, ALPHA, dt, eps0, mu0, 0.0)
    return dict(dt=dt, eps0=eps0, mu0=mu0, nodes=nodes, keep=(nd, st), cw=cw, hw=hw, ez=ez, hx=hx, hy=hy, prob=prob)


def test_batch_gamma_and_energy_per_rhs():
    """16 right-hand sides from the same fields, each with its own gamma:
    fields and Eq. 20 energies after 300 steps equal 16 oracle runs (FP32)."""
    import dataclasses
    ctx = M.Ctx(0)
    P = _setup(ctx)
    bt = M.Batch(ctx, [(P["cw"], P["hw"], P["dt"], P["eps0"], P["mu0"], -1e-3)], nrhs=16)
    lcs = np.linspace(-4.0, -2.0, 16)
    gam = -(10.0 ** lcs)  # (-1)^(alpha - 1) = -1
    bt.set_gamma(0, gam)
    for comp, v in ((M.MFD_EZ, P["ez"]), (M.MFD_HX, P["hx"]), (M.MFD_HY, P["hy"])):
        bt.set_field(0, comp, np.repeat(v[:, None], 16, axis=1))
    u0 = bt.energy(0)
    steps = 300
    bt.step(steps)
    u1 = bt.energy(0)
    got = bt.get_field(0, M.MFD_EZ)
    for r in range(16):
        p = dataclasses.replace(P["prob"], gamma=gam[r])
        e = O.run_tmz(p, P["ez"], P["hx"], P["hy"], steps + 1, energy=True)[4]  # U at the start of each step
        ez = O.run_tmz(p, P["ez"], P["hx"], P["hy"], steps)[0]
        assert np.linalg.norm(got[:, r] - ez) <= 1e-5 * np.linalg.norm(ez), r
        assert abs(u0[r] - e[0]) <= 1e-6 * e[0]
        assert abs(u1[r] - e[steps]) <= 1e-5 * e[steps], (r, u1[r], e[steps])


def _decided(um, tol):
    """Oracle decisions that FP32 rounding cannot flip: clearly below or above 1 + tol."""
    return um <= 1.0 + 0.5 * tol or um >= 1.0 + 2.0 * tol


def test_hv_search_matches_oracle():
    ctx = M.Ctx(0)
    P = _setup(ctx)
    lo, hi, ncand, rounds, nsteps, every, tol = -4.0, -1.9, 16, 2, 3000, 100, 0.01
    c, hist = M.hv_search(ctx, P["cw"], P["hw"], P["dt"], P["eps0"], P["mu0"], P["ez"], P["hx"], P["hy"], lo, hi,
                          ncand=ncand, rounds=rounds, nsteps=nsteps, check_every=every, tol=tol)
    run = S.tmz_runner(P["prob"], P["ez"], P["hx"], P["hy"], nsteps, every, ALPHA)
    rc, rhist = S.search(run, lo, hi, ncand, rounds, tol)
    assert math.isfinite(c) and math.isfinite(rc)
    for r in range(rounds):
        g = hist[r]
        o = np.array(rhist[r])
        if not np.allclose(g[:, 0], o[:, 0], atol=1e-12):
            break  # an earlier near-threshold decision moved the interval
        for k in range(ncand):
            if _decided(o[k, 1], tol):
                assert (g[k, 1] <= 1 + tol) == (o[k, 1] <= 1 + tol), (r, k, g[k], o[k])
            if o[k, 1] <= 1.5:
                assert abs(g[k, 2] - o[k, 2]) <= 1e-3 * o[k, 2], (r, k, g[k], o[k])
    # the answers agree to the resolution of the search (two final intervals)
    width = (hi - lo) / ncand ** rounds
    assert abs(math.log10(c) - rc) <= 2 * width + 1e-12, (math.log10(c), rc)
    # and the GPU's answer is stable in the oracle's own run
    (um, ue), = run([math.log10(c)])
    assert um <= 1.0 + 2 * tol


def test_hv_search_without_a_stable_candidate_fails_cleanly():
    ctx = M.Ctx(0)
    P = _setup(ctx)
    with pytest.raises(M.MfdError) as ei:
        M.hv_search(ctx, P["cw"], P["hw"], P["dt"], P["eps0"], P["mu0"], P["ez"], P["hx"], P["hy"], -9.0, -6.0,
                    ncand=8, rounds=2, nsteps=3000, check_every=100, tol=0.01)
    assert ei.value.status == M.MFD_ERR_UNSTABLE
