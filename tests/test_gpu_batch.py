"""Batched domains x right-hand sides (one persistent cooperative kernel) against the oracle.

Each domain (PEC squares and disks of different sizes and stencil sizes
n in {12, 20, 30, 40}, PHS r^3 with the largest m such that 2 M_m <= n,
Delta^2 hyperviscosity) carries R right-hand sides; right-hand side r has its
own random initial fields and its own Ricker source. Every right-hand side of
every domain must match an independent single-RHS oracle run: relative L2
over the domain's fields (all right-hand sides) and probe series within 1e-5
(FP32).
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_2508_18205_gb300")

S, C_HV, ALPHA = 0.5, 4e-3, 2


def _domains(ctx, specs):
    dt, eps0, mu0, c0, eta0 = W.units(S)
    doms, keep = [], []
    for ns, n in specs:
        m = W.poly_degree_for(n)
        nd = M.Nodes(ctx, ns.xyz, ns.period)
        st = M.Stencils(nd, nd, max(n, 31))
        cw = M.Weights(st, n, 3, m, M.MFD_OP_GRAD)
        hw = M.Weights(st, 31, 5, 4, M.MFD_OP_LAP_POW, ALPHA)
        doms.append((cw, hw, dt, eps0, mu0, -C_HV))
        keep.append((nd, st))
    return doms, keep


@pytest.mark.parametrize("R,variant", [(16, 0), (16, 1), (4, 0), (32, 1), (16, 2), (16, 3), (8, 2), (32, 3)])
def test_batch_matches_single_rhs_oracle(R, variant):
    ctx = M.Ctx(0)
    dt, eps0, mu0, c0, eta0 = W.units(S)
    specs = [(W.pec_box((30, 30), 0.25, 1), 12), (W.disk(15.0, 0.25, 2), 20),
             (W.pec_box((41, 33), 0.25, 3), 30), (W.disk(19.5, 0.25, 4), 40),
             (W.pec_box((9, 9), 0.25, 5), 12)]
    if R != 16:
        specs = specs[:2]
    doms, keep = _domains(ctx, specs)
    bt = M.Batch(ctx, doms, nrhs=R)
    bt.set_variant(variant)
    assert bt.variant == variant
    nsteps = 150
    rng = np.random.default_rng(R)
    init, srcs, probes = [], [], []
    for d, (ns, n) in enumerate(specs):
        eps = W.eps_r_uniform(ns.n, 100 + d)
        bt.set_materials(d, eps, ns.pec)
        f = 0.1 * rng.standard_normal((3, ns.n, R))
        f[0][ns.pec == 1] = 0
        for c, comp in enumerate((M.MFD_EZ, M.MFD_HX, M.MFD_HY)):
            bt.set_field(d, comp, f[c])
        src = W.ricker_sources(ns, R, 200 + d, c0, nrhs=R, one_per_rhs=True)
        bt.set_sources(d, src.node, src.rhs, src.amp, src.f0, src.t0)
        pr = W.interior_nodes(ns, 4, 300 + d)
        bt.set_probes(d, pr, nsteps)
        init.append((f, eps))
        srcs.append(src)
        probes.append(pr)
    bt.step(nsteps)
    for d, (ns, n) in enumerate(specs):
        f, eps = init[d]
        prob, _ = O.tmz_collocated(ns, n, 3, W.poly_degree_for(n), ALPHA, dt, eps0, mu0, -C_HV, eps_r=eps)
        got = [bt.get_field(d, comp) for comp in (M.MFD_EZ, M.MFD_HX, M.MFD_HY)]
        gp = bt.read_probes(d)
        ref = [np.zeros((ns.n, R)) for _ in range(3)]
        rp = np.zeros((nsteps, len(probes[d]), R))
        for r in range(R):
            sel = srcs[d].rhs == r
            sub = W.Sources(node=srcs[d].node[sel], rhs=srcs[d].rhs[sel], amp=srcs[d].amp[sel],
                            f0=srcs[d].f0[sel], t0=srcs[d].t0[sel])
            e1, x1, y1, p1, _ = O.run_tmz(prob, f[0][:, r], f[1][:, r], f[2][:, r], nsteps, sources=sub,
                                          probes=probes[d])
            ref[0][:, r], ref[1][:, r], ref[2][:, r] = e1, x1, y1
            rp[:, :, r] = p1
        g = np.concatenate([x.reshape(-1) for x in got])
        rr = np.concatenate([x.reshape(-1) for x in ref])
        err = np.linalg.norm(g - rr) / np.linalg.norm(rr)
        perr = np.linalg.norm(gp - rp) / np.linalg.norm(rp)
        assert err <= 1e-5, (d, err)
        assert perr <= 1e-5, (d, perr)
        assert np.all(got[0][ns.pec == 1] == 0)


@pytest.mark.parametrize("variant", [0, 2])
def test_batch_repeated_steps_continue(variant):
    """Two step calls of k steps equal one call of 2k steps (the step counter, the sources
    and, in variant 2, H* carry on)."""
    ctx = M.Ctx(0)
    dt, eps0, mu0, c0, eta0 = W.units(S)
    specs = [(W.pec_box((20, 20), 0.25, 7), 12), (W.disk(11.0, 0.25, 8), 20)]
    out = []
    for split in (False, True):
        doms, keep = _domains(ctx, specs)
        bt = M.Batch(ctx, doms, nrhs=16)
        bt.set_variant(variant)
        for d, (ns, n) in enumerate(specs):
            bt.set_materials(d, None, ns.pec)
            src = W.ricker_sources(ns, 16, 400 + d, c0, nrhs=16, one_per_rhs=True)
            bt.set_sources(d, src.node, src.rhs, src.amp, src.f0, src.t0)
        if split:
            bt.step(40)
            bt.step(40)
        else:
            bt.step(80)
        out.append([bt.get_field(d, M.MFD_EZ) for d in range(len(specs))])
    for a, b in zip(*out):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("R", [16, 8])
def test_variants_are_bit_identical_and_autotune_leaves_the_state(R):
    """Variants with and without stream prefetch (three or four resident blocks
    per SM) take every stencil sum in the same order: within each form of the
    H row's HV term (H pass: variants 0, 1; E pass of the step before, with H*:
    variants 2, 3) the fields, probes and energies agree bit for bit, and the
    two forms agree to rounding (1e-6 relative). The autotuner times all four
    and puts the fields, probes and step count back."""
    ctx = M.Ctx(0)
    dt, eps0, mu0, c0, eta0 = W.units(S)
    specs = [(W.pec_box((26, 22), 0.25, 11), 12), (W.disk(13.0, 0.25, 12), 30), (W.pec_box((17, 17), 0.25, 13), 40),
             (W.disk(8.0, 0.25, 14), 20)]
    doms, keep = _domains(ctx, specs)
    runs = []
    for variant in (0, 1, 2, 3):
        bt = M.Batch(ctx, doms, nrhs=R)
        bt.set_variant(variant)
        for d, (ns, n) in enumerate(specs):
            bt.set_materials(d, W.eps_r_uniform(ns.n, 20 + d), ns.pec)
            src = W.ricker_sources(ns, R, 30 + d, c0, nrhs=R, one_per_rhs=True)
            bt.set_sources(d, src.node, src.rhs, src.amp, src.f0, src.t0)
            bt.set_probes(d, W.interior_nodes(ns, 3, 40 + d), 200)
        bt.step(70)
        if variant == 1:
            before = [bt.get_field(d, c) for d in range(len(specs)) for c in (M.MFD_EZ, M.MFD_HX, M.MFD_HY)]
            probes_before = bt.read_probes(0)
            chosen, ms = bt.autotune(5)
            assert chosen in (0, 1, 2, 3) and bt.variant == chosen and np.all(ms > 0) and ms.shape == (4,)
            after = [bt.get_field(d, c) for d in range(len(specs)) for c in (M.MFD_EZ, M.MFD_HX, M.MFD_HY)]
            for x, y in zip(before, after):
                assert np.array_equal(x, y)
            assert np.array_equal(bt.read_probes(0), probes_before)
            bt.set_variant(1)
        bt.step(50)
        runs.append(([bt.get_field(d, c) for d in range(len(specs)) for c in (M.MFD_EZ, M.MFD_HX, M.MFD_HY)],
                     [bt.read_probes(d) for d in range(len(specs))], [bt.energy(d) for d in range(len(specs))]))
    for i, j in ((0, 1), (2, 3)):
        for a, b in zip(runs[i][0], runs[j][0]):
            assert np.array_equal(a, b)
        for a, b in zip(runs[i][1], runs[j][1]):
            assert a.shape[0] == 120 and np.array_equal(a, b)
        for a, b in zip(runs[i][2], runs[j][2]):
            assert np.array_equal(a, b)
    for a, b in zip(runs[0][0], runs[2][0]):
        assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(a)
    for a, b in zip(runs[0][1], runs[2][1]):
        assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(a)
    for a, b in zip(runs[0][2], runs[2][2]):
        assert np.allclose(a, b, rtol=1e-6, atol=0)
