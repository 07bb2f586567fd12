"""Parity at the benchmark's full size (pulse2d-staggered, 1000 x 1000 E nodes and
1000 x 1000 H nodes), in the launch configuration bench.py times.

The oracle cannot step 2M nodes in seconds, so it computes outputs one by one:
* kNN: the GPU stencils of sampled centres equal the oracle's (bit-exact).
* weights: the GPU weights of sampled centres match the oracle's (1e-8, as in
  the small-size tests).
* one leapfrog step from the seeded initial pulse: the new Ez at 48 sampled
  E nodes and the new H at 48 sampled H nodes (plus every H node the sampled
  E nodes depend on), where the pulse is, match the oracle's step from the
  same seeded state: relative L2 over the sampled values 1e-12 in FP64, 1e-6
  in FP32 (one step of FP32 arithmetic and FP32-rounded weights). Every input
  of the oracle comes from the seeded generators, none from the GPU.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_2508_18205_gb300")
bench = pytest.importorskip("bench")


@pytest.fixture(scope="module")
def setup():
    ctx = M.Ctx(0)
    e, h = bench.node_sets(1000)
    wts, _, nhv = bench.build_weights(M, ctx, e, h)
    return ctx, e, h, wts, nhv


def test_fullsize_stencils_and_weights_sampled(setup):
    ctx, e, h, wts, nhv = setup
    hc, hv, ec, ev = wts
    p = bench.PARAMS
    ids_h = W.interior_nodes(h, 64, 81)
    ids_e = W.interior_nodes(e, 64, 82)
    for w, xs_set, xc_set, ids, n, k, m, op, alpha in (
            (hc, e, h, ids_h, p["n"], p["k"], p["m"], O.OP_GRAD, 0),
            (hv, h, h, ids_h, nhv, 2 * p["alpha"] + 1, 2 * p["alpha"], O.OP_LAP_POW, p["alpha"]),
            (ec, h, e, ids_e, p["n"], p["k"], p["m"], O.OP_GRAD, 0),
            (ev, e, e, ids_e, nhv, 2 * p["alpha"] + 1, 2 * p["alpha"], O.OP_LAP_POW, p["alpha"])):
        gi = w.st.read()[ids]
        ri = O.knn_cells(xc_set.xyz[ids], xs_set.xyz, xs_set.period, n)
        assert np.array_equal(gi, ri)
        gw = w.read()[:, ids, :]
        rw = O.weights(xc_set.xyz[ids], xs_set.xyz, xs_set.period, ri, n, k, m, op, alpha)
        scale = np.max(np.abs(rw), axis=2, keepdims=True)
        assert np.max(np.abs(gw - rw) / scale) <= 1e-8


@pytest.mark.parametrize("prec,tol", [(1, 1e-12), (0, 1e-6)])
def test_fullsize_one_step_sampled(setup, prec, tol):
    ctx, e, h, wts, nhv = setup
    p = bench.PARAMS
    sim = bench.make_sim(M, ctx, wts, prec, prec == 0)
    dt, eps0, mu0, c0, eta0 = W.units(p["S"])
    ez, hx, hy = bench.pulse_fields(e, h, 1000, dt)
    sim.set_field(M.MFD_EZ, ez)
    sim.set_field(M.MFD_HX, hx)
    sim.set_field(M.MFD_HY, hy)
    s0 = [ez, hx, hy]
    sim.step(1)
    s1 = [sim.get_field(c) for c in (M.MFD_EZ, M.MFD_HX, M.MFD_HY)]
    # sample where the pulse is (the fields are ~0 far from it)
    near_e = np.nonzero(np.abs(ez) > 0.05)[0]
    near_h = np.nonzero(np.abs(hy) > 0.05)[0]
    rng = np.random.default_rng(5)
    ids_e = np.sort(rng.choice(near_e, 48, replace=False))
    ids_h = np.sort(rng.choice(near_h, 48, replace=False))
    gamma = p["c"] * (-1) ** (p["alpha"] - 1)
    ez1, hx1, hy1, hs = O.tmz_sample_step(e, h, ids_e, p["n"], p["k"], p["m"], p["alpha"], dt, eps0, mu0,
                                          gamma, s0[0], s0[1], s0[2], h_ids=ids_h)
    got = np.concatenate([s1[0][ids_e], s1[1][hs], s1[2][hs]])
    ref = np.concatenate([ez1, hx1, hy1])
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= tol, err


def _crop(nodes, lo, size):
    """The cells [lo, lo + size) of a cell-centred PEC box as a PEC box of their
    own (shifted to the origin; coordinates shift exactly)."""
    cell = np.floor(nodes.xyz).astype(np.int64)
    sub = np.nonzero(np.all((cell >= lo) & (cell < np.asarray(lo) + size), axis=1))[0]
    crop = W.NodeSet(xyz=nodes.xyz[sub] - np.asarray(lo, dtype=np.float64), pec=np.zeros(len(sub), np.uint8),
                     period=np.zeros(3), box_lo=np.zeros(3), box_hi=np.asarray(size, dtype=np.float64),
                     normal_axes=np.zeros(len(sub), np.uint8))
    return crop, sub


def test_cube3d_8M_one_step_sampled():
    """The 3D workload at its full size: the 200^3 PEC cube (walls by images,
    40-node curl stencils and 44 in the layer next to the walls, Delta^2 HV on
    71 nodes, eps_r field), one step from seeded random fields on all six
    components, in the launch configuration bench.py times. Sampled against
    the oracle: 24 nodes away from the walls (the oracle's plain stencils,
    which no image reaches there), 24 in a corner and 24 next to the middle of
    the x = 200 face (the oracle's image scheme on a box of cells around them
    whose other faces lie beyond what those nodes' first step reads). FP32
    1e-6, FP64 1e-12."""
    ctx = M.Ctx(0)
    C = bench.CUBE
    S, c, n, k, m, alpha = (C[x] for x in ("S", "c", "n", "k", "m", "alpha"))
    dt, eps0, mu0, c0, eta0 = W.units(S)
    sim32, keep, nodes, er, _, _, _ = bench._pec_cube(M, ctx, 200)
    del sim32
    nd, st, cw, hw = keep
    rng = np.random.default_rng(12)
    E0 = rng.standard_normal((3, nodes.n))
    H0 = rng.standard_normal((3, nodes.n))
    cell = np.floor(nodes.xyz).astype(np.int64)
    ids_in = np.sort(rng.choice(np.nonzero(np.all((cell >= 12) & (cell < 188), axis=1))[0], 24, replace=False))
    regions = {"corner": ((0, 0, 0), (20, 20, 20), np.all(cell < 6, axis=1)),
               "face": ((180, 80, 80), (20, 40, 40),
                        (cell[:, 0] >= 194) & np.all((cell[:, 1:] >= 90) & (cell[:, 1:] < 110), axis=1))}
    refs = {}
    RE, RH, hs = O.max3d_sample_step(nodes, ids_in, n, k, m, alpha, dt, eps0, mu0, -c, E0, H0, eps_r=er, h_ids=ids_in)
    refs["interior"] = (ids_in, RE, RH[:, np.searchsorted(hs, ids_in)])
    for name, (lo, size, sel) in regions.items():
        ids = np.sort(rng.choice(np.nonzero(sel)[0], 24, replace=False))
        crop, sub = _crop(nodes, lo, size)
        prob = O.max3d_images(crop, n, k, m, alpha, dt, eps0, mu0, -c, eps_r=er[sub], n_wall=C["n_wall"])
        RE, RH, _, _ = O.run_3d(prob, E0[:, sub], H0[:, sub], 1)
        at = np.searchsorted(sub, ids)
        refs[name] = (ids, RE[:, at], RH[:, at])
    for prec, tol in ((M.MFD_FP32, 1e-6), (M.MFD_FP64, 1e-12)):
        sim = M.Sim(ctx, 3, prec, dt, eps0, mu0, -c, cw, hw, compensated=True)
        sim.set_materials(er, None)
        for comp, v in zip(range(6), (*E0, *H0)):
            sim.set_field(comp, v)
        sim.step(1)
        E1 = np.stack([sim.get_field(a) for a in range(3)])
        H1 = np.stack([sim.get_field(3 + a) for a in range(3)])
        for name, (ids, RE, RH) in refs.items():
            got = np.concatenate([E1[:, ids].ravel(), H1[:, ids].ravel()])
            ref = np.concatenate([RE.ravel(), RH.ravel()])
            err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert err <= tol, (prec, name, err)
        del sim


def test_batched_256_domains_sampled_domains():
    """The batched workload at full size (256 domains, 4.3M nodes, 16 RHS): three
    whole domains (every right-hand side) after 120 steps against single-RHS
    oracle runs (1e-5, FP32)."""
    ctx = M.Ctx(0)
    S, c = 0.5, 4e-3
    dt, eps0, mu0, c0, eta0 = W.units(S)
    specs = W.batch_domains(256, 4)
    doms, keep = [], []
    for ns, n in specs:
        nd = M.Nodes(ctx, ns.xyz, ns.period)
        st = M.Stencils(nd, nd, max(n, 31))
        cw = M.Weights(st, n, 3, W.poly_degree_for(n), M.MFD_OP_GRAD)
        hw = M.Weights(st, 31, 5, 4, M.MFD_OP_LAP_POW, 2)
        doms.append((cw, hw, dt, eps0, mu0, -c))
        keep.append((nd, st))
    bt = M.Batch(ctx, doms, nrhs=16)
    srcs = []
    for d, (ns, n) in enumerate(specs):
        bt.set_materials(d, None, ns.pec)
        src = W.ricker_sources(ns, 16, 500 + d, c0, nrhs=16, one_per_rhs=True)
        bt.set_sources(d, src.node, src.rhs, src.amp, src.f0, src.t0)
        srcs.append(src)
    nsteps = 120
    bt.step(nsteps)
    sizes = np.array([ns.n for ns, _ in specs])
    pick = list(np.argsort(sizes)[:2]) + [int(np.argsort(sizes)[len(sizes) // 2])]
    for d in pick:
        ns, n = specs[d]
        prob, _ = O.tmz_collocated(ns, n, 3, W.poly_degree_for(n), 2, dt, eps0, mu0, -c)
        got = bt.get_field(int(d), M.MFD_EZ)
        ref = np.zeros((ns.n, 16))
        z = np.zeros(ns.n)
        for r in range(16):
            sel = srcs[d].rhs == r
            sub = W.Sources(node=srcs[d].node[sel], rhs=srcs[d].rhs[sel], amp=srcs[d].amp[sel],
                            f0=srcs[d].f0[sel], t0=srcs[d].t0[sel])
            ref[:, r] = O.run_tmz(prob, z, z, z, nsteps, sources=sub)[0]
        assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref), d


def test_fullsize_index_formats_bit_identical(setup):
    """The benchmark's launch configuration (FP32, compensated sums, 16-bit
    indices with two windows per slice, 32-bit fallback): three steps from
    random fields equal the 32-bit index format on every node, bit for bit."""
    ctx, e, h, wts, nhv = setup
    sim = bench.make_sim(M, ctx, wts, 0, True)
    stats = sim.index_stats()
    for p in ("h", "e"):
        assert stats[p][0] == 1000 * 1000 // 32
        assert 0 < stats[p][1] < stats[p][0] // 50 and 0 < stats[p][2] < stats[p][0] // 50, stats
    rng = np.random.default_rng(83)
    f = [rng.standard_normal(e.n), rng.standard_normal(h.n), rng.standard_normal(h.n)]
    comps = (M.MFD_EZ, M.MFD_HX, M.MFD_HY)
    runs = []
    for fmt in (M.MFD_INDEX_Q16, M.MFD_INDEX_I32):
        sim.set_index_format(fmt)
        for cc, v in zip(comps, f):
            sim.set_field(cc, v)
        sim.step(3)
        runs.append([sim.get_field(cc) for cc in comps])
    for a, b in zip(*runs):
        assert np.array_equal(a, b)
