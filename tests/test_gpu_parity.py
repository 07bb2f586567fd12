"""GPU path (through the C ABI) against the FP64 oracle, element by element.

* kNN stencils: bit-exact (same ids, same order) on regular grids with distance
  ties, jittered grids, periodic boxes (including boxes so small that rings
  wrap), cross-set (staggered) queries, 3D, and node counts that are not a
  multiple of the 32-node slice.
* Weights (FP64 on both sides): max-norm per stencil within 1e-8 of the
  oracle's, relative to the stencil's largest weight; and the GPU weights
  differentiate every monomial of the augmentation degree exactly (1e-10).
* Stepping in FP64: relative L2 error of every field and of the probe series
  within 1e-10 of the oracle (collocated PEC cavity with sources, staggered
  periodic, 3D periodic and PEC). FP32 (plain and compensated sums): relative
  L2 error of all fields together (eta0 = 1) and of the probes within 1e-5.
  (A single near-zero component, such as Hx of an x-directed pulse, is not
  compared on its own in FP32: its norm is set by round-off.)
* Energy (Eq. 20) within 1e-12 of the oracle's in FP64.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_2508_18205_gb300")


@pytest.fixture(scope="module")
def ctx():
    return M.Ctx(0)


def _nodes(kind):
    if kind == "grid2_ties":
        return W.pec_box((40, 40), 0.0, 1)
    if kind == "pec2_ragged":
        return W.pec_box((37, 23), 0.25, 2)
    if kind == "per2":
        return W.periodic_box((64, 64), 0.25, 3)
    if kind == "per2_tiny":
        return W.periodic_box((6, 6), 0.25, 4)
    if kind == "pec3":
        return W.pec_box((16, 16, 16), 0.25, 5)
    if kind == "per3":
        return W.periodic_box((12, 12, 12), 0.25, 6)
    if kind == "grid3_ties":
        return W.periodic_box((9, 9, 9), 0.0, 7)
    raise KeyError(kind)


@pytest.mark.parametrize("kind,n", [("grid2_ties", 31), ("pec2_ragged", 31), ("per2", 57), ("per2_tiny", 20),
                                    ("pec3", 71), ("per3", 40), ("grid3_ties", 27), ("pec2_ragged", 1)])
def test_knn_bit_exact(ctx, kind, n):
    ns = _nodes(kind)
    nd = M.Nodes(ctx, ns.xyz, ns.period)
    got = M.Stencils(nd, nd, n).read()
    ref = O.knn(ns.xyz, ns.xyz, ns.period, n)
    assert np.array_equal(got, ref)


def test_knn_cross_set_bit_exact(ctx):
    e = W.periodic_box((48, 48), 0.25, 8)
    h = W.periodic_box((48, 48), 0.25, 9, offset=(0.5, 0.5))
    de = M.Nodes(ctx, e.xyz, e.period)
    dh = M.Nodes(ctx, h.xyz, h.period)
    assert np.array_equal(M.Stencils(dh, de, 30).read(), O.knn(h.xyz, e.xyz, e.period, 30))
    assert np.array_equal(M.Stencils(de, dh, 30).read(), O.knn(e.xyz, h.xyz, h.period, 30))


def test_morton_permutation_is_a_permutation(ctx):
    ns = _nodes("pec2_ragged")
    nd = M.Nodes(ctx, ns.xyz, ns.period)
    p = nd.permutation()
    assert np.array_equal(np.sort(p), np.arange(ns.n))


WCASES = [
    # (kind, n_use, stencil n, phs_k, m, op, alpha, delta)
    ("pec2_ragged", 12, 31, 3, 2, 0, 0, 0.0),
    ("pec2_ragged", 31, 31, 5, 4, 1, 2, 0.0),
    ("per2", 30, 57, 5, 4, 0, 0, 0.0),
    ("per2", 57, 57, 7, 6, 1, 3, 0.0),
    ("pec3", 40, 71, 3, 3, 0, 0, 0.0),
    ("pec3", 71, 71, 5, 4, 1, 2, 0.0),
    ("pec2_ragged", 12, 31, 3, 2, 2, 0, 0.5),
    ("grid2_ties", 20, 31, 3, 2, 0, 0, 0.0),
]


def _exps(d, m):
    return [e for e in O.monomials(d, m)]


@pytest.mark.parametrize("case", WCASES)
def test_weights_match_oracle(ctx, case):
    kind, n_use, n, k, m, op, alpha, delta = case
    ns = _nodes(kind)
    nd = M.Nodes(ctx, ns.xyz, ns.period)
    st = M.Stencils(nd, nd, n)
    w = M.Weights(st, n_use, k, m, op, alpha, delta).read()
    idx = st.read()
    ref = O.weights(ns.xyz, ns.xyz, ns.period, idx, n_use, k, m, op, alpha, delta)
    scale = np.max(np.abs(ref), axis=2, keepdims=True)
    rel = np.max(np.abs(w - ref) / scale)
    assert rel <= 1e-8, rel
    # monomial exactness of the GPU weights on every node
    d = ns.dim
    rel_xyz = ns.xyz[idx[:, :n_use]] - ns.xyz[:, None, :]
    for a in range(d):
        if ns.period[a] > 0:
            p = ns.period[a]
            r = rel_xyz[..., a]
            rel_xyz[..., a] = np.where(r > p / 2, r - p, np.where(r < -p / 2, r + p, r))
    deg = 2 * alpha if op == 1 else m
    for e in _exps(d, deg):
        pv = np.prod(rel_xyz ** np.asarray(e), axis=2)
        for o in range(w.shape[0]):
            got = np.sum(w[o] * pv, axis=1)
            if op == 1:
                import sympy as sp
                xs = sp.symbols("x0:%d" % d)
                poly = sp.Integer(1)
                for a in range(d):
                    poly *= xs[a] ** int(e[a])
                for _ in range(alpha):
                    poly = sum(sp.diff(poly, xs[a], 2) for a in range(d))
                exact = float(poly.subs({x: 0 for x in xs}))
            else:
                exact = 1.0 if (sum(e) == 1 and e[o] == 1) else 0.0
            sc = np.maximum(np.sum(np.abs(w[o] * pv), axis=1), 1.0)
            assert np.max(np.abs(got - exact) / sc) <= 1e-10, (e, o)


# ------------------------------------------------------------------ stepping

def _gpu_colloc(ctx, nodes, n, k, m, alpha, dt, eps0, mu0, gamma, prec, comp=False, vfd=None):
    import math as _m
    nhv = 2 * _m.comb(2 * alpha + nodes.dim, nodes.dim) + 1
    nd = M.Nodes(ctx, nodes.xyz, nodes.period)
    st = M.Stencils(nd, nd, max(n, nhv))
    if vfd is None:
        curl = M.Weights(st, n, k, m, M.MFD_OP_GRAD)
    else:
        curl = M.Weights(st, n, k, m, M.MFD_OP_GRAD_VFD, 0, vfd)
    hv = M.Weights(st, nhv, 2 * alpha + 1, 2 * alpha, M.MFD_OP_LAP_POW, alpha)
    sim = M.Sim(ctx, nodes.dim, prec, dt, eps0, mu0, gamma, curl, hv, compensated=comp)
    return sim


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _rel_all(got, ref):
    """Relative L2 error over all fields together (eta0 = 1, so E and H share units)."""
    return _rel(np.concatenate(got), np.concatenate(ref))


@pytest.mark.parametrize("prec,comp,tol", [(1, False, 1e-10), (0, False, 1e-5), (0, True, 1e-5)])
def test_collocated_pec_cavity_with_sources(ctx, prec, comp, tol):
    S, c = 0.5, 4e-3
    dt, eps0, mu0, c0, eta0 = W.units(S)
    nodes = W.pec_box((37, 29), 0.25, 11)
    er = W.eps_r_uniform(nodes.n, 12)
    sim = _gpu_colloc(ctx, nodes, 12, 3, 2, 2, dt, eps0, mu0, -c, prec, comp)
    sim.set_materials(er, nodes.pec)
    ez, hx, hy = W.tm11_fields(nodes.xyz, 36.0, c0, mu0, 0.0, -0.5 * dt)
    ez[nodes.pec == 1] = 0
    src = W.ricker_sources(nodes, 3, 13, c0)
    probes = W.interior_nodes(nodes, 16, 14)
    for comp_, v in ((M.MFD_EZ, ez), (M.MFD_HX, hx), (M.MFD_HY, hy)):
        sim.set_field(comp_, v)
    sim.set_sources(src.node, src.amp, src.f0, src.t0)
    sim.set_probes(probes, 300)
    sim.step(300)
    prob, _ = O.tmz_collocated(nodes, 12, 3, 2, 2, dt, eps0, mu0, -c, eps_r=er)
    re, rx, ry, rp, _ = O.run_tmz(prob, ez, hx, hy, 300, sources=src, probes=probes)
    got = [sim.get_field(c) for c in (M.MFD_EZ, M.MFD_HX, M.MFD_HY)]
    assert _rel_all(got, [re, rx, ry]) <= tol
    assert _rel(sim.read_probes(), rp) <= tol
    if prec == 1:  # FP64: every field on its own
        for g, r in zip(got, (re, rx, ry)):
            assert _rel(g, r) <= tol
    assert np.all(got[0][nodes.pec == 1] == 0)


@pytest.mark.parametrize("prec,comp,tol", [(1, False, 1e-10), (0, True, 1e-5)])
def test_staggered_periodic_pulse(ctx, prec, comp, tol):
    S, c, alpha = 0.5, 4e-5, 3
    dt, eps0, mu0, c0, eta0 = W.units(S)
    nx = 40
    e = W.periodic_box((nx, nx), 0.25, 21, seed_line_y=nx // 2)
    h = W.periodic_box((nx, nx), 0.25, 22, offset=(0.5, 0.5))
    de, dh = M.Nodes(ctx, e.xyz, e.period), M.Nodes(ctx, h.xyz, h.period)
    n, nhv = 30, 57
    hc = M.Weights(M.Stencils(dh, de, n), n, 5, 4, M.MFD_OP_GRAD)
    hv = M.Weights(M.Stencils(dh, dh, nhv), nhv, 7, 6, M.MFD_OP_LAP_POW, alpha)
    ec = M.Weights(M.Stencils(de, dh, n), n, 5, 4, M.MFD_OP_GRAD)
    ev = M.Weights(M.Stencils(de, de, nhv), nhv, 7, 6, M.MFD_OP_LAP_POW, alpha)
    sim = M.Sim(ctx, 2, prec, dt, eps0, mu0, c, hc, hv, ec, ev, compensated=comp)
    ez, _, _ = W.gaussian_pulse(e.xyz, nx, nx / 2, 6.0, c0, eta0, dt, 12.0)
    _, hx, hy = W.gaussian_pulse(h.xyz, nx, nx / 2, 6.0, c0, eta0, dt, 12.0)
    sim.set_field(M.MFD_EZ, ez)
    sim.set_field(M.MFD_HX, hx)
    sim.set_field(M.MFD_HY, hy)
    probes = W.interior_nodes(e, 8, 23)
    sim.set_probes(probes, 200)
    sim.step(200)
    prob = O.tmz_staggered(e, h, n, 5, 4, alpha, dt, eps0, mu0, c)
    re, rx, ry, rp, _ = O.run_tmz(prob, ez, hx, hy, 200, probes=probes)
    got = [sim.get_field(c) for c in (M.MFD_EZ, M.MFD_HX, M.MFD_HY)]
    assert _rel_all(got, [re, rx, ry]) <= tol
    assert _rel(sim.read_probes(), rp) <= tol
    if prec == 1:
        for g, r in zip(got, (re, rx, ry)):
            assert _rel(g, r) <= tol


@pytest.mark.parametrize("pec", [False, True])
@pytest.mark.parametrize("prec,tol", [(1, 1e-10), (0, 1e-5)])
def test_3d_maxwell(ctx, pec, prec, tol):
    S, c = 0.5, 1e-3
    dt, eps0, mu0, c0, eta0 = W.units(S)
    nodes = W.pec_box((9, 10, 11), 0.25, 31) if pec else W.periodic_box((10, 10, 10), 0.25, 32)
    er = W.eps_r_smooth_3d(nodes.xyz, np.maximum(nodes.box_hi, 1), 33)
    steps = 8 if pec else 40
    sim = _gpu_colloc(ctx, nodes, 40, 3, 3, 2, dt, eps0, mu0, -c, prec, comp=True)
    sim.set_materials(er, nodes.normal_axes if pec else None)
    rng = np.random.default_rng(3)
    E = rng.standard_normal((3, nodes.n))
    H = rng.standard_normal((3, nodes.n))
    if pec:
        m = nodes.normal_axes
        for b in range(3):
            for a in range(3):
                if a != b:
                    E[b][((m >> a) & 1) == 1] = 0
    for a in range(3):
        sim.set_field(M.MFD_EX + a, E[a])
        sim.set_field(M.MFD_HX + a, H[a])
    sim.step(steps)
    prob, _ = O.max3d_collocated(nodes, 40, 3, 3, 2, dt, eps0, mu0, -c, eps_r=er)
    if not pec:
        prob.wall[:] = 0
    RE, RH, _, _ = O.run_3d(prob, E, H, steps)
    got = [sim.get_field(M.MFD_EX + a) for a in range(3)] + [sim.get_field(M.MFD_HX + a) for a in range(3)]
    assert _rel_all(got, list(RE) + list(RH)) <= tol
    if prec == 1:
        for g, r in zip(got, list(RE) + list(RH)):
            assert _rel(g, r) <= tol


@pytest.mark.parametrize("layout", ["colloc", "stag", "3d"])
def test_energy_matches_oracle(ctx, layout):
    S = 0.5
    dt, eps0, mu0, c0, eta0 = W.units(S)
    rng = np.random.default_rng(7)
    if layout == "colloc":
        nodes = W.pec_box((20, 20), 0.25, 41)
        er = W.eps_r_uniform(nodes.n, 42)
        sim = _gpu_colloc(ctx, nodes, 12, 3, 2, 2, dt, eps0, mu0, -4e-3, 1)
        sim.set_materials(er, nodes.pec)
        prob, _ = O.tmz_collocated(nodes, 12, 3, 2, 2, dt, eps0, mu0, -4e-3, eps_r=er)
        ez, hx, hy = rng.standard_normal((3, nodes.n))
        ez[nodes.pec == 1] = 0
        ne = nh = nodes.n
    elif layout == "stag":
        e = W.periodic_box((20, 20), 0.25, 43)
        h = W.periodic_box((20, 20), 0.25, 44, offset=(0.5, 0.5))
        de, dh = M.Nodes(ctx, e.xyz, e.period), M.Nodes(ctx, h.xyz, h.period)
        hc = M.Weights(M.Stencils(dh, de, 12), 12, 3, 2, M.MFD_OP_GRAD)
        hv = M.Weights(M.Stencils(dh, dh, 31), 31, 5, 4, M.MFD_OP_LAP_POW, 2)
        ec = M.Weights(M.Stencils(de, dh, 12), 12, 3, 2, M.MFD_OP_GRAD)
        ev = M.Weights(M.Stencils(de, de, 31), 31, 5, 4, M.MFD_OP_LAP_POW, 2)
        sim = M.Sim(ctx, 2, 1, dt, eps0, mu0, -1e-3, hc, hv, ec, ev)
        er = W.eps_r_uniform(e.n, 45)
        sim.set_materials(er, None)
        prob = O.tmz_staggered(e, h, 12, 3, 2, 2, dt, eps0, mu0, -1e-3, eps_r=er)
        ez = rng.standard_normal(e.n)
        hx, hy = rng.standard_normal((2, h.n))
        ne, nh = e.n, h.n
    else:
        nodes = W.periodic_box((8, 8, 8), 0.25, 46)
        er = W.eps_r_uniform(nodes.n, 47)
        sim = _gpu_colloc(ctx, nodes, 40, 3, 3, 2, dt, eps0, mu0, -1e-3, 1)
        sim.set_materials(er, None)
        prob, _ = O.max3d_collocated(nodes, 40, 3, 3, 2, dt, eps0, mu0, -1e-3, eps_r=er)
        E = rng.standard_normal((3, nodes.n))
        H = rng.standard_normal((3, nodes.n))
        for a in range(3):
            sim.set_field(M.MFD_EX + a, E[a])
            sim.set_field(M.MFD_HX + a, H[a])
        u_gpu = sim.energy()
        _, _, _, en = O.run_3d(prob, E, H, 1, energy=True)
        assert abs(u_gpu - en[0]) <= 1e-12 * abs(en[0])
        return
    sim.set_field(M.MFD_EZ, ez)
    sim.set_field(M.MFD_HX, hx)
    sim.set_field(M.MFD_HY, hy)
    u_gpu = sim.energy()
    _, _, _, _, en = O.run_tmz(prob, ez, hx, hy, 1, energy=True)
    assert abs(u_gpu - en[0]) <= 1e-12 * abs(en[0])


def test_graph_and_direct_launches_agree(ctx):
    """Long runs replay a captured graph; the result equals step-by-step launches bit for bit."""
    S = 0.5
    dt, eps0, mu0, c0, eta0 = W.units(S)
    e = W.periodic_box((24, 24), 0.25, 51)
    h = W.periodic_box((24, 24), 0.25, 52, offset=(0.5, 0.5))
    sims = []
    for _ in range(2):
        de, dh = M.Nodes(ctx, e.xyz, e.period), M.Nodes(ctx, h.xyz, h.period)
        hc = M.Weights(M.Stencils(dh, de, 12), 12, 3, 2, M.MFD_OP_GRAD)
        hv = M.Weights(M.Stencils(dh, dh, 31), 31, 5, 4, M.MFD_OP_LAP_POW, 2)
        ec = M.Weights(M.Stencils(de, dh, 12), 12, 3, 2, M.MFD_OP_GRAD)
        ev = M.Weights(M.Stencils(de, de, 31), 31, 5, 4, M.MFD_OP_LAP_POW, 2)
        sim = M.Sim(ctx, 2, 0, dt, eps0, mu0, -1e-3, hc, hv, ec, ev)
        rng = np.random.default_rng(1)
        sim.set_field(M.MFD_EZ, rng.standard_normal(e.n))
        sim.set_field(M.MFD_HX, rng.standard_normal(h.n))
        sim.set_field(M.MFD_HY, rng.standard_normal(h.n))
        sims.append(sim)
    sims[0].step(131)          # one direct step, 4 graph replays, 2 direct
    for _ in range(131):
        sims[1].step(1)
    assert sims[0].steps == sims[1].steps == 131
    for c in (M.MFD_EZ, M.MFD_HX, M.MFD_HY):
        assert np.array_equal(sims[0].get_field(c), sims[1].get_field(c))


@pytest.mark.parametrize("layout", ["colloc", "stag"])
def test_fp32_within_1e5_at_every_100th_step(ctx, layout):
    """FP32 with compensated curl sums against the FP64 oracle over 1000 steps:
    the relative L2 error of all fields stays <= 1e-5 at every 100th step and
    at the end, and so does the probe series over the whole run (the largest
    error seen is in the assertion message)."""
    S = 0.5
    dt, eps0, mu0, c0, eta0 = W.units(S)
    if layout == "colloc":
        c = 4e-3
        nodes = W.pec_box((33, 33), 0.25, 31)
        er = W.eps_r_uniform(nodes.n, 32)
        sim = _gpu_colloc(ctx, nodes, 12, 3, 2, 2, dt, eps0, mu0, -c, 0, True)
        assert sim.index_stats() == {"h": (0, 0, 0), "e": (0, 0, 0)}  # collocated 2D: 32-bit indices
        sim.set_materials(er, nodes.pec)
        ez, hx, hy = W.tm11_fields(nodes.xyz, 32.0, c0, mu0, 0.0, -0.5 * dt)
        ez[nodes.pec == 1] = 0
        src = W.ricker_sources(nodes, 3, 33, c0)
        probes = W.interior_nodes(nodes, 16, 34)
        prob, _ = O.tmz_collocated(nodes, 12, 3, 2, 2, dt, eps0, mu0, -c, eps_r=er)
    else:
        c, alpha, nx, n, nhv = 4e-5, 3, 36, 30, 57
        e = W.periodic_box((nx, nx), 0.25, 35, seed_line_y=nx // 2)
        h = W.periodic_box((nx, nx), 0.25, 36, offset=(0.5, 0.5))
        de, dh = M.Nodes(ctx, e.xyz, e.period), M.Nodes(ctx, h.xyz, h.period)
        hc = M.Weights(M.Stencils(dh, de, n), n, 5, 4, M.MFD_OP_GRAD)
        hv = M.Weights(M.Stencils(dh, dh, nhv), nhv, 7, 6, M.MFD_OP_LAP_POW, alpha)
        ec = M.Weights(M.Stencils(de, dh, n), n, 5, 4, M.MFD_OP_GRAD)
        ev = M.Weights(M.Stencils(de, de, nhv), nhv, 7, 6, M.MFD_OP_LAP_POW, alpha)
        sim = M.Sim(ctx, 2, 0, dt, eps0, mu0, c, hc, hv, ec, ev, compensated=True)
        ez, _, _ = W.gaussian_pulse(e.xyz, nx, nx / 2, 6.0, c0, eta0, dt, 12.0)
        _, hx, hy = W.gaussian_pulse(h.xyz, nx, nx / 2, 6.0, c0, eta0, dt, 12.0)
        src = None
        probes = W.interior_nodes(e, 8, 37)
        prob = O.tmz_staggered(e, h, n, 5, 4, alpha, dt, eps0, mu0, c)
    for comp_, v in ((M.MFD_EZ, ez), (M.MFD_HX, hx), (M.MFD_HY, hy)):
        sim.set_field(comp_, v)
    if src is not None:
        sim.set_sources(src.node, src.amp, src.f0, src.t0)
    sim.set_probes(probes, 1000)
    ref = [ez, hx, hy]
    rprobes, worst = [], 0.0
    for k in range(10):
        sim.step(100)
        out = O.run_tmz(prob, *ref, 100, step0=100 * k, sources=src, probes=probes)
        ref = list(out[:3])
        rprobes.append(out[3])
        got = [sim.get_field(cc) for cc in (M.MFD_EZ, M.MFD_HX, M.MFD_HY)]
        err = _rel_all(got, ref)
        worst = max(worst, err)
        assert err <= 1e-5, (layout, 100 * (k + 1), err)
    perr = _rel(sim.read_probes(), np.concatenate(rprobes))
    assert perr <= 1e-5, (layout, perr, worst)


@pytest.mark.parametrize("prec,comp,tol", [(1, False, 1e-10), (0, True, 1e-5)])
def test_staggered_q16_indices_with_two_windows_and_wide_slices(ctx, prec, comp, tol):
    """400 x 400 nodes per set: the Morton seams and the periodic wraps give
    slices whose neighbours need two 16-bit index windows and slices that keep
    32-bit indices. Every field after 20 steps against the oracle, and the
    32-bit index format gives bit-identical fields."""
    S, c, alpha, nx, n, nhv = 0.5, 4e-5, 3, 400, 30, 57
    dt, eps0, mu0, c0, eta0 = W.units(S)
    e = W.periodic_box((nx, nx), 0.25, 35)
    h = W.periodic_box((nx, nx), 0.25, 36, offset=(0.5, 0.5))
    de, dh = M.Nodes(ctx, e.xyz, e.period), M.Nodes(ctx, h.xyz, h.period)
    hc = M.Weights(M.Stencils(dh, de, n), n, 5, 4, M.MFD_OP_GRAD)
    hv = M.Weights(M.Stencils(dh, dh, nhv), nhv, 7, 6, M.MFD_OP_LAP_POW, alpha)
    ec = M.Weights(M.Stencils(de, dh, n), n, 5, 4, M.MFD_OP_GRAD)
    ev = M.Weights(M.Stencils(de, de, nhv), nhv, 7, 6, M.MFD_OP_LAP_POW, alpha)
    sim = M.Sim(ctx, 2, prec, dt, eps0, mu0, c, hc, hv, ec, ev, compensated=comp)
    with pytest.raises(M.MfdError) as ei:
        sim.set_index_format(7)
    assert ei.value.status == M.MFD_ERR_ARG
    stats = sim.index_stats()
    for p in ("h", "e"):
        assert stats[p][0] == nx * nx // 32
        assert stats[p][1] > 0 and stats[p][2] > 0, stats  # some slices keep 32-bit indices
        assert stats[p][1] < stats[p][0] // 100 and stats[p][2] < stats[p][0] // 100, stats
    rng = np.random.default_rng(37)
    f = [rng.standard_normal(nx * nx) for _ in range(3)]
    if prec == 0:
        f = [a.astype(np.float32).astype(np.float64) for a in f]
    comps = (M.MFD_EZ, M.MFD_HX, M.MFD_HY)
    runs = []
    for fmt in (M.MFD_INDEX_Q16, M.MFD_INDEX_I32):
        sim.set_index_format(fmt)
        for cc, v in zip(comps, f):
            sim.set_field(cc, v)
        sim.step(20)
        runs.append([sim.get_field(cc) for cc in comps])
    for a, b in zip(*runs):
        assert np.array_equal(a, b)
    prob = O.tmz_staggered(e, h, n, 5, 4, alpha, dt, eps0, mu0, c)
    re, rx, ry, _, _ = O.run_tmz(prob, *f, 20)
    assert _rel_all(runs[0], [re, rx, ry]) <= tol


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("prec,tol", [(1, 1e-10), (0, 1e-5)])
def test_collocated_with_separate_stencil_objects(ctx, dim, prec, tol):
    """Collocated curl and HV weights built on two stencils objects (the kernels
    then read two index streams, one thread per node): the same stencils as the
    shared row the oracle builds, so the same fields within the tolerance."""
    import math as _m
    S, c = 0.5, (4e-3 if dim == 2 else 1e-3)
    dt, eps0, mu0, c0, eta0 = W.units(S)
    if dim == 2:
        nodes = W.pec_box((23, 19), 0.25, 51)
        n, k, m, alpha, steps = 12, 3, 2, 2, 60
    else:
        nodes = W.periodic_box((10, 10, 10), 0.25, 52)
        n, k, m, alpha, steps = 40, 3, 3, 2, 20
    nhv = 2 * _m.comb(2 * alpha + dim, dim) + 1
    nd = M.Nodes(ctx, nodes.xyz, nodes.period)
    curl = M.Weights(M.Stencils(nd, nd, n), n, k, m, M.MFD_OP_GRAD)
    hv = M.Weights(M.Stencils(nd, nd, nhv), nhv, 2 * alpha + 1, 2 * alpha, M.MFD_OP_LAP_POW, alpha)
    sim = M.Sim(ctx, dim, prec, dt, eps0, mu0, -c, curl, hv, compensated=prec == 0)
    rng = np.random.default_rng(53)
    f = [rng.standard_normal(nodes.n) for _ in range(3 if dim == 2 else 6)]
    if dim == 2:
        sim.set_materials(None, nodes.pec)
        f[0][nodes.pec == 1] = 0
        comps = (M.MFD_EZ, M.MFD_HX, M.MFD_HY)
    else:
        comps = tuple(range(6))
    if prec == 0:
        f = [a.astype(np.float32).astype(np.float64) for a in f]
    for cc, v in zip(comps, f):
        sim.set_field(cc, v)
    sim.step(steps)
    got = [sim.get_field(cc) for cc in comps]
    if dim == 2:
        prob, _ = O.tmz_collocated(nodes, n, k, m, alpha, dt, eps0, mu0, -c)
        ref = list(O.run_tmz(prob, *f, steps)[:3])
    else:
        prob, _ = O.max3d_collocated(nodes, n, k, m, alpha, dt, eps0, mu0, -c)
        prob.wall[:] = 0
        RE, RH, _, _ = O.run_3d(prob, np.array(f[:3]), np.array(f[3:]), steps)
        ref = list(RE) + list(RH)
    assert _rel_all(got, ref) <= tol
