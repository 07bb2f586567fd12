"""Edge cases of the path against the oracle, through the C ABI.

* an empty node set is refused (MFD_ERR_ARG) before any work;
* the smallest useful sets: every node in every stencil (N = n = 16, 2D) and a
  3D set of exactly 71 nodes, stepped against the oracle (FP64 1e-10);
* one node past a slice of 32 (N = 33) and a single partial slice (N = 20):
  the padded lanes of the sliced streams neither read nor write outside;
* the largest stencil the kNN takes (128 entries, 3D, degree-3 monomials:
  local systems of 148 unknowns): kNN bit-exact, weights within 1e-8;
* zero steps leave fields and the step index alone; a second set of sources
  and probes replaces the first.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_2508_18205_gb300")


def _status(fn, *args):
    try:
        fn(*args)
    except M.MfdError as e:
        return e.status
    return M.MFD_OK


def test_empty_node_set_is_refused():
    ctx = M.Ctx(0)
    assert _status(M.Nodes, ctx, np.zeros((0, 2)), None) == M.MFD_ERR_ARG
    assert _status(M.Nodes, ctx, np.zeros((0, 3)), np.zeros(3)) == M.MFD_ERR_ARG


def _run_2d(nodes, n, nh, m_hv, steps, prec=M.MFD_FP64):
    ctx = M.Ctx(0)
    dt, eps0, mu0, c0, eta0 = W.units(0.3)
    nd = M.Nodes(ctx, nodes.xyz, nodes.period)
    st = M.Stencils(nd, nd, max(n, nh))
    cw = M.Weights(st, n, 3, 2, M.MFD_OP_GRAD)
    hw = M.Weights(st, nh, 5, m_hv, M.MFD_OP_LAP_POW, 2)
    sim = M.Sim(ctx, 2, prec, dt, eps0, mu0, -2e-3, cw, hw)
    rng = np.random.default_rng(nodes.n)
    f = rng.standard_normal((3, nodes.n))
    for comp, v in zip((M.MFD_EZ, M.MFD_HX, M.MFD_HY), f):
        sim.set_field(comp, v)
    sim.step(steps)
    got = np.concatenate([sim.get_field(c) for c in (M.MFD_EZ, M.MFD_HX, M.MFD_HY)])
    idx = O.knn(nodes.xyz, nodes.xyz, nodes.period, max(n, nh))
    c = O.Stencil(idx=np.ascontiguousarray(idx[:, :n]),
                  w=O.weights(nodes.xyz, nodes.xyz, nodes.period, idx, n, 3, 2, O.OP_GRAD))
    v = O.Stencil(idx=np.ascontiguousarray(idx[:, :nh]),
                  w=O.weights(nodes.xyz, nodes.xyz, nodes.period, idx, nh, 5, m_hv, O.OP_LAP_POW, 2))
    prob = O.TMz(nh=nodes.n, ne=nodes.n, hc=c, hv=v, ec=c, ev=v, eps_r=np.ones(nodes.n),
                 pec=np.zeros(nodes.n, np.uint8), dt=dt, eps0=eps0, mu0=mu0, gamma=-2e-3)
    ref = np.concatenate(O.run_tmz(prob, *f, steps)[:3])
    return got, ref


# (4, 4): every node in every stencil (N = n = N_h = 16; HV with degree-2
# monomials, as 16 nodes cannot carry the 15 of degree 4 and an RBF part);
# (11, 3): one node past a slice of 32; (5, 4): one partial slice
@pytest.mark.parametrize("shape,n,nh,m_hv,steps", [((4, 4), 16, 16, 2, 20), ((11, 3), 12, 31, 4, 40),
                                                    ((5, 4), 12, 20, 2, 40)])
def test_small_and_ragged_sets_match_the_oracle(shape, n, nh, m_hv, steps):
    nodes = W.periodic_box(shape, 0.25, 90 + shape[0])
    got, ref = _run_2d(nodes, n, nh, m_hv, steps)
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


def test_a_3d_set_of_exactly_one_hv_stencil():
    ctx = M.Ctx(0)
    dt, eps0, mu0, c0, eta0 = W.units(0.3)
    # 71 nodes: a 4 x 5 x 4 periodic lattice less nine nodes
    full = W.periodic_box((4, 5, 4), 0.25, 95)
    keep = np.arange(full.n) >= 9
    nodes = W.NodeSet(xyz=full.xyz[keep], pec=full.pec[keep], period=full.period, box_lo=full.box_lo,
                      box_hi=full.box_hi, normal_axes=full.normal_axes[keep])
    assert nodes.n == 71
    nd = M.Nodes(ctx, nodes.xyz, nodes.period)
    st = M.Stencils(nd, nd, 71)
    cw = M.Weights(st, 40, 3, 3, M.MFD_OP_GRAD)
    hw = M.Weights(st, 71, 5, 4, M.MFD_OP_LAP_POW, 2)
    sim = M.Sim(ctx, 3, M.MFD_FP64, dt, eps0, mu0, -1e-3, cw, hw)
    rng = np.random.default_rng(96)
    E0, H0 = rng.standard_normal((3, 71)), rng.standard_normal((3, 71))
    for b in range(3):
        sim.set_field(b, E0[b])
        sim.set_field(3 + b, H0[b])
    sim.step(20)
    got = np.concatenate([sim.get_field(b) for b in range(6)])
    prob, _ = O.max3d_collocated(nodes, 40, 3, 3, 2, dt, eps0, mu0, -1e-3)
    E1, H1, _, _ = O.run_3d(prob, E0, H0, 20)
    ref = np.concatenate([E1.ravel(), H1.ravel()])
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


def test_the_largest_stencil():
    ctx = M.Ctx(0)
    box = W.periodic_box((9, 8, 7), 0.25, 97)
    nd = M.Nodes(ctx, box.xyz, box.period)
    st = M.Stencils(nd, nd, 128)
    ids = O.knn(box.xyz, box.xyz, box.period, 128)
    assert np.array_equal(st.read(), ids)
    gw = M.Weights(st, 128, 3, 3, M.MFD_OP_GRAD).read()
    rw = O.weights(box.xyz, box.xyz, box.period, ids, 128, 3, 3, O.OP_GRAD)
    scale = np.max(np.abs(rw), axis=2, keepdims=True)
    assert np.max(np.abs(gw - rw) / scale) <= 1e-8
    assert _status(M.Stencils, nd, nd, 129) == M.MFD_ERR_ARG


def test_zero_steps_and_replaced_sources_and_probes():
    ctx = M.Ctx(0)
    dt, eps0, mu0, c0, eta0 = W.units(0.5)
    sq = W.pec_box((18, 18), 0.25, 98)
    nd = M.Nodes(ctx, sq.xyz, sq.period)
    st = M.Stencils(nd, nd, 31)
    cw = M.Weights(st, 12, 3, 2, M.MFD_OP_GRAD)
    hw = M.Weights(st, 31, 5, 4, M.MFD_OP_LAP_POW, 2)
    sim = M.Sim(ctx, 2, M.MFD_FP64, dt, eps0, mu0, -4e-3, cw, hw)
    sim.set_materials(None, sq.pec)
    rng = np.random.default_rng(99)
    ez = rng.standard_normal(sq.n)
    ez[sq.pec == 1] = 0
    sim.set_field(M.MFD_EZ, ez)
    sim.step(0)
    assert sim.steps == 0 and np.array_equal(sim.get_field(M.MFD_EZ), ez)
    first = W.ricker_sources(sq, 3, 100, c0)
    second = W.ricker_sources(sq, 2, 101, c0)
    sim.set_sources(first.node, first.amp, first.f0, first.t0)
    sim.set_probes(W.interior_nodes(sq, 3, 102), 5)
    sim.set_sources(second.node, second.amp, second.f0, second.t0)
    probes = W.interior_nodes(sq, 4, 103)
    sim.set_probes(probes, 30)
    sim.step(30)
    prob, _ = O.tmz_collocated(sq, 12, 3, 2, 2, dt, eps0, mu0, -4e-3)
    order = np.argsort(second.node)
    srt = W.Sources(node=second.node[order], rhs=second.rhs[order], amp=second.amp[order], f0=second.f0[order],
                    t0=second.t0[order])
    e1, x1, y1, pr, _ = O.run_tmz(prob, ez, np.zeros(sq.n), np.zeros(sq.n), 30, sources=srt, probes=probes)
    got = sim.get_field(M.MFD_EZ)
    assert np.linalg.norm(got - e1) <= 1e-10 * np.linalg.norm(e1)
    gp = sim.read_probes().reshape(pr.shape)
    assert np.linalg.norm(gp - pr) <= 1e-10 * np.linalg.norm(pr)
