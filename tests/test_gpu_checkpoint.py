"""Checkpoint / resume through the C ABI: a run split by mfd_*_save_state and
mfd_*_load_state into a second object built the same way equals the unbroken
run bit for bit (fields and the whole probe series), for the collocated,
staggered and 3D layouts, FP32 and FP64, and for the batch. A blob that does
not fit the receiving object is refused with MFD_ERR_ARG and changes nothing.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_2508_18205_gb300")

S = 0.5


def _colloc(ctx, prec, seed=1):
    dt, eps0, mu0, c0, eta0 = W.units(S)
    ns = W.pec_box((28, 28), 0.25, seed)
    nd = M.Nodes(ctx, ns.xyz, ns.period)
    st = M.Stencils(nd, nd, 31)
    cw = M.Weights(st, 12, 3, 2, M.MFD_OP_GRAD)
    hw = M.Weights(st, 31, 5, 4, M.MFD_OP_LAP_POW, 2)
    src = W.ricker_sources(ns, 3, 11, c0)
    probes = W.interior_nodes(ns, 5, 12)
    ez, hx, hy = W.tm11_fields(ns.xyz, 27.0, c0, mu0, 0.0, -0.5 * dt)
    ez[ns.pec == 1] = 0

    def make():
        sim = M.Sim(ctx, 2, prec, dt, eps0, mu0, -4e-3, cw, hw, compensated=prec == M.MFD_FP32)
        sim.set_materials(W.eps_r_uniform(ns.n, 13), ns.pec)
        sim.set_sources(src.node, src.amp, src.f0, src.t0)
        return sim

    def init(sim):
        for comp, f in ((M.MFD_EZ, ez), (M.MFD_HX, hx), (M.MFD_HY, hy)):
            sim.set_field(comp, f)
        sim.set_probes(probes, 400)

    return make, init, (M.MFD_EZ, M.MFD_HX, M.MFD_HY), (nd, st, cw, hw)


def _stag(ctx, prec):
    dt, eps0, mu0, c0, eta0 = W.units(S)
    e = W.periodic_box((40, 40), 0.25, 21, seed_line_y=20)
    h = W.periodic_box((40, 40), 0.25, 22, offset=(0.5, 0.5))
    de, dh = M.Nodes(ctx, e.xyz, e.period), M.Nodes(ctx, h.xyz, h.period)
    hc = M.Weights(M.Stencils(dh, de, 30), 30, 5, 4, M.MFD_OP_GRAD)
    hv = M.Weights(M.Stencils(dh, dh, 57), 57, 7, 6, M.MFD_OP_LAP_POW, 3)
    ec = M.Weights(M.Stencils(de, dh, 30), 30, 5, 4, M.MFD_OP_GRAD)
    ev = M.Weights(M.Stencils(de, de, 57), 57, 7, 6, M.MFD_OP_LAP_POW, 3)
    ez, _, _ = W.gaussian_pulse(e.xyz, 40, 20, 6.0, c0, eta0, dt, 12.0)
    _, hx, hy = W.gaussian_pulse(h.xyz, 40, 20, 6.0, c0, eta0, dt, 12.0)
    probes = W.interior_nodes(e, 4, 23)

    def make():
        return M.Sim(ctx, 2, prec, dt, eps0, mu0, 4e-5, hc, hv, ec, ev, compensated=prec == M.MFD_FP32)

    def init(sim):
        for comp, f in ((M.MFD_EZ, ez), (M.MFD_HX, hx), (M.MFD_HY, hy)):
            sim.set_field(comp, f)
        sim.set_probes(probes, 400)

    return make, init, (M.MFD_EZ, M.MFD_HX, M.MFD_HY), (de, dh, hc, hv, ec, ev)


def _cube(ctx, prec):
    dt, eps0, mu0, c0, eta0 = W.units(S)
    ns = W.periodic_box((12, 12, 12), 0.25, 31)
    nd = M.Nodes(ctx, ns.xyz, ns.period)
    st = M.Stencils(nd, nd, 71)
    cw = M.Weights(st, 40, 3, 3, M.MFD_OP_GRAD)
    hw = M.Weights(st, 71, 5, 4, M.MFD_OP_LAP_POW, 2)
    (ex, ey, ez), (hx, hy, hz) = W.tm110_fields_3d(ns.xyz, 6.0, c0, mu0, 0.0, -0.5 * dt)
    probes = W.interior_nodes(ns, 3, 32)

    def make():
        sim = M.Sim(ctx, 3, prec, dt, eps0, mu0, -1e-3, cw, hw, compensated=prec == M.MFD_FP32)
        sim.set_materials(W.eps_r_uniform(ns.n, 33, 1.0, 3.0), None)
        return sim

    def init(sim):
        for comp, f in enumerate((ex, ey, ez, hx, hy, hz)):
            sim.set_field(comp, f)
        sim.set_probes(probes, 400)

    return make, init, tuple(range(6)), (nd, st, cw, hw)


@pytest.mark.parametrize("kind,prec", [("colloc", M.MFD_FP32), ("colloc", M.MFD_FP64), ("stag", M.MFD_FP32),
                                       ("stag", M.MFD_FP64), ("cube", M.MFD_FP32)])
def test_split_run_equals_unbroken_run(kind, prec):
    ctx = M.Ctx(0)
    make, init, comps, keep = {"colloc": _colloc, "stag": _stag, "cube": _cube}[kind](ctx, prec)
    first, second = 77, 100  # odd: the checkpoint sits on the second ping-pong buffer
    a = make()
    init(a)
    a.step(first)
    blob = a.save_state()
    a.step(second)
    ref = [a.get_field(c) for c in comps]
    ref_p = a.read_probes()
    assert ref_p.shape[0] == first + second
    b = make()
    init(b)  # same probes; fields and step index come from the blob
    b.step(5)  # whatever b did before is replaced
    b.load_state(blob)
    assert b.steps == first
    b.step(second)
    assert b.steps == first + second
    for c, r in zip(comps, ref):
        assert np.array_equal(b.get_field(c), r), c
    assert np.array_equal(b.read_probes(), ref_p)


def test_mismatched_blobs_are_refused():
    ctx = M.Ctx(0)
    make_c, init_c, _, keep_c = _colloc(ctx, M.MFD_FP32)
    make_s, init_s, _, keep_s = _stag(ctx, M.MFD_FP32)
    a = make_c()
    init_c(a)
    a.step(10)
    blob = a.save_state()
    s = make_s()
    init_s(s)
    s.step(3)
    before = s.get_field(M.MFD_EZ)

    def status(b):
        try:
            s.load_state(b)
        except M.MfdError as e:
            return e.status
        return M.MFD_OK

    assert status(blob) == M.MFD_ERR_ARG  # another layout
    assert status(blob[:40]) == M.MFD_ERR_ARG  # truncated header
    assert status(b"x" * len(blob)) == M.MFD_ERR_ARG  # not a state
    own = s.save_state()
    assert status(own[:-8]) == M.MFD_ERR_ARG  # truncated body
    a64 = _colloc(ctx, M.MFD_FP64)[0]()
    try:
        a64.load_state(blob)
        raise AssertionError("an FP32 state loaded into an FP64 simulation")
    except M.MfdError as e:
        assert e.status == M.MFD_ERR_ARG
    assert s.steps == 3 and np.array_equal(s.get_field(M.MFD_EZ), before)


@pytest.mark.parametrize("variant", [0, 2])
def test_batch_split_run_equals_unbroken_run(variant):
    """A batch run split by save and load equals the unbroken run bit for bit;
    with variant 2 the state blob holds no H*, which the first step after the
    load recomputes with the same sums the E pass made it with."""
    ctx = M.Ctx(0)
    dt, eps0, mu0, c0, eta0 = W.units(S)
    R = 8
    specs = [(W.pec_box((24, 24), 0.25, 41), 12), (W.disk(12.0, 0.25, 42), 30)]
    doms, keep = [], []
    for ns, n in specs:
        nd = M.Nodes(ctx, ns.xyz, ns.period)
        st = M.Stencils(nd, nd, max(n, 31))
        cw = M.Weights(st, n, 3, W.poly_degree_for(n), M.MFD_OP_GRAD)
        hw = M.Weights(st, 31, 5, 4, M.MFD_OP_LAP_POW, 2)
        doms.append((cw, hw, dt, eps0, mu0, -4e-3))
        keep.append((nd, st))

    def make():
        bt = M.Batch(ctx, doms, nrhs=R)
        bt.set_variant(variant)
        for d, (ns, n) in enumerate(specs):
            bt.set_materials(d, W.eps_r_uniform(ns.n, 50 + d), ns.pec)
            src = W.ricker_sources(ns, R, 60 + d, c0, nrhs=R, one_per_rhs=True)
            bt.set_sources(d, src.node, src.rhs, src.amp, src.f0, src.t0)
            bt.set_probes(d, W.interior_nodes(ns, 3, 70 + d), 300)
        return bt

    a = make()
    a.step(50)
    blob = a.save_state()
    a.step(70)
    ref = [a.get_field(d, c) for d in range(2) for c in (M.MFD_EZ, M.MFD_HX, M.MFD_HY)]
    ref_p = [a.read_probes(d) for d in range(2)]
    b = make()
    b.step(9)
    b.load_state(blob)
    b.step(70)
    got = [b.get_field(d, c) for d in range(2) for c in (M.MFD_EZ, M.MFD_HX, M.MFD_HY)]
    for x, y in zip(got, ref):
        assert np.array_equal(x, y)
    for d in range(2):
        assert ref_p[d].shape[0] == 120
        assert np.array_equal(b.read_probes(d), ref_p[d])
