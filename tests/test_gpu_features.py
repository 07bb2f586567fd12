"""GPU features around the step: the block-size autotuner, the energy watchdog,
RBF-VFD curl weights in the step, and the FP64 FMA peak probe.

* autotune restores the fields (the simulation does not advance) and any block
  size gives bit-identical fields (one thread per node, same arithmetic);
* the watchdog returns MFD_ERR_UNSTABLE for the unstabilised scheme on
  scattered nodes (App. A) and stays silent with hyperviscosity;
* a collocated step with RBF-VFD (delta = h/2) curl weights matches the oracle
  (FP64 1e-10).
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_2508_18205_gb300")


def _colloc(ctx, nodes, gamma, prec=1, vfd=None, S=0.5):
    dt, eps0, mu0, c0, eta0 = W.units(S)
    nd = M.Nodes(ctx, nodes.xyz, nodes.period)
    st = M.Stencils(nd, nd, 31)
    if vfd is None:
        cw = M.Weights(st, 12, 3, 2, M.MFD_OP_GRAD)
    else:
        cw = M.Weights(st, 12, 3, 2, M.MFD_OP_GRAD_VFD, 0, vfd)
    hw = M.Weights(st, 31, 5, 4, M.MFD_OP_LAP_POW, 2)
    return M.Sim(ctx, 2, prec, dt, eps0, mu0, gamma, cw, hw)


def test_autotune_keeps_state_and_blocks_do_not_change_results():
    ctx = M.Ctx(0)
    dt, eps0, mu0, c0, eta0 = W.units(0.5)
    e = W.periodic_box((40, 40), 0.25, 1)
    h = W.periodic_box((40, 40), 0.25, 2, offset=(0.5, 0.5))
    de, dh = M.Nodes(ctx, e.xyz, e.period), M.Nodes(ctx, h.xyz, h.period)
    hc = M.Weights(M.Stencils(dh, de, 30), 30, 5, 4, M.MFD_OP_GRAD)
    hv = M.Weights(M.Stencils(dh, dh, 57), 57, 7, 6, M.MFD_OP_LAP_POW, 3)
    ec = M.Weights(M.Stencils(de, dh, 30), 30, 5, 4, M.MFD_OP_GRAD)
    ev = M.Weights(M.Stencils(de, de, 57), 57, 7, 6, M.MFD_OP_LAP_POW, 3)
    rng = np.random.default_rng(3)
    f = [rng.standard_normal(e.n), rng.standard_normal(h.n), rng.standard_normal(h.n)]
    outs = []
    for blocks in ("tune", (128, 512), (512, 64)):
        sim = M.Sim(ctx, 2, 0, dt, eps0, mu0, 4e-5, hc, hv, ec, ev, compensated=True)
        for c, v in zip((M.MFD_EZ, M.MFD_HX, M.MFD_HY), f):
            sim.set_field(c, v)
        if blocks == "tune":
            ch = sim.autotune(5)
            assert all(b in (64, 128, 256, 512) for b in ch)
            assert sim.steps == 0
            assert np.array_equal(sim.get_field(M.MFD_EZ), f[0].astype(np.float32).astype(np.float64))
        else:
            sim.set_blocks(*blocks)
        sim.step(70)
        outs.append([sim.get_field(c) for c in (M.MFD_EZ, M.MFD_HX, M.MFD_HY)])
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert np.array_equal(a, b)


def test_watchdog_flags_the_unstabilised_scheme():
    ctx = M.Ctx(0)
    S = 1.0 / (10.0 * np.sqrt(2.0))
    dt, eps0, mu0, c0, eta0 = W.units(S)
    nodes = W.periodic_box((30, 30), 0.25, 4)
    ez, hx, hy = W.gaussian_pulse(nodes.xyz, 30, 15, 4.0, c0, eta0, dt)
    for gamma, expect_unstable in ((0.0, True), (-3e-3, False)):
        sim = _colloc(ctx, nodes, gamma, prec=1, S=S)
        sim.set_field(M.MFD_EZ, ez)
        sim.set_field(M.MFD_HX, hx)
        sim.set_field(M.MFD_HY, hy)
        sim.set_watchdog(100, 1.5)
        if expect_unstable:
            with pytest.raises(M.MfdError) as ex:
                sim.step(6000)
            assert ex.value.status == M.MFD_ERR_UNSTABLE
            assert 0 < sim.steps < 6000
        else:
            sim.step(3000)
            assert sim.steps == 3000


def test_vfd_curl_weights_step_matches_oracle():
    ctx = M.Ctx(0)
    dt, eps0, mu0, c0, eta0 = W.units(0.5)
    nodes = W.pec_box((31, 27), 0.25, 6)
    sim = _colloc(ctx, nodes, -4e-3, prec=1, vfd=0.5)
    sim.set_materials(None, nodes.pec)
    ez, hx, hy = W.tm11_fields(nodes.xyz, 30.0, c0, mu0, 0.0, -0.5 * dt)
    ez[nodes.pec == 1] = 0
    sim.set_field(M.MFD_EZ, ez)
    sim.set_field(M.MFD_HX, hx)
    sim.set_field(M.MFD_HY, hy)
    sim.step(100)
    prob, _ = O.tmz_collocated(nodes, 12, 3, 2, 2, dt, eps0, mu0, -4e-3, vfd_delta=0.5)
    re, rx, ry, _, _ = O.run_tmz(prob, ez, hx, hy, 100)
    got = np.concatenate([sim.get_field(c) for c in (M.MFD_EZ, M.MFD_HX, M.MFD_HY)])
    ref = np.concatenate([re, rx, ry])
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


def test_fma_peak_probe_is_sane():
    g64, g32 = M.fma_peak(0)
    assert 100.0 < g64 < 1e5 and 1e3 < g32 < 1e6 and g32 > g64


def test_handles_may_be_destroyed_in_any_order():
    """Objects are reference counted: dropping the context, node set, stencils and
    weights handles before the simulation leaves the simulation usable."""
    ctx = M.Ctx(0)
    dt, eps0, mu0, c0, eta0 = W.units(0.5)
    nodes = W.pec_box((20, 20), 0.25, 8)
    nd = M.Nodes(ctx, nodes.xyz, nodes.period)
    st = M.Stencils(nd, nd, 31)
    cw = M.Weights(st, 12, 3, 2, M.MFD_OP_GRAD)
    hw = M.Weights(st, 31, 5, 4, M.MFD_OP_LAP_POW, 2)
    sim = M.Sim(ctx, 2, 1, dt, eps0, mu0, -4e-3, cw, hw)
    L = M.lib()
    for obj, fn in ((ctx, L.mfd_ctx_destroy), (nd, L.mfd_nodes_destroy), (st, L.mfd_stencils_destroy),
                    (cw, L.mfd_weights_destroy), (hw, L.mfd_weights_destroy)):
        fn(obj.h)
        obj.h = None
    ez, hx, hy = W.tm11_fields(nodes.xyz, 19.0, c0, mu0, 0.0, -0.5 * dt)
    sim.set_field(M.MFD_EZ, ez)
    sim.set_field(M.MFD_HX, hx)
    sim.set_field(M.MFD_HY, hy)
    sim.step(40)
    assert np.all(np.isfinite(sim.get_field(M.MFD_EZ)))
    L.mfd_sim_destroy(sim.h)
    sim.h = None


def test_zero_copy_field_io_matches_host_path():
    """mfd_set_field_device / mfd_get_field_device (torch CUDA tensors on the
    current stream) give the same state and results as the host path, for a
    simulation and a batch."""
    torch = pytest.importorskip("torch")
    ctx = M.Ctx(0)
    dt, eps0, mu0, c0, eta0 = W.units(0.5)
    nodes = W.pec_box((30, 26), 0.25, 71)
    nd = M.Nodes(ctx, nodes.xyz, nodes.period)
    st = M.Stencils(nd, nd, 31)
    cw = M.Weights(st, 12, 3, 2, M.MFD_OP_GRAD)
    hw = M.Weights(st, 31, 5, 4, M.MFD_OP_LAP_POW, 2)
    rng = np.random.default_rng(2)
    f = {c: rng.standard_normal(nodes.n) for c in (M.MFD_EZ, M.MFD_HX, M.MFD_HY)}
    out = []
    for device in (False, True):
        sim = M.Sim(ctx, 2, M.MFD_FP32, dt, eps0, mu0, -4e-3, cw, hw, compensated=True)
        sim.set_materials(None, nodes.pec)
        for c, v in f.items():
            sim.set_field(c, torch.tensor(v, device="cuda") if device else v)
        sim.step(50)
        if device:
            res = [sim.get_field(c, out=torch.empty(nodes.n, dtype=torch.float64, device="cuda")) for c in f]
            torch.cuda.synchronize()
            out.append(np.concatenate([r.cpu().numpy() for r in res]))
        else:
            out.append(np.concatenate([sim.get_field(c) for c in f]))
    assert np.array_equal(out[0], out[1])
    bt = M.Batch(ctx, [(cw, hw, dt, eps0, mu0, -4e-3)], nrhs=4)
    v = rng.standard_normal((nodes.n, 4))
    bt.set_field(0, M.MFD_EZ, torch.tensor(v, device="cuda"))
    back = bt.get_field(0, M.MFD_EZ, out=torch.empty((nodes.n, 4), dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    assert np.array_equal(back.cpu().numpy(), v.astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("prec,tol", [(M.MFD_FP64, 1e-10), (M.MFD_FP32, 1e-5)])
def test_lanes_per_node_match_the_oracle(prec, tol):
    """1, 2 or 4 threads per node (each summing a share of the stencil chunks)
    give the oracle's fields on a collocated PEC cavity with sources and probes;
    the autotuner's choice is one of them and leaves the state."""
    ctx = M.Ctx(0)
    S, c = 0.5, 4e-3
    dt, eps0, mu0, c0, eta0 = W.units(S)
    nodes = W.pec_box((160, 160), 0.25, 21)
    nd = M.Nodes(ctx, nodes.xyz, nodes.period)
    st = M.Stencils(nd, nd, 31)
    cw = M.Weights(st, 20, 3, 2, M.MFD_OP_GRAD)
    hw = M.Weights(st, 31, 5, 4, M.MFD_OP_LAP_POW, 2)
    eps = W.eps_r_uniform(nodes.n, 22)
    src = W.ricker_sources(nodes, 4, 23, c0)
    probes = W.interior_nodes(nodes, 8, 24)
    ez, hx, hy = W.tm11_fields(nodes.xyz, 159.0, c0, mu0, 0.0, -0.5 * dt)
    ez[nodes.pec == 1] = 0
    order = np.argsort(src.node)
    srt = W.Sources(node=src.node[order], rhs=src.rhs[order], amp=src.amp[order], f0=src.f0[order], t0=src.t0[order])
    prob, _ = O.tmz_collocated(nodes, 20, 3, 2, 2, dt, eps0, mu0, -c, eps_r=eps)
    e1, x1, y1, pr, _ = O.run_tmz(prob, ez, hx, hy, 120, sources=srt, probes=probes)
    ref = np.concatenate([e1, x1, y1])
    for lanes in ((1, 1), (2, 2), (4, 2), "tune"):
        sim = M.Sim(ctx, 2, prec, dt, eps0, mu0, -c, cw, hw, compensated=prec == M.MFD_FP32)
        sim.set_materials(eps, nodes.pec)
        for comp, f in ((M.MFD_EZ, ez), (M.MFD_HX, hx), (M.MFD_HY, hy)):
            sim.set_field(comp, f)
        sim.set_sources(src.node, src.amp, src.f0, src.t0)
        sim.set_probes(probes, 120)
        if lanes == "tune":
            sim.autotune(3)
            assert sim.steps == 0
            blocks, ln = sim.launch_config()
            assert all(x in (1, 2, 4) for x in ln) and all(b in (64, 128, 256, 512) for b in blocks)
        else:
            sim.set_lanes(*lanes)
            assert sim.launch_config()[1] == lanes
        sim.step(120)
        got = np.concatenate([sim.get_field(cc) for cc in (M.MFD_EZ, M.MFD_HX, M.MFD_HY)])
        assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref), lanes
        gp = sim.read_probes()
        assert np.linalg.norm(gp - pr) <= tol * np.linalg.norm(pr), lanes


def test_probes_of_other_components_match_the_oracle():
    """Probes record Hx (collocated 2D) or Ex, Hz (3D) after each step, H at the
    half step the leapfrog holds: the oracle's state sampled after each of its
    steps (FP64, 1e-10); the staggered layout and the gradient refuse them."""
    ctx = M.Ctx(0)
    dt, eps0, mu0, c0, eta0 = W.units(0.5)
    sq = W.pec_box((20, 20), 0.25, 31)
    nd = M.Nodes(ctx, sq.xyz, sq.period)
    st = M.Stencils(nd, nd, 31)
    cw = M.Weights(st, 12, 3, 2, M.MFD_OP_GRAD)
    hw = M.Weights(st, 31, 5, 4, M.MFD_OP_LAP_POW, 2)
    src = W.ricker_sources(sq, 2, 32, c0)
    probes = W.interior_nodes(sq, 5, 33)
    sim = M.Sim(ctx, 2, M.MFD_FP64, dt, eps0, mu0, -4e-3, cw, hw)
    sim.set_materials(None, sq.pec)
    sim.set_sources(src.node, src.amp, src.f0, src.t0)
    sim.set_probes(probes, 30)
    sim.set_probe_component(M.MFD_HX)
    sim.step(30)
    got = sim.read_probes()
    prob, _ = O.tmz_collocated(sq, 12, 3, 2, 2, dt, eps0, mu0, -4e-3)
    order = np.argsort(src.node)
    srt = W.Sources(node=src.node[order], rhs=src.rhs[order], amp=src.amp[order], f0=src.f0[order], t0=src.t0[order])
    ez, hx, hy = np.zeros((3, sq.n))
    ref = []
    for n in range(30):
        ez, hx, hy, _, _ = O.run_tmz(prob, ez, hx, hy, 1, step0=n, sources=srt)
        ref.append(hx[probes])
    ref = np.array(ref)
    assert np.linalg.norm(got.reshape(ref.shape) - ref) <= 1e-10 * np.linalg.norm(ref)
    with pytest.raises(M.MfdError):  # the gradient's objective is over Ez probes
        sim.grad(10, 0, len(src.node))
    # 3D: Ex and Hz
    box = W.periodic_box((8, 8, 8), 0.25, 34)
    nd3 = M.Nodes(ctx, box.xyz, box.period)
    st3 = M.Stencils(nd3, nd3, 71)
    cw3 = M.Weights(st3, 40, 3, 3, M.MFD_OP_GRAD)
    hw3 = M.Weights(st3, 71, 5, 4, M.MFD_OP_LAP_POW, 2)
    rng = np.random.default_rng(35)
    E0, H0 = rng.standard_normal((3, box.n)), rng.standard_normal((3, box.n))
    p3 = W.interior_nodes(box, 4, 36)
    prob3, _ = O.max3d_collocated(box, 40, 3, 3, 2, dt, eps0, mu0, -1e-3)
    for comp in (M.MFD_EX, M.MFD_HZ):
        sim3 = M.Sim(ctx, 3, M.MFD_FP64, dt, eps0, mu0, -1e-3, cw3, hw3)
        for b in range(3):
            sim3.set_field(b, E0[b])
            sim3.set_field(3 + b, H0[b])
        sim3.set_probes(p3, 12)
        sim3.set_probe_component(comp)
        sim3.step(12)
        got3 = sim3.read_probes().reshape(12, len(p3))
        E, H = E0, H0
        ref3 = []
        for n in range(12):
            E, H, _, _ = O.run_3d(prob3, E, H, 1, step0=n)
            ref3.append((E[0] if comp == M.MFD_EX else H[2])[p3])
        ref3 = np.array(ref3)
        assert np.linalg.norm(got3 - ref3) <= 1e-10 * np.linalg.norm(ref3), comp
    e = W.periodic_box((12, 12), 0.25, 37)
    h = W.periodic_box((12, 12), 0.25, 38, offset=(0.5, 0.5))
    de, dh = M.Nodes(ctx, e.xyz, e.period), M.Nodes(ctx, h.xyz, h.period)
    stag = M.Sim(ctx, 2, M.MFD_FP32, dt, eps0, mu0, 4e-5,
                 M.Weights(M.Stencils(dh, de, 30), 30, 5, 4, M.MFD_OP_GRAD),
                 M.Weights(M.Stencils(dh, dh, 57), 57, 7, 6, M.MFD_OP_LAP_POW, 3),
                 M.Weights(M.Stencils(de, dh, 30), 30, 5, 4, M.MFD_OP_GRAD),
                 M.Weights(M.Stencils(de, de, 57), 57, 7, 6, M.MFD_OP_LAP_POW, 3))
    with pytest.raises(M.MfdError):
        stag.set_probe_component(M.MFD_HX)


def test_l2_keep_leaves_results_bit_identical():
    """The L2 policy of the stencil streams (mfd_sim_set_l2_keep) changes where
    lines live, not what is computed: staggered and collocated steps and a
    collocated gradient give the same bits for every kept fraction. A problem
    whose streams fit in the L2 keeps all of them by default; a fraction above 1
    is refused."""
    ctx = M.Ctx(0)
    dt, eps0, mu0, c0, eta0 = W.units(0.5)
    e = W.periodic_box((40, 40), 0.25, 1)
    h = W.periodic_box((40, 40), 0.25, 2, offset=(0.5, 0.5))
    de, dh = M.Nodes(ctx, e.xyz, e.period), M.Nodes(ctx, h.xyz, h.period)
    hc = M.Weights(M.Stencils(dh, de, 30), 30, 5, 4, M.MFD_OP_GRAD)
    hv = M.Weights(M.Stencils(dh, dh, 57), 57, 7, 6, M.MFD_OP_LAP_POW, 3)
    ec = M.Weights(M.Stencils(de, dh, 30), 30, 5, 4, M.MFD_OP_GRAD)
    ev = M.Weights(M.Stencils(de, de, 57), 57, 7, 6, M.MFD_OP_LAP_POW, 3)
    rng = np.random.default_rng(5)
    f = [rng.standard_normal(e.n), rng.standard_normal(h.n), rng.standard_normal(h.n)]
    box = W.pec_box((30, 30), 0.25, 6)
    eps = W.eps_r_uniform(box.n, 7)
    src = W.ricker_sources(box, 3, 8, c0)
    probes = W.interior_nodes(box, 4, 9)
    outs, grads = [], []
    for keep in (-1.0, 0.0, 0.4, 1.0):
        sim = M.Sim(ctx, 2, 0, dt, eps0, mu0, 4e-5, hc, hv, ec, ev, compensated=True)
        sim.set_l2_keep(keep)
        if keep < 0:
            assert sim.l2_keep == 1.0  # a 1600 + 1600 node problem: its streams fit in the L2
        else:
            assert sim.l2_keep == pytest.approx(keep)
        for c, v in zip((M.MFD_EZ, M.MFD_HX, M.MFD_HY), f):
            sim.set_field(c, v)
        sim.step(40)
        col = _colloc(ctx, box, -4e-3, prec=0)
        col.set_l2_keep(keep)
        col.set_materials(eps, box.pec)
        col.set_sources(src.node, src.amp, src.f0, src.t0)
        col.set_probes(probes, 60)
        col.step(30)
        outs.append([sim.get_field(c) for c in (M.MFD_EZ, M.MFD_HX, M.MFD_HY)] +
                    [col.get_field(c) for c in (M.MFD_EZ, M.MFD_HX, M.MFD_HY)])
        col.set_field(M.MFD_EZ, np.zeros(box.n))
        col.set_field(M.MFD_HX, np.zeros(box.n))
        col.set_field(M.MFD_HY, np.zeros(box.n))
        col.set_probes(probes, 60)
        grads.append(col.grad(60, 0, len(src.node)))
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert np.array_equal(a, b)
    for J, ge, ga in grads[1:]:
        assert J == grads[0][0] and np.array_equal(ge, grads[0][1]) and np.array_equal(ga, grads[0][2])
    with pytest.raises(M.MfdError):
        sim.set_l2_keep(1.5)
