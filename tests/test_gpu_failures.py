"""Failure detection through the C ABI, with faults made on the host or by a
bounded wait that is told to give up, never by a GPU fault.

* MFD_ERR_TIMEOUT: the batched kernel's grid barriers poll a bounded number of
  times; with the bound set to 0 a waiting block gives up at its first poll,
  every block leaves the kernel and mfd_batch_step returns the status. The
  batch then steps on normally once the bound is back (checked against the
  oracle), with its step counter unchanged by the failed call.
* MFD_ERR_SINGULAR: stencils whose weight system (Eq. 9) is exactly singular,
  a node given twice (two equal rows) and a cluster of nodes on one line
  (the y-monomials of the augmentation vanish on it).
* MFD_ERR_ARG: sizes and combinations the calls reject before any work
  (a stencil larger than its source set, n_use beyond the stencil, ...).
* MFD_ERR_OOM: an injected failure of the k-th device allocation
  (mfd_debug_fail_alloc) for every allocation a whole run makes; each call that
  meets it returns MFD_ERR_OOM, and a run after it gives the same bits as a run
  that never failed.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_2508_18205_gb300")

S, C_HV = 0.5, 4e-3


def _status(fn, *args, **kw):
    try:
        fn(*args, **kw)
    except M.MfdError as e:
        return e.status
    return M.MFD_OK


def _batch(ctx, specs, R):
    doms, keep = [], []
    dt, eps0, mu0, c0, eta0 = W.units(S)
    for ns, n in specs:
        nd = M.Nodes(ctx, ns.xyz, ns.period)
        st = M.Stencils(nd, nd, max(n, 31))
        cw = M.Weights(st, n, 3, W.poly_degree_for(n), M.MFD_OP_GRAD)
        hw = M.Weights(st, 31, 5, 4, M.MFD_OP_LAP_POW, 2)
        doms.append((cw, hw, dt, eps0, mu0, -C_HV))
        keep.append((nd, st))
    return M.Batch(ctx, doms, nrhs=R), keep


def _set_batch_state(bt, specs, R, seed):
    rng = np.random.default_rng(seed)
    init = []
    for d, (ns, n) in enumerate(specs):
        bt.set_materials(d, None, ns.pec)
        f = 0.1 * rng.standard_normal((3, ns.n, R))
        f[0][ns.pec == 1] = 0
        for c, comp in enumerate((M.MFD_EZ, M.MFD_HX, M.MFD_HY)):
            bt.set_field(d, comp, f[c])
        init.append(f)
    return init


def test_batch_barrier_timeout_returns_status_and_batch_recovers():
    ctx = M.Ctx(0)
    R = 16
    specs = [(W.pec_box((30, 30), 0.25, 31), 12), (W.disk(16.0, 0.25, 32), 20)]
    bt, keep = _batch(ctx, specs, R)
    _set_batch_state(bt, specs, R, 1)
    for d, (ns, n) in enumerate(specs):
        bt.set_probes(d, W.interior_nodes(ns, 3, 40 + d), 200)
    bt.set_spin_limit(0)
    for _ in range(2):  # graph captured with the zero bound, then replayed
        assert _status(bt.step, 60) == M.MFD_ERR_TIMEOUT
        assert bt.read_probes(0).shape[0] == 0  # the failed call advanced nothing
    bt.set_spin_limit(1 << 25)
    init = _set_batch_state(bt, specs, R, 2)
    nsteps = 60
    for d, (ns, n) in enumerate(specs):
        bt.set_probes(d, W.interior_nodes(ns, 3, 40 + d), nsteps)
    bt.step(nsteps)
    dt, eps0, mu0, c0, eta0 = W.units(S)
    for d, (ns, n) in enumerate(specs):
        assert bt.read_probes(d).shape[0] == nsteps
        prob, _ = O.tmz_collocated(ns, n, 3, W.poly_degree_for(n), 2, dt, eps0, mu0, -C_HV)
        got = bt.get_field(d, M.MFD_EZ)
        f = init[d]
        ref = np.stack([O.run_tmz(prob, f[0][:, r], f[1][:, r], f[2][:, r], nsteps)[0] for r in range(R)], 1)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= 1e-5, (d, err)


def test_singular_stencils():
    ctx = M.Ctx(0)
    # a node given twice: two equal rows of [A P; P^T 0]
    grid = W.pec_box((12, 12), 0.25, 33)
    xyz = np.vstack([grid.xyz, grid.xyz[70:71]])
    nd = M.Nodes(ctx, xyz, np.zeros(2))
    st = M.Stencils(nd, nd, 12)
    assert _status(M.Weights, st, 12, 3, 2, M.MFD_OP_GRAD) == M.MFD_ERR_SINGULAR
    assert _status(M.Weights, st, 12, 3, 1, M.MFD_OP_LAP_POW, 1) == M.MFD_ERR_SINGULAR
    # a cluster of 12 nodes on the line y = 100, far from a 10 x 10 grid: the
    # stencils of its nodes are collinear, so the monomials y, xy, y^2 vanish
    line = np.c_[0.1 * np.arange(12), np.full(12, 100.0)]
    g2 = W.pec_box((10, 10), 0.25, 34).xyz
    nd2 = M.Nodes(ctx, np.vstack([g2, line]), np.zeros(2))
    st2 = M.Stencils(nd2, nd2, 12)
    idx = st2.read()
    assert set(idx[100:].reshape(-1).tolist()) == set(range(100, 112))
    assert _status(M.Weights, st2, 12, 3, 2, M.MFD_OP_GRAD) == M.MFD_ERR_SINGULAR
    # the context stays usable: a regular set still gives weights
    ok = M.Nodes(ctx, grid.xyz, np.zeros(2))
    M.Weights(M.Stencils(ok, ok, 12), 12, 3, 2, M.MFD_OP_GRAD)


def test_argument_errors():
    ctx = M.Ctx(0)
    ns = W.pec_box((6, 6), 0.25, 35)
    nd = M.Nodes(ctx, ns.xyz, ns.period)
    assert _status(M.Stencils, nd, nd, ns.n + 1) == M.MFD_ERR_ARG  # n > N
    assert _status(M.Stencils, nd, nd, 0) == M.MFD_ERR_ARG
    assert _status(M.Nodes, ctx, np.zeros((4, 4)), None) == M.MFD_ERR_ARG  # dim 4
    st = M.Stencils(nd, nd, 12)
    assert _status(M.Weights, st, 13, 3, 2, M.MFD_OP_GRAD) == M.MFD_ERR_ARG  # n_use > n
    assert _status(M.Weights, st, 12, 4, 2, M.MFD_OP_GRAD) == M.MFD_ERR_ARG  # even PHS power
    assert _status(M.Weights, st, 12, 3, 2, M.MFD_OP_LAP_POW, 2) == M.MFD_ERR_ARG  # r^3 for Delta^2
    assert _status(M.Weights, st, 12, 3, 2, M.MFD_OP_GRAD_VFD, 0, 0.0) == M.MFD_ERR_ARG  # delta = 0
    curl = M.Weights(st, 12, 3, 2, M.MFD_OP_GRAD)
    hv = M.Weights(st, 12, 3, 2, M.MFD_OP_LAP_POW, 1)
    dt, eps0, mu0, c0, eta0 = W.units(S)
    assert _status(M.Sim, ctx, 2, M.MFD_FP64, dt, eps0, mu0, 0.0, hv, curl) == M.MFD_ERR_ARG  # swapped
    assert _status(M.Sim, ctx, 2, M.MFD_FP64, -dt, eps0, mu0, 0.0, curl, hv) == M.MFD_ERR_ARG
    sim = M.Sim(ctx, 2, M.MFD_FP64, dt, eps0, mu0, 0.0, curl, hv)
    assert _status(sim.set_field, M.MFD_HZ, np.zeros(ns.n)) == M.MFD_ERR_ARG  # not a TMz component
    assert _status(sim.set_materials, np.zeros(ns.n), None) == M.MFD_ERR_ARG  # eps_r = 0
    assert _status(sim.set_probes, [ns.n], 10) == M.MFD_ERR_ARG
    assert _status(sim.grad, 5, -1) == M.MFD_ERR_ARG
    assert _status(M.Batch, ctx, [(curl, hv, dt, eps0, mu0, 0.0)], 5) == M.MFD_ERR_ARG  # nrhs
    # a rejected call changes nothing: the simulation still steps
    sim.set_field(M.MFD_EZ, np.ones(ns.n))
    sim.step(3)
    assert sim.steps == 3


def _run_everything(ns, src, probes, nsteps=12):
    """Every object kind, from the context on, through a short run of each."""
    dt, eps0, mu0, c0, eta0 = W.units(S)
    ctx = M.Ctx(0)
    nd = M.Nodes(ctx, ns.xyz, ns.period)
    st = M.Stencils(nd, nd, 31)
    curl = M.Weights(st, 12, 3, 2, M.MFD_OP_GRAD)
    hv = M.Weights(st, 31, 5, 4, M.MFD_OP_LAP_POW, 2)
    sim = M.Sim(ctx, 2, M.MFD_FP32, dt, eps0, mu0, -C_HV, curl, hv, compensated=True)
    sim.set_materials(W.eps_r_uniform(ns.n, 36), ns.pec)
    ez, hx, hy = W.tm11_fields(ns.xyz, float(np.max(ns.xyz[:, 0])), c0, mu0, 0.0, -0.5 * dt)
    ez[ns.pec == 1] = 0
    for comp, f in ((M.MFD_EZ, ez), (M.MFD_HX, hx), (M.MFD_HY, hy)):
        sim.set_field(comp, f)
    sim.set_sources(src.node, src.amp, src.f0, src.t0)
    sim.set_probes(probes, 2 * nsteps)
    sim.step(nsteps)
    J, ge, ga = sim.grad(nsteps, 0, len(src.node))
    out = [sim.get_field(M.MFD_EZ), sim.read_probes(), np.array([J]), ge, ga]
    bt = M.Batch(ctx, [(curl, hv, dt, eps0, mu0, -C_HV)], nrhs=4)
    bt.set_materials(0, None, ns.pec)
    bt.set_field(0, M.MFD_EZ, np.repeat(ez[:, None], 4, 1))
    bt.set_probes(0, probes, nsteps)
    bt.step(nsteps)
    out += [bt.get_field(0, M.MFD_EZ), bt.read_probes(0)]
    y = M.Yee(ctx, 16, 16, M.MFD_FP32, dt, 1.0, eps0, mu0)
    y.set_field(M.MFD_EZ, np.ones((16, 16)))
    y.set_probes([5, 9], nsteps)
    y.step(nsteps)
    out += [y.read_probes()]
    return out


def test_injected_allocation_failures_return_oom_and_leave_the_library_usable():
    ns = W.pec_box((16, 16), 0.25, 37)
    dt, eps0, mu0, c0, eta0 = W.units(S)
    src = W.ricker_sources(ns, 2, 38, c0)
    probes = W.interior_nodes(ns, 3, 39)
    M.debug_fail_alloc(-1)
    ref = _run_everything(ns, src, probes)
    fired = 0
    try:
        for k in range(400):
            M.debug_fail_alloc(k)
            st = _status(_run_everything, ns, src, probes)
            if st == M.MFD_OK:
                assert M.debug_alloc_pending() >= 0  # every allocation of the run comes before k
                break
            assert st == M.MFD_ERR_OOM, (k, st)
            assert M.debug_alloc_pending() == -1  # the injected failure fired
            fired += 1
        else:
            pytest.fail("the run never completed without meeting the injected failure")
    finally:
        M.debug_fail_alloc(-1)
    assert fired >= 30  # every object kind allocates on the way
    again = _run_everything(ns, src, probes)
    for a, b in zip(ref, again):
        assert np.allclose(a, b, rtol=1e-12, atol=0)
