"""The GPU adjoint (mfd_grad: transposed stencil gathers run backwards with
checkpointed recomputation) against the FP64 oracle adjoint and against central
finite differences.

* small PEC box, FP64: J, dJ/deps_r and dJ/d amplitude match the oracle's
  gradient (orc_grad_tmz) to 1e-9 (relative, max-norm); FP32 to 1e-4.
* checkpoint spacing does not change the result (FP64: identical).
* torch.autograd through ProbeEnergy returns the adjoint gradients.
* full config (250k nodes, n = 20, 4000 FP32 steps, 8 probes, 4 sources,
  eps_r = 1 + 0.5 U[0,1], checkpoints every 64 steps): the FP32 adjoint is
  within 1e-4 of the FP64 adjoint, and the FP64 adjoint within 1e-4 of central
  finite differences (step 1e-3, FP64 forward runs) at 32 random nodes and all
  source amplitudes (relative L2 over the sampled gradient entries).
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

M = pytest.importorskip("paper_2508_18205_gb300")

S, C_HV = 0.5, 4e-3


def _problem(ctx, nodes, prec, n=20, m=2):
    dt, eps0, mu0, c0, eta0 = W.units(S)
    nd = M.Nodes(ctx, nodes.xyz, nodes.period)
    st = M.Stencils(nd, nd, max(n, 31))
    cw = M.Weights(st, n, 3, m, M.MFD_OP_GRAD)
    hw = M.Weights(st, 31, 5, 4, M.MFD_OP_LAP_POW, 2)
    sim = M.Sim(ctx, 2, prec, dt, eps0, mu0, -C_HV, cw, hw)
    sim._nodes_keep = (nd, st)
    return sim


def _setup(nodes, seed):
    dt, eps0, mu0, c0, eta0 = W.units(S)
    src = W.ricker_sources(nodes, 3, seed, c0)
    probes = W.interior_nodes(nodes, 4, seed + 1)
    eps = W.eps_r_uniform(nodes.n, seed + 2)
    rng = np.random.default_rng(seed)
    ez = 0.1 * rng.standard_normal(nodes.n)
    ez[nodes.pec == 1] = 0
    hx, hy = 0.1 * rng.standard_normal((2, nodes.n))
    return src, probes, eps, ez, hx, hy


def _gpu_grad(sim, nodes, src, probes, eps, ez, hx, hy, nsteps, every):
    sim.set_materials(eps, nodes.pec)
    sim.set_field(M.MFD_EZ, ez)
    sim.set_field(M.MFD_HX, hx)
    sim.set_field(M.MFD_HY, hy)
    sim.set_sources(src.node, src.amp, src.f0, src.t0)
    sim.set_probes(probes, nsteps)
    return sim.grad(nsteps, every, len(src.node))


@pytest.mark.parametrize("prec,tol", [(1, 1e-9), (0, 1e-4)])
def test_adjoint_matches_oracle(prec, tol):
    ctx = M.Ctx(0)
    dt, eps0, mu0, c0, eta0 = W.units(S)
    nodes = W.pec_box((23, 19), 0.25, 91)
    src, probes, eps, ez, hx, hy = _setup(nodes, 92)
    nsteps = 60
    sim = _problem(ctx, nodes, prec)
    J, ge, ga = _gpu_grad(sim, nodes, src, probes, eps, ez, hx, hy, nsteps, 7)
    prob, _ = O.tmz_collocated(nodes, 20, 3, 2, 2, dt, eps0, mu0, -C_HV, eps_r=eps)
    rJ, rge, rga = O.grad_tmz(prob, ez, hx, hy, nsteps, src, probes)
    assert abs(J - rJ) <= tol * abs(rJ)
    assert np.max(np.abs(ge - rge)) <= tol * np.max(np.abs(rge))
    assert np.max(np.abs(ga - rga)) <= tol * np.max(np.abs(rga))
    assert np.all(ge[nodes.pec == 1] == 0)
    assert sim.steps == nsteps


def test_checkpoint_spacing_does_not_change_the_gradient():
    """Checkpoints every 1, 8 or 1000 steps, or the whole Ez history (every = 0,
    no recomputation): the same operations in the same order, the same bits."""
    ctx = M.Ctx(0)
    nodes = W.pec_box((17, 17), 0.25, 93)
    src, probes, eps, ez, hx, hy = _setup(nodes, 94)
    assert len(set(src.node)) == len(src.node) and len(set(probes)) == len(probes)
    out = []
    for every in (0, 1, 8, 1000, 64):
        sim = _problem(ctx, nodes, 1)
        out.append(_gpu_grad(sim, nodes, src, probes, eps, ez, hx, hy, 40, every))
    for J, ge, ga in out[1:]:
        assert J == out[0][0]
        assert np.array_equal(ge, out[0][1]) and np.array_equal(ga, out[0][2])


def test_autograd_function_returns_adjoint_gradients():
    torch = pytest.importorskip("torch")
    ctx = M.Ctx(0)
    nodes = W.pec_box((15, 15), 0.25, 95)
    src, probes, eps, ez, hx, hy = _setup(nodes, 96)
    sim = _problem(ctx, nodes, 1)
    obj = M.ProbeObjective(sim, nodes.pec, {M.MFD_EZ: ez, M.MFD_HX: hx, M.MFD_HY: hy}, src, probes, 30, 8)
    e = torch.tensor(eps, dtype=torch.float64, requires_grad=True)
    a = torch.tensor(src.amp, dtype=torch.float64, requires_grad=True)
    J = M.probe_energy(e, a, obj)
    (3.0 * J).backward()
    J2, ge, ga = obj.run(eps, src.amp)
    assert abs(float(J.detach()) - J2) <= 1e-12 * abs(J2)
    assert np.allclose(e.grad.numpy(), 3.0 * ge, rtol=0, atol=1e-15 * np.max(np.abs(ge)) + 0)
    assert np.allclose(a.grad.numpy(), 3.0 * ga)


def test_autograd_on_device_tensors_and_no_grad_forward():
    """CUDA tensors in and out (zero copy): the gradient equals mfd_grad's bit for
    bit; under torch.no_grad() (or without requires_grad) the forward pass records
    no tape and no adjoint sweep runs, and J is the same."""
    torch = pytest.importorskip("torch")
    ctx = M.Ctx(0)
    nodes = W.pec_box((18, 18), 0.25, 97)
    src, probes, eps, ez, hx, hy = _setup(nodes, 98)
    for prec in (1, 0):
        sim = _problem(ctx, nodes, prec)
        obj = M.ProbeObjective(sim, nodes.pec, {M.MFD_EZ: ez, M.MFD_HX: hx, M.MFD_HY: hy}, src, probes, 50, 0)
        J_ref, ge_ref, ga_ref = obj.run(eps, src.amp)
        sweeps = sim.adjoint_sweeps
        e = torch.tensor(eps, dtype=torch.float64, device="cuda", requires_grad=True)
        a = torch.tensor(src.amp, dtype=torch.float64, device="cuda", requires_grad=True)
        with torch.no_grad():
            J0 = M.probe_energy(e, a, obj)
        assert obj.last_forward_taped is False and sim.adjoint_sweeps == sweeps
        J1 = M.probe_energy(e.detach(), a.detach(), obj)
        assert obj.last_forward_taped is False and sim.adjoint_sweeps == sweeps
        J = M.probe_energy(e, a, obj)
        assert obj.last_forward_taped is True and sim.adjoint_sweeps == sweeps  # forward only so far
        J.backward()
        assert sim.adjoint_sweeps == sweeps + 1
        assert e.grad.is_cuda and a.grad.is_cuda
        for Jx in (J0, J1, J):
            assert abs(float(Jx) - J_ref) <= 1e-12 * abs(J_ref)
        assert np.array_equal(e.grad.cpu().numpy(), ge_ref)
        assert np.array_equal(a.grad.cpu().numpy(), ga_ref)


def test_tape_sweeps_once_and_refuses_a_moved_simulation():
    ctx = M.Ctx(0)
    nodes = W.pec_box((14, 14), 0.25, 99)
    src, probes, eps, ez, hx, hy = _setup(nodes, 100)
    sim = _problem(ctx, nodes, 1)
    obj = M.ProbeObjective(sim, nodes.pec, {M.MFD_EZ: ez, M.MFD_HX: hx, M.MFD_HY: hy}, src, probes, 20, 0)
    lib = M.lib()
    import ctypes as C
    ge = np.zeros(nodes.n)
    ga = np.zeros(len(src.node))
    for moved in (False, True):
        J, tape = obj.forward(eps, src.amp, True)
        if moved:
            sim.step(1)
            st = lib.mfd_grad_backward(tape, C.c_void_p(ge.ctypes.data), C.c_void_p(ga.ctypes.data), 0, None)
            assert st == M.MFD_ERR_STATE
        else:
            assert lib.mfd_grad_backward(tape, C.c_void_p(ge.ctypes.data), C.c_void_p(ga.ctypes.data), 0, None) == 0
            st = lib.mfd_grad_backward(tape, C.c_void_p(ge.ctypes.data), C.c_void_p(ga.ctypes.data), 0, None)
            assert st == M.MFD_ERR_STATE
        lib.mfd_tape_destroy(tape)
    J2, ge2, ga2 = obj.run(eps, src.amp)
    J3, tape = obj.forward(eps, src.amp, True)
    ge3, ga3 = obj.backward(tape, "cpu")
    assert J3 == J2 and np.array_equal(ge3.numpy(), ge2) and np.array_equal(ga3.numpy(), ga2)


def test_full_config_adjoint_fp32_fp64_and_finite_differences():
    """250k nodes (500 x 500 PEC box), n = 20, 4000 steps, checkpoints every 64 steps."""
    ctx = M.Ctx(0)
    dt, eps0, mu0, c0, eta0 = W.units(S)
    nodes = W.pec_box((500, 500), 0.25, 5)
    eps = W.eps_r_uniform(nodes.n, 55)
    src = W.ricker_sources(nodes, 4, 56, c0)
    probes = W.interior_nodes(nodes, 8, 57)
    z = np.zeros(nodes.n)
    nsteps, every = 4000, 64
    res = {}
    sims = {}
    for prec in (0, 1):
        sims[prec] = _problem(ctx, nodes, prec)
        res[prec] = _gpu_grad(sims[prec], nodes, src, probes, eps, z, z, z, nsteps, every)
    J32, g32, a32 = res[0]
    J64, g64, a64 = res[1]
    assert abs(J32 - J64) <= 1e-4 * abs(J64)
    assert np.linalg.norm(g32 - g64) <= 1e-4 * np.linalg.norm(g64)
    assert np.linalg.norm(a32 - a64) <= 1e-4 * np.linalg.norm(a64)
    # central finite differences of the FP64 forward run
    s64 = sims[1]

    def J_of(e, amp):
        s64.set_materials(e, nodes.pec)
        for c in (M.MFD_EZ, M.MFD_HX, M.MFD_HY):
            s64.set_field(c, z)
        s64.set_sources(src.node, amp, src.f0, src.t0)
        s64.set_probes(probes, nsteps)
        s64.step(nsteps)
        p = s64.read_probes()
        return dt * float(np.sum(p * p))

    d = 1e-3
    sample = W.interior_nodes(nodes, 32, 58)
    fd, ad = [], []
    for i in sample:
        e1 = eps.copy()
        e1[i] += d
        e2 = eps.copy()
        e2[i] -= d
        fd.append((J_of(e1, src.amp) - J_of(e2, src.amp)) / (2 * d))
        ad.append(g64[i])
    for k in range(len(src.node)):
        a1 = src.amp.copy()
        a1[k] += d
        a2 = src.amp.copy()
        a2[k] -= d
        fd.append((J_of(eps, a1) - J_of(eps, a2)) / (2 * d))
        ad.append(a64[k])
    fd, ad = np.array(fd), np.array(ad)
    assert np.linalg.norm(ad - fd) <= 1e-4 * np.linalg.norm(fd), (ad[:8], fd[:8])
