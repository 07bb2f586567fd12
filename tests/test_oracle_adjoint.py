"""Pins of the oracle's adjoint (the transpose of the Eq. 19 step) and its gradient.

* Dot-product test: <M v, w> = <v, M^T w> for the homogeneous one-step map M
  (the forward oracle) and the oracle's transposed step, to FP64 round-off, on
  the collocated PEC box with varying eps_r and on the staggered periodic layout.
* The gradient of J = dt sum_n sum_p (Ez_p^n)^2 with respect to eps_r and the
  source amplitudes matches central finite differences of the forward oracle (FP64).
"""
import math

import numpy as np

import oracle as O
import workloads as W


def _colloc(seed=1):
    S = 0.5
    dt, eps0, mu0, c0, eta0 = W.units(S)
    nodes = W.pec_box((12, 12), 0.25, seed)
    er = W.eps_r_uniform(nodes.n, 77)
    prob, _ = O.tmz_collocated(nodes, 12, 3, 2, 2, dt, eps0, mu0, -4e-3, eps_r=er)
    return nodes, prob, c0


def _dot_test(prob, ne, nh):
    rng = np.random.default_rng(11)
    v = rng.standard_normal(ne + 2 * nh)
    w = rng.standard_normal(ne + 2 * nh)
    e, x, y, _, _ = O.run_tmz(prob, v[:ne], v[ne:ne + nh], v[ne + nh:], 1)
    Mv = np.r_[e, x, y]
    le, lx, ly = O.adjoint_step_tmz(prob, w[:ne], w[ne:ne + nh], w[ne + nh:])
    Mtw = np.r_[le, lx, ly]
    a, b = np.dot(Mv, w), np.dot(v, Mtw)
    assert abs(a - b) <= 1e-12 * (np.linalg.norm(Mv) * np.linalg.norm(w))


def test_dot_product_collocated_pec():
    nodes, prob, _ = _colloc()
    _dot_test(prob, nodes.n, nodes.n)


def test_dot_product_staggered():
    S = 0.5
    dt, eps0, mu0, c0, eta0 = W.units(S)
    e = W.periodic_box((14, 14), 0.25, 2)
    h = W.periodic_box((14, 14), 0.25, 3, offset=(0.5, 0.5))
    prob = O.tmz_staggered(e, h, 12, 3, 2, 2, dt, eps0, mu0, -1e-3,
                           eps_r=W.eps_r_uniform(e.n, 5))
    _dot_test(prob, e.n, h.n)


def test_gradient_matches_central_differences():
    nodes, prob, c0 = _colloc(4)
    src = W.ricker_sources(nodes, 2, 31, c0)
    probes = W.interior_nodes(nodes, 3, 32)
    rng = np.random.default_rng(5)
    ez = 0.1 * rng.standard_normal(nodes.n)
    ez[nodes.pec == 1] = 0
    hx, hy = 0.1 * rng.standard_normal((2, nodes.n))
    nsteps = 40
    J, ge, ga = O.grad_tmz(prob, ez, hx, hy, nsteps, src, probes)

    def Jof(p, s):
        _, _, _, pr, _ = O.run_tmz(p, ez, hx, hy, nsteps, sources=s, probes=probes)
        return p.dt * float(np.sum(pr * pr))

    assert abs(Jof(prob, src) - J) <= 1e-12 * abs(J)
    d = 1e-3
    for i in W.interior_nodes(nodes, 5, 33):
        er0 = prob.eps_r[i]
        prob.eps_r[i] = er0 + d
        jp = Jof(prob, src)
        prob.eps_r[i] = er0 - d
        jm = Jof(prob, src)
        prob.eps_r[i] = er0
        fd = (jp - jm) / (2 * d)
        assert abs(fd - ge[i]) <= 1e-5 * max(abs(fd), 1e-3 * np.max(np.abs(ge)))
    for s in range(2):
        a0 = src.amp[s]
        src.amp[s] = a0 + d
        jp = Jof(prob, src)
        src.amp[s] = a0 - d
        jm = Jof(prob, src)
        src.amp[s] = a0
        fd = (jp - jm) / (2 * d)
        assert abs(fd - ga[s]) <= 1e-8 * max(abs(fd), 1.0)
    # PEC nodes carry no permittivity gradient
    assert np.all(ge[nodes.pec == 1] == 0)
