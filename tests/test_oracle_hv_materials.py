"""Pins of the hyperviscosity term (Eqs. 17-19) and of the relative permittivity
in the E row (eps0 -> eps0 eps_r, hyperviscosity included) of the oracle's
TMz and 3D steppers.

* 3D plus stencil: with 7 nodes (centre and the six axis neighbours at
  distance h), PHS r^k and monomials of degree <= 1, symmetry gives one arm
  weight a and a centre weight -6a for the Laplacian (constants are
  annihilated); the RBF row of an arm node then reads
  a (2^k + 4 2^(k/2) - 12) h^k ... = k (k + 1) h^(k-2), the 3D Laplacian of
  r^k being k (k + 1) r^(k-2). So a = k (k + 1) / ((2^k + 2^(2 + k/2) - 12) h^2).
* Curl-free Fourier modes: on a regular periodic grid with those stencils the
  central differences act on exp(i k.x) as i s_b (s_b = sin(k_b h) / h), so the
  field F_a = s_a cos(k.x) has zero discrete curl, and the hyperviscosity
  stencil acts on it as the number v = a sum_b (2 cos(k_b h) - 2). Such a
  field only feels the hyperviscosity term: each step multiplies E by
  1 + dt gamma v / (eps0 eps_r) and H by 1 + dt gamma v / mu0, exactly.
* The full one-step map on a Fourier mode (App. A, extended by the
  hyperviscosity and eps_r terms) and its eigenvalues: |lambda| = 1 without
  hyperviscosity below the stability limit, |lambda| < 1 with the dissipative
  sign of gamma (Sec. 5.1: gamma = c (-1)^(alpha-1) h^(2 alpha), c > 0), and
  some |lambda| > 1 with the opposite sign.
* Discrete plane waves in a uniform medium eps_r: the leapfrog with central
  differences carries E = p cos(k.x - w t) exactly when
  sin(w dt / 2) = (dt |s| / 2) / sqrt(mu0 eps0 eps_r); the phase speed tends
  to c0 / sqrt(eps_r) for small k (c0 / 2 at eps_r = 4).
* TM11 cavity filled with eps_r = 4 on jittered nodes follows the closed-form
  mode whose frequency is half the vacuum one, w = sqrt(2) pi c0 / (L sqrt(eps_r)).
* A non-uniform eps_r on regular grids: the oracle equals a numpy central
  difference leapfrog with the plus-stencil Laplacian, the E row divided by the
  node's own eps_r (curl and hyperviscosity terms alike).
* 3D energy (Eq. 20, Sec. 5.1 / App. A): with hyperviscosity u(t) stays in
  [0.99, 1.01] on jittered nodes at S_c = 1/(10 sqrt 2); without it the energy grows.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


def _plus_problem_3d(P, gamma, eps_r, S, k_phs=3):
    """Regular periodic P^3 cube, 7-point curl and Laplacian (alpha = 1) stencils."""
    dt, eps0, mu0, c0, eta0 = W.units(S)
    nodes = W.periodic_box((P, P, P), 0.0, 1)
    idx = O.knn(nodes.xyz, nodes.xyz, nodes.period, 7)
    wc = O.weights(nodes.xyz, nodes.xyz, nodes.period, idx, 7, k_phs, 1, O.OP_GRAD)
    wv = O.weights(nodes.xyz, nodes.xyz, nodes.period, idx, 7, k_phs, 1, O.OP_LAP_POW, 1)
    er = np.full(nodes.n, float(eps_r)) if np.isscalar(eps_r) else np.asarray(eps_r, float)
    prob = O.Max3D(n=nodes.n, c=O.Stencil(idx=idx.copy(), w=wc), v=O.Stencil(idx=idx.copy(), w=wv),
                   eps_r=er, wall=np.zeros(nodes.n, np.uint8), dt=dt, eps0=eps0, mu0=mu0, gamma=gamma)
    return nodes, prob


def _plus_problem_2d(P, gamma, eps_r, S, k_phs=3):
    """Regular periodic P^2 square, 5-point curl and Laplacian (alpha = 1) stencils."""
    dt, eps0, mu0, c0, eta0 = W.units(S)
    nodes = W.periodic_box((P, P), 0.0, 1)
    idx = O.knn(nodes.xyz, nodes.xyz, nodes.period, 5)
    wc = O.weights(nodes.xyz, nodes.xyz, nodes.period, idx, 5, k_phs, 1, O.OP_GRAD)
    wv = O.weights(nodes.xyz, nodes.xyz, nodes.period, idx, 5, k_phs, 1, O.OP_LAP_POW, 1)
    er = np.full(nodes.n, float(eps_r)) if np.isscalar(eps_r) else np.asarray(eps_r, float)
    curl = O.Stencil(idx=idx.copy(), w=wc)
    hv = O.Stencil(idx=idx.copy(), w=wv)
    prob = O.TMz(nh=nodes.n, ne=nodes.n, hc=curl, hv=hv, ec=curl, ev=hv, eps_r=er,
                 pec=np.zeros(nodes.n, np.uint8), dt=dt, eps0=eps0, mu0=mu0, gamma=gamma)
    return nodes, prob


def _arm_3d(k, h=1.0):
    return k * (k + 1) / ((2 ** k + 2 ** (2 + k / 2) - 12) * h * h)


def _arm_2d(k, h=1.0):
    return k * k / ((2 ** k + 2 ** (1 + k / 2) - 8) * h * h)


@pytest.mark.parametrize("k", [3, 5, 7])
@pytest.mark.parametrize("h", [1.0, 0.37])
def test_3d_plus_stencil_closed_forms(k, h):
    rel = np.array([[0, 0, 0], [h, 0, 0], [-h, 0, 0], [0, h, 0], [0, -h, 0], [0, 0, h], [0, 0, -h]], float)
    w = O.stencil_weights(rel, k, 1, O.OP_GRAD)
    for a in range(3):
        exp = np.zeros(7)
        exp[1 + 2 * a], exp[2 + 2 * a] = 1 / (2 * h), -1 / (2 * h)
        assert np.allclose(w[a], exp, rtol=0, atol=1e-13 / h)
    wl = O.stencil_weights(rel, k, 1, O.OP_LAP_POW, 1)[0]
    a = _arm_3d(k, h)
    assert np.allclose(wl, [-6 * a] + [a] * 6, rtol=1e-12, atol=0)


def _mode_k(P, m):
    return 2 * math.pi * np.asarray(m, float) / P


def test_3d_curl_free_modes_decay_only_by_hyperviscosity():
    """E (and H) = s cos(k.x) has zero discrete curl: the step multiplies it by
    1 + dt gamma v / (eps0 eps_r) (E) and 1 + dt gamma v / mu0 (H), v the HV symbol."""
    P, S, gamma, er = 8, 0.3, 0.05, 2.5
    nodes, prob = _plus_problem_3d(P, gamma, er, S)
    dt, eps0, mu0 = prob.dt, prob.eps0, prob.mu0
    k = _mode_k(P, (1, 2, 3))
    s = np.sin(k)
    a = _arm_3d(3)
    v = a * np.sum(2 * np.cos(k) - 2)
    ph = np.cos(nodes.xyz @ k)
    F = np.outer(s, ph)
    nst = 20
    fe = (1 + dt * gamma * v / (eps0 * er)) ** nst
    fh = (1 + dt * gamma * v / mu0) ** nst
    assert fe < 1 and fh < fe  # dissipative, and E slower by 1/eps_r
    E1, H1, _, _ = O.run_3d(prob, F, np.zeros_like(F), nst)
    assert np.allclose(E1, fe * F, rtol=0, atol=1e-12)
    assert np.max(np.abs(H1)) < 1e-12
    E1, H1, _, _ = O.run_3d(prob, np.zeros_like(F), F, nst)
    assert np.allclose(H1, fh * F, rtol=0, atol=1e-12)
    assert np.max(np.abs(E1)) < 1e-12


def test_2d_curl_free_h_mode_decays_only_by_hyperviscosity():
    P, S, gamma = 16, 0.3, 0.05
    nodes, prob = _plus_problem_2d(P, gamma, 2.0, S)
    k = _mode_k(P, (2, 3))
    s = np.sin(k)
    v = _arm_2d(3) * np.sum(2 * np.cos(k) - 2)
    ph = np.cos(nodes.xyz @ k)
    nst = 25
    fh = (1 + prob.dt * gamma * v / prob.mu0) ** nst
    ez, hx, hy, _, _ = O.run_tmz(prob, np.zeros(nodes.n), s[0] * ph, s[1] * ph, nst)
    assert np.allclose(hx, fh * s[0] * ph, rtol=0, atol=1e-12)
    assert np.allclose(hy, fh * s[1] * ph, rtol=0, atol=1e-12)
    assert np.max(np.abs(ez)) < 1e-12


def _curl_symbol(s):
    """i s x . as a 3 x 3 matrix."""
    return 1j * np.array([[0, -s[2], s[1]], [s[2], 0, -s[0]], [-s[1], s[0], 0]])


def _one_step_map_3d(prob, nodes, k):
    ph = np.exp(1j * (nodes.xyz @ k))
    G = np.zeros((6, 6), complex)
    for col in range(6):
        v = np.zeros((6, nodes.n), complex)
        v[col] = ph
        re = O.run_3d(prob, v[:3].real, v[3:].real, 1)
        im = O.run_3d(prob, v[:3].imag, v[3:].imag, 1)
        out = np.r_[re[0] + 1j * im[0], re[1] + 1j * im[1]]
        for row in range(6):
            G[row, col] = np.mean(out[row] / ph)
            assert np.allclose(out[row], G[row, col] * ph, atol=1e-12)
    return G


@pytest.mark.parametrize("gamma", [0.0, 0.04])
def test_3d_one_step_map_with_hyperviscosity_and_eps_r(gamma):
    P, S, er = 8, 0.3, 2.5
    nodes, prob = _plus_problem_3d(P, gamma, er, S)
    k = _mode_k(P, (1, 2, 3))
    s = np.sin(k)
    v = _arm_3d(3) * np.sum(2 * np.cos(k) - 2)
    c1, c2 = prob.dt / prob.mu0, prob.dt / (prob.eps0 * er)
    Cs = _curl_symbol(s)
    I = np.eye(3)
    # H' = (1 + c1 gamma v) H - c1 curl E;  E' = (1 + c2 gamma v) E + c2 curl H'
    GE_E = (1 + c2 * gamma * v) * I - c1 * c2 * Cs @ Cs
    GE_H = c2 * (1 + c1 * gamma * v) * Cs
    GH_E = -c1 * Cs
    GH_H = (1 + c1 * gamma * v) * I
    ref = np.block([[GE_E, GE_H], [GH_E, GH_H]])
    G = _one_step_map_3d(prob, nodes, k)
    assert np.allclose(G, ref, atol=1e-12)
    lam = np.abs(np.linalg.eigvals(G))
    if gamma == 0.0:
        assert np.allclose(lam, 1.0, atol=1e-10)
    else:
        assert np.all(lam < 1.0)


def test_3d_antidissipative_sign_grows():
    """With the opposite sign of gamma the hyperviscosity feeds the mode: some |lambda| > 1."""
    P, S = 8, 0.3
    nodes, prob = _plus_problem_3d(P, -0.04, 1.0, S)
    G = _one_step_map_3d(prob, nodes, _mode_k(P, (1, 2, 3)))
    assert np.max(np.abs(np.linalg.eigvals(G))) > 1.0 + 1e-3


def test_2d_one_step_map_with_hyperviscosity_and_eps_r():
    """App. A's Eq. A.6 with the hyperviscosity and eps_r terms of the E and H rows."""
    P, S, er, gamma = 16, 0.35, 3.0, 0.03
    nodes, prob = _plus_problem_2d(P, gamma, er, S)
    k = _mode_k(P, (2, 5))
    s = np.sin(k)
    v = _arm_2d(3) * np.sum(2 * np.cos(k) - 2)
    ph = np.exp(1j * (nodes.xyz @ k))
    G = np.zeros((3, 3), complex)  # state (Hx, Hy, Ez)
    for col in range(3):
        u = [np.zeros(nodes.n, complex) for _ in range(3)]
        u[col] = ph
        re = O.run_tmz(prob, u[2].real, u[0].real, u[1].real, 1)
        im = O.run_tmz(prob, u[2].imag, u[0].imag, u[1].imag, 1)
        res = [re[1] + 1j * im[1], re[2] + 1j * im[2], re[0] + 1j * im[0]]
        for row in range(3):
            G[row, col] = np.mean(res[row] / ph)
    c1, c2 = prob.dt / prob.mu0, prob.dt / (prob.eps0 * er)
    wx, wy = 1j * s[0], 1j * s[1]
    dh, de = 1 + c1 * gamma * v, 1 + c2 * gamma * v
    ref = np.array([[dh, 0, -c1 * wy], [0, dh, c1 * wx],
                    [-c2 * wy * dh, c2 * wx * dh, de + c1 * c2 * (wx * wx + wy * wy)]])
    assert np.allclose(G, ref, atol=1e-12)
    assert np.all(np.abs(np.linalg.eigvals(G)) < 1.0)


def _discrete_omega(s_norm, dt, mu0, eps0, er):
    return 2 * math.asin(0.5 * dt * s_norm / math.sqrt(mu0 * eps0 * er)) / dt


@pytest.mark.parametrize("er", [1.0, 4.0])
def test_2d_discrete_plane_wave_in_a_medium(er):
    P, S, nst = 32, 0.4, 150
    nodes, prob = _plus_problem_2d(P, 0.0, er, S)
    dt, eps0, mu0 = prob.dt, prob.eps0, prob.mu0
    k = _mode_k(P, (3, 2))
    s = np.sin(k)
    sn = np.linalg.norm(s)
    w = _discrete_omega(sn, dt, mu0, eps0, er)
    # E = z cos(k.x - w t), H = q cos(k.x - w t) with q = c1 (s x z) / (2 sin(w dt/2)) (3D form)
    q = (dt / mu0) * np.array([s[1], -s[0]]) / (2 * math.sin(0.5 * w * dt))
    x = nodes.xyz

    def fields(n):
        return (np.cos(x @ k - w * n * dt), q[0] * np.cos(x @ k - w * (n - 0.5) * dt),
                q[1] * np.cos(x @ k - w * (n - 0.5) * dt))

    ez, hx, hy = fields(0)
    e1, x1, y1, _, _ = O.run_tmz(prob, ez, hx, hy, nst)
    ea, xa, ya = fields(nst)
    assert np.allclose(e1, ea, atol=1e-11)
    assert np.allclose(x1, xa, atol=1e-11)
    assert np.allclose(y1, ya, atol=1e-11)
    if er == 4.0:
        # the same data in vacuum would be a different wave: the medium matters
        vac = _discrete_omega(sn, dt, mu0, eps0, 1.0)
        assert abs(vac - w) * nst * dt > 0.5


def test_3d_discrete_plane_wave_in_a_medium():
    P, S, er, nst = 12, 0.3, 4.0, 120
    nodes, prob = _plus_problem_3d(P, 0.0, er, S)
    dt, eps0, mu0 = prob.dt, prob.eps0, prob.mu0
    k = _mode_k(P, (1, 2, 1))
    s = np.sin(k)
    p = np.cross(s, [1.0, 0.0, 0.0])
    p /= np.linalg.norm(p)
    w = _discrete_omega(np.linalg.norm(s), dt, mu0, eps0, er)
    q = (dt / mu0) * np.cross(s, p) / (2 * math.sin(0.5 * w * dt))
    x = nodes.xyz
    E0 = np.outer(p, np.cos(x @ k))
    H0 = np.outer(q, np.cos(x @ k + 0.5 * w * dt))
    E1, H1, _, _ = O.run_3d(prob, E0, H0, nst)
    assert np.allclose(E1, np.outer(p, np.cos(x @ k - w * nst * dt)), atol=1e-11)
    assert np.allclose(H1, np.outer(q, np.cos(x @ k - w * (nst - 0.5) * dt)), atol=1e-11)


def test_discrete_phase_speed_tends_to_c0_over_sqrt_eps_r():
    S, er = 0.4, 4.0
    dt, eps0, mu0, c0, eta0 = W.units(S)
    for kk, tol in ((0.05, 1e-3), (0.01, 4e-5)):
        w = _discrete_omega(math.sin(kk), dt, mu0, eps0, er)
        assert abs(w / kk - c0 / 2) < tol * c0


def _tm11_run(nx, steps, er, c=4e-3, S=0.5):
    dt, eps0, mu0, c0, eta0 = W.units(S)
    nodes = W.pec_box((nx, nx), 0.25, 1)
    prob, _ = O.tmz_collocated(nodes, 12, 3, 2, 2, dt, eps0, mu0, -c, eps_r=np.full(nodes.n, er))
    L = nx - 1
    cm = c0 / math.sqrt(er)
    ez, hx, hy = W.tm11_fields(nodes.xyz, L, cm, mu0, 0.0, -0.5 * dt)
    ez[nodes.pec == 1] = 0.0
    e1, x1, y1, _, _ = O.run_tmz(prob, ez, hx, hy, steps)
    T = steps * dt

    def err(speed):
        ea, xa, ya = W.tm11_fields(nodes.xyz, L, speed, mu0, T, T - 0.5 * dt)
        return (np.linalg.norm(np.r_[e1 - ea, x1 - xa, y1 - ya])
                / np.linalg.norm(np.r_[ea, xa, ya]))

    return err(cm), err(c0)


def test_tm11_cavity_in_a_medium_runs_at_half_the_frequency():
    """eps_r = 4 everywhere: w = sqrt(2) pi c0 / (2 L); the vacuum mode is far off."""
    e_med, e_vac = _tm11_run(41, 336, 4.0)
    assert e_med < 3e-3
    assert e_vac > 0.3


def test_nonuniform_eps_r_equals_numpy_leapfrog_2d():
    P, S, gamma = 12, 0.3, 0.05
    er = W.eps_r_uniform(P * P, 5, 1.0, 3.0)
    nodes, prob = _plus_problem_2d(P, gamma, er, S)
    dt, eps0, mu0 = prob.dt, prob.eps0, prob.mu0
    a = _arm_2d(3)
    rng = np.random.default_rng(11)
    ez, hx, hy = rng.standard_normal((3, nodes.n))
    out = O.run_tmz(prob, ez, hx, hy, 6)
    E, X, Y = (f.reshape(P, P).copy() for f in (ez, hx, hy))
    R = er.reshape(P, P)

    def r(f, dj, di):
        return np.roll(np.roll(f, -dj, axis=0), -di, axis=1)

    def dx(f):
        return 0.5 * (r(f, 0, 1) - r(f, 0, -1))

    def dy(f):
        return 0.5 * (r(f, 1, 0) - r(f, -1, 0))

    def lap(f):
        return a * (r(f, 0, 1) + r(f, 0, -1) + r(f, 1, 0) + r(f, -1, 0) - 4 * f)

    for _ in range(6):
        X1 = X + dt / mu0 * (-dy(E) + gamma * lap(X))
        Y1 = Y + dt / mu0 * (dx(E) + gamma * lap(Y))
        E = E + dt / (eps0 * R) * (dx(Y1) - dy(X1) + gamma * lap(E))
        X, Y = X1, Y1
    assert np.allclose(out[0], E.reshape(-1), atol=1e-12)
    assert np.allclose(out[1], X.reshape(-1), atol=1e-12)
    assert np.allclose(out[2], Y.reshape(-1), atol=1e-12)


def test_nonuniform_eps_r_equals_numpy_leapfrog_3d():
    P, S, gamma = 6, 0.3, 0.05
    er = W.eps_r_uniform(P ** 3, 6, 1.0, 3.0)
    nodes, prob = _plus_problem_3d(P, gamma, er, S)
    dt, eps0, mu0 = prob.dt, prob.eps0, prob.mu0
    a = _arm_3d(3)
    rng = np.random.default_rng(12)
    E0 = rng.standard_normal((3, nodes.n))
    H0 = rng.standard_normal((3, nodes.n))
    E1, H1, _, _ = O.run_3d(prob, E0, H0, 4)
    E = [E0[c].reshape(P, P, P).copy() for c in range(3)]
    H = [H0[c].reshape(P, P, P).copy() for c in range(3)]
    R = er.reshape(P, P, P)

    def d(f, ax_):  # array index [z, y, x]
        ax = 2 - ax_
        return 0.5 * (np.roll(f, -1, axis=ax) - np.roll(f, 1, axis=ax))

    def lap(f):
        return a * sum(np.roll(f, sh, axis=ax) for ax in range(3) for sh in (-1, 1)) - 6 * a * f

    def curl(F):
        return [d(F[2], 1) - d(F[1], 2), d(F[0], 2) - d(F[2], 0), d(F[1], 0) - d(F[0], 1)]

    for _ in range(4):
        cE = curl(E)
        H = [H[c] + dt / mu0 * (-cE[c] + gamma * lap(H[c])) for c in range(3)]
        cH = curl(H)
        E = [E[c] + dt / (eps0 * R) * (cH[c] + gamma * lap(E[c])) for c in range(3)]
    for c in range(3):
        assert np.allclose(E1[c], E[c].reshape(-1), atol=1e-12)
        assert np.allclose(H1[c], H[c].reshape(-1), atol=1e-12)


def _smooth_3d_fields(nodes, P):
    x = nodes.xyz
    k = 2 * math.pi / P
    E = np.zeros((3, nodes.n))
    E[2] = np.sin(k * x[:, 0]) * np.sin(k * x[:, 1])
    E[0] = np.cos(k * x[:, 1] + 0.3) * np.sin(k * x[:, 2])
    return E, np.zeros((3, nodes.n))


def test_3d_energy_band_with_hyperviscosity():
    """Sec. 5.1 criterion u in [0.99, 1.01] on a jittered periodic cube, alpha = 2,
    S_c = 1/(10 sqrt 2), c = 3e-4 (n = 40, r^3, m = 3; HV r^5, m = 4, 71 nodes)."""
    S = 1.0 / (10.0 * math.sqrt(2.0))
    dt, eps0, mu0, c0, eta0 = W.units(S)
    P = 24
    nodes = W.periodic_box((P, P, P), 0.25, 91)
    prob, _ = O.max3d_collocated(nodes, 40, 3, 3, 2, dt, eps0, mu0, -3e-4)
    E, H = _smooth_3d_fields(nodes, P)
    _, _, _, en = O.run_3d(prob, E, H, 1500, energy=True)
    u = en / en[0]
    assert np.all((u > 0.99) & (u < 1.01)), (u.min(), u.max())
    # Eq. 20's discrete energy is not the scheme's exact invariant, so it may
    # wiggle; it must not rise above its start by more than round-off-sized steps
    assert u.max() <= 1.0 + 1e-6, u.max()


def test_3d_energy_grows_without_hyperviscosity():
    """App. A in 3D: gamma = 0 on jittered nodes is unstable."""
    S = 1.0 / (10.0 * math.sqrt(2.0))
    dt, eps0, mu0, c0, eta0 = W.units(S)
    P = 16
    nodes = W.periodic_box((P, P, P), 0.25, 91)
    prob, _ = O.max3d_collocated(nodes, 40, 3, 3, 2, dt, eps0, mu0, 0.0)
    E, H = _smooth_3d_fields(nodes, P)
    _, _, _, en = O.run_3d(prob, E, H, 1500, energy=True)
    assert en[-1] / en[0] > 4.0
