"""Pins of the oracle's weights (Eq. 9 system, RBF-FD Eq. 13, RBF-VFD Eqs. 14-15, Sec. 5.1 HV).

* P-1 monomial exactness: the P^T rows of Eq. 9 force sum_j w_j p(x_j) = L p(x_c)
  for every monomial up to the augmentation degree. L p(x_c) is computed here
  with sympy, independently of the oracle's own right-hand side.
* P-2 the solver against LAPACK, and the residual of the saddle system.
* P-3 closed forms on the 5-point plus stencil with m = 1: by the reflection
  symmetries and linear exactness the d/dx weights are exactly +-1/(2h) on the
  x arms and 0 elsewhere, for every PHS r^k. For the Laplacian, symmetry leaves
  one unknown a (arm weight; centre -4a). Subtracting the centre row of Eq. 9
  from an arm row gives a h^k (2^k + 2^{1+k/2} - 8) = k^2 h^{k-2}, since
  Delta r^k = k^2 r^{k-2} in 2D; so a = k^2 / ((2^k + 2^{1+k/2} - 8) h^2)
  (r^3: 9 / (4 sqrt(2) h^2)), not the 5-point value 1/h^2.
* The RBF-VFD reading (central difference divided by 2 delta) differentiates x exactly.
* RBF-FD convergence: the derivative error of a smooth function falls with h.
"""
import math

import numpy as np
import pytest
import sympy as sp

import oracle as O
import workloads as W


def _exps(d, m):
    out = []
    for deg in range(m + 1):
        if d == 2:
            for a in range(deg, -1, -1):
                out.append((a, deg - a))
        else:
            for a in range(deg, -1, -1):
                for b in range(deg - a, -1, -1):
                    out.append((a, b, deg - a - b))
    return out


def _sym_op(d, e, op, axis=0, alpha=1):
    """L p at the origin by sympy, for p = prod x_a^e_a."""
    xs = sp.symbols("x0:%d" % d)
    p = sp.Integer(1)
    for a in range(d):
        p = p * xs[a] ** e[a]
    if op == "grad":
        q = sp.diff(p, xs[axis])
    else:
        q = p
        for _ in range(alpha):
            q = sum(sp.diff(q, xs[a], 2) for a in range(d))
    return float(q.subs({x: 0 for x in xs}))


def _stencil(nodes, c, n):
    idx = O.knn_brute(nodes.xyz[c:c + 1], nodes.xyz, nodes.period, n)[0]
    return nodes.xyz[idx] - nodes.xyz[c]


def test_monomial_order_graded():
    assert O.monomials(2, 2).tolist() == [[0, 0], [1, 0], [0, 1], [2, 0], [1, 1], [0, 2]]
    assert len(O.monomials(3, 3)) == math.comb(6, 3)
    assert len(O.monomials(2, 6)) == 28


@pytest.mark.parametrize("d,n,k,m", [(2, 12, 3, 2), (2, 30, 5, 4), (2, 20, 3, 2), (3, 40, 3, 3),
                                     (2, 40, 3, 4)])
def test_grad_monomial_exactness(d, n, k, m):
    nodes = W.pec_box((12, 12) if d == 2 else (7, 7, 7), 0.25, 21)
    c = nodes.n // 2 + 3
    rel = _stencil(nodes, c, n)
    w = O.stencil_weights(rel, k, m, O.OP_GRAD)
    for axis in range(d):
        for e in _exps(d, m):
            pv = np.prod(rel ** np.array(e), axis=1)
            got = float(np.dot(w[axis], pv))
            scale = float(np.sum(np.abs(w[axis] * pv))) + 1e-300
            assert abs(got - _sym_op(d, e, "grad", axis)) <= 1e-10 * max(scale, 1.0)


@pytest.mark.parametrize("d,alpha", [(2, 1), (2, 2), (2, 3), (3, 2)])
def test_lap_pow_monomial_exactness(d, alpha):
    mhv = 2 * alpha
    nhv = 2 * math.comb(mhv + d, d) + 1
    nodes = W.pec_box((16, 16) if d == 2 else (9, 9, 9), 0.25, 22)
    c = nodes.n // 2 + 5
    rel = _stencil(nodes, c, nhv)
    w = O.stencil_weights(rel, 2 * alpha + 1, mhv, O.OP_LAP_POW, alpha)
    for e in _exps(d, mhv):
        pv = np.prod(rel ** np.array(e), axis=1)
        got = float(np.dot(w[0], pv))
        scale = float(np.sum(np.abs(w[0] * pv)))
        assert abs(got - _sym_op(d, e, "lap", alpha=alpha)) <= 1e-10 * max(scale, 1.0), e


@pytest.mark.parametrize("k", [3, 5, 7, 9])
@pytest.mark.parametrize("h", [1.0, 0.37])
def test_plus_stencil_closed_forms(k, h):
    rel = np.array([[0, 0], [h, 0], [-h, 0], [0, h], [0, -h]], float)
    w = O.stencil_weights(rel, k, 1, O.OP_GRAD)
    exp_x = np.array([0, 1, -1, 0, 0]) / (2 * h)
    exp_y = np.array([0, 0, 0, 1, -1]) / (2 * h)
    assert np.allclose(w[0], exp_x, rtol=0, atol=1e-13 / h)
    assert np.allclose(w[1], exp_y, rtol=0, atol=1e-13 / h)
    wl = O.stencil_weights(rel, k, 1, O.OP_LAP_POW, 1)[0]
    a = k * k / ((2 ** k + 2 ** (1 + k / 2) - 8) * h * h)
    assert np.allclose(wl, [-4 * a, a, a, a, a], rtol=1e-12, atol=0)
    if k == 3:
        assert abs(a - 9 / (4 * math.sqrt(2) * h * h)) < 1e-12 / (h * h)


def test_vfd_differentiates_linear_exactly_and_reading():
    nodes = W.pec_box((12, 12), 0.25, 23)
    c = 60
    rel = _stencil(nodes, c, 12)
    w = O.stencil_weights(rel, 3, 2, O.OP_GRAD_VFD, 0, 0.5)
    # d/dx x = 1, d/dx y = 0, d/dx 1 = 0; a 1/delta (instead of 1/(2 delta)) reading would give 2
    assert abs(np.dot(w[0], rel[:, 0]) - 1.0) < 1e-12
    assert abs(np.dot(w[0], rel[:, 1])) < 1e-12
    assert abs(np.sum(w[0])) < 1e-12
    # x^2: the central difference of the interpolant is exact for quadratics -> 0 at x_c
    assert abs(np.dot(w[0], rel[:, 0] ** 2)) < 1e-11
    # on the plus stencil with m = 1 the VFD weights differ from the FD ones
    # only through the RBF part; both are antisymmetric in x
    rel5 = np.array([[0, 0], [1, 0], [-1, 0], [0, 1], [0, -1]], float)
    wv = O.stencil_weights(rel5, 3, 1, O.OP_GRAD_VFD, 0, 0.5)
    assert abs(wv[0][1] + wv[0][2]) < 1e-13 and abs(wv[0][0]) < 1e-13


def test_gepp_matches_lapack_and_residual():
    rng = np.random.default_rng(5)
    for K in (6, 18, 46, 85):
        A = rng.standard_normal((K, K))
        B = rng.standard_normal((K, 3))
        X = O.gepp(A, B)
        Xl = np.linalg.solve(A, B)
        assert np.allclose(X, Xl, rtol=1e-9, atol=1e-9)


def test_weights_solve_residual_vs_lapack():
    """The oracle weights equal LAPACK's solution of the same Eq. 9 system."""
    nodes = W.pec_box((14, 14), 0.25, 24)
    c = 100
    n, k, m = 30, 5, 4
    rel = _stencil(nodes, c, n)
    s = np.max(np.linalg.norm(rel, axis=1))
    z = rel / s
    E = _exps(2, m)
    Mm = len(E)
    A = np.zeros((n + Mm, n + Mm))
    r = np.linalg.norm(z[:, None, :] - z[None, :, :], axis=2)
    A[:n, :n] = r ** k
    P = np.stack([np.prod(z ** np.array(e), axis=1) for e in E], axis=1)
    A[:n, n:] = P
    A[n:, :n] = P.T
    rj = np.linalg.norm(z, axis=1)
    b = np.zeros(n + Mm)
    b[:n] = -k * rj ** (k - 2) * z[:, 0]
    b[n + E.index((1, 0))] = 1.0
    wl = np.linalg.solve(A, b)[:n] / s
    w = O.stencil_weights(rel, k, m, O.OP_GRAD)[0]
    assert np.max(np.abs(w - wl)) <= 1e-9 * np.max(np.abs(wl))


def test_rbf_fd_derivative_converges():
    """RBF-FD d/dx of sin on jittered stencils: error O(h^m) (Sec. 4.2, m + 1 - l = m)."""
    errs = []
    for h in (0.2, 0.1, 0.05):
        nodes = W.pec_box((11, 11), 0.25, 25)
        xyz = nodes.xyz * h
        c = 60
        idx = O.knn_brute(xyz[c:c + 1], xyz, nodes.period, 30)[0]
        rel = xyz[idx] - xyz[c]
        w = O.stencil_weights(rel, 5, 4, O.OP_GRAD)[0]
        f = np.sin(1.3 * xyz[idx, 0] + 0.7 * xyz[idx, 1])
        exact = 1.3 * math.cos(1.3 * xyz[c, 0] + 0.7 * xyz[c, 1])
        errs.append(abs(np.dot(w, f) - exact))
    rate = 0.5 * math.log2(errs[0] / errs[2])  # mean order over two halvings
    assert rate > 3.0, (errs, rate)
