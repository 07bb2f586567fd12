"""Parity at the benchmark's full size (pulse2d-staggered, 1000 x 1000 E nodes and
1000 x 1000 H nodes), in the launch configuration bench.py times.

The oracle cannot step 2M nodes in seconds, so it computes outputs one by one:
* kNN: the GPU stencils of sampled centres equal the oracle's (bit-exact).
* weights: the GPU weights of sampled centres match the oracle's (1e-8, as in
  the small-size tests).
* one leapfrog step from the GPU state after 70 steps: the new Ez at 48 sampled
  E nodes and the new H at 48 sampled H nodes (plus every H node the sampled
  E nodes depend on) match the oracle's step from the same state: relative L2
  over the sampled values 1e-12 in FP64, 1e-6 in FP32 (one step of FP32
  arithmetic and FP32-rounded weights).
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
    sim.step(70)
    s0 = [sim.get_field(c) for c in (M.MFD_EZ, M.MFD_HX, M.MFD_HY)]
    sim.step(1)
    s1 = [sim.get_field(c) for c in (M.MFD_EZ, M.MFD_HX, M.MFD_HY)]
    # sample where the pulse is (the fields are ~0 far from it)
    near_e = np.nonzero(np.abs(s0[0]) > 0.05)[0]
    near_h = np.nonzero(np.abs(s0[2]) > 0.05)[0]
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
