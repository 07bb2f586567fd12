"""The dispersion analysis of Sec. 6 on the GPU (mfd_dispersion,
mfd_sim_dispersion) against the oracle's analysis of the same samples; the
host-only Yee phase speed (Eq. 6) against the oracle's."""
import math

import numpy as np
import pytest

import oracle as O
import oracle.dispersion as D
import workloads as W

M = pytest.importorskip("paper_2508_18205_gb300")


def test_fdtd_phase_speed_matches_oracle():
    """Host only (no GPU): Eq. 6 solved by the library and by the oracle."""
    for S in (0.2, 0.5, 1 / math.sqrt(2)):
        for phi in (0.0, 0.2, math.pi / 8, math.pi / 4, 1.1):
            for wdt in (0.01, 0.2, 0.5, 0.9, 1.4):
                a = M.fdtd_phase_speed(wdt, S, phi)
                b = D.fdtd_phase_speed(wdt, S, phi)
                if math.isnan(b):
                    assert math.isnan(a)
                else:
                    assert abs(a - b) <= 1e-12 * b, (S, phi, wdt, a, b)


def _compare(got, ref, clear=1e-9):
    spec, kidx, c, l1 = got
    rspec, ridx, rc, rl1 = ref
    scale = rspec.max()
    assert np.max(np.abs(spec - rspec)) <= 1e-11 * scale
    # the argmax is unique wherever the two largest entries of a row differ
    # by more than the transform's rounding; elsewhere either is right
    srt = np.sort(rspec, axis=1)
    if rspec.shape[1] == 1:
        sure = np.ones(rspec.shape[0], dtype=bool)
    else:
        sure = (srt[:, -1] - srt[:, -2]) > clear * scale
    assert np.array_equal(kidx[sure], ridx[sure])
    for j in np.nonzero(~sure)[0]:
        assert rspec[j, kidx[j]] >= srt[j, -1] - clear * scale
    same = sure & np.isfinite(rc)
    assert np.allclose(c[same], rc[same], rtol=1e-14, atol=0)
    if np.all(sure[1:]):
        assert l1 == rl1 if math.isinf(rl1) else l1 == pytest.approx(rl1, rel=1e-13)


@pytest.mark.gpu
@pytest.mark.parametrize("nt,nx", [(37, 50), (1, 9), (8, 1), (64, 4096), (4096, 24), (1250, 1000)])
def test_dispersion_matches_oracle(nt, nx):
    ctx = M.Ctx(0)
    rng = np.random.default_rng(nt * 7 + nx)
    # a travelling packet plus noise: a clear ridge and near-ties off it
    x = np.arange(nx)[None, :]
    t = np.arange(nt)[:, None]
    s = np.cos(0.3 * x - 0.11 * t) * np.exp(-((x - nx / 2 - 0.4 * t) / (nx / 6 + 1)) ** 2) + 0.05 * rng.standard_normal((nt, nx))
    h, dts, cref = 1.0, 4.0, 0.5
    jmax = min(45, nt - 1)
    got = M.dispersion(ctx, s, h, dts, cref, jmax)
    ref = D.dispersion(s, h, dts, cref, jmax)
    _compare(got, ref)


@pytest.mark.gpu
def test_dispersion_recovers_a_wave_speed():
    ctx = M.Ctx(0)
    nx, nt, h = 128, 90, 0.75
    i0, j0, v = 9, 11, 0.61
    k = 2 * math.pi * i0 / (nx * h)
    dt = 2 * math.pi * j0 / (nt * v * k)
    x = np.arange(nx)[None, :] * h
    tt = np.arange(nt)[:, None] * dt
    spec, kidx, c, l1 = M.dispersion(ctx, np.cos(k * x - v * k * tt), h, dt, v, 20)
    assert kidx[j0] == i0 and abs(c[j0] - v) < 1e-12
    assert math.isnan(c[0])


@pytest.mark.gpu
def test_dispersion_rejects_bad_sizes():
    ctx = M.Ctx(0)
    with pytest.raises(M.MfdError):
        M.dispersion(ctx, np.zeros((4, 4097)), 1.0, 1.0, 0.5, 2)
    with pytest.raises(M.MfdError):
        M.dispersion(ctx, np.zeros((4, 8)), 1.0, 1.0, 0.5, 4)
    with pytest.raises(M.MfdError):
        M.dispersion(ctx, np.zeros((4, 8)), 0.0, 1.0, 0.5, 2)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [M.MFD_FP64, M.MFD_FP32])
def test_sim_dispersion_of_probe_series(prec):
    """The analysis of a simulation's own probe buffer (no host round trip)
    equals the oracle's analysis of the same series read back, and in FP64
    the series itself is the oracle's run."""
    ctx = M.Ctx(0)
    nx, ny, S = 96, 24, 0.5
    dt, eps0, mu0, c0, eta0 = W.units(S)
    nodes = W.periodic_box((nx, ny), 0.25, 31, seed_line_y=ny // 2)
    nd = M.Nodes(ctx, nodes.xyz, nodes.period)
    st = M.Stencils(nd, nd, 31)
    cw = M.Weights(st, 12, 3, 2, M.MFD_OP_GRAD)
    hw = M.Weights(st, 31, 5, 4, M.MFD_OP_LAP_POW, 2)
    sim = M.Sim(ctx, 2, prec, dt, eps0, mu0, -4e-3, cw, hw, compensated=True)
    lam = 12.0
    ez, hx, hy = W.gaussian_pulse(nodes.xyz, nx, nx / 2, 2 * lam, c0, eta0, dt, lam)
    for comp, v in ((M.MFD_EZ, ez), (M.MFD_HX, hx), (M.MFD_HY, hy)):
        sim.set_field(comp, v)
    line = np.nonzero(np.abs(nodes.xyz[:, 1] - ny // 2) < 1e-12)[0]
    line = line[np.argsort(nodes.xyz[line, 0])]
    stride, nt = 4, 60
    sim.set_probes(line, stride * nt)
    sim.step(stride * nt)
    series = sim.read_probes()
    samples = series[stride - 1::stride]
    got = sim.dispersion(stride, nt, 1.0, c0, 20)
    _compare(got, D.dispersion(samples, 1.0, stride * dt, c0, 20))
    if prec == M.MFD_FP64:
        prob, _ = O.tmz_collocated(nodes, 12, 3, 2, 2, dt, eps0, mu0, -4e-3)
        ref = O.run_tmz(prob, ez, hx, hy, stride * nt, probes=line)[3]
        assert np.linalg.norm(series - ref) <= 1e-10 * np.linalg.norm(ref)
    with pytest.raises(M.MfdError):
        sim.dispersion(stride, nt + 1, 1.0, c0, 20)  # more samples than recorded steps
