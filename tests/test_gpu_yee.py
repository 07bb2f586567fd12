"""The FDTD (Yee) kernel (mfd_yee_*, Eq. 5) against the oracle's Yee scheme:
bit for bit in FP64 (the kernel follows the reference arithmetic term by
term), within FP32 rounding in FP32, with sources and probes, on ragged and
tiny grids and at the size the benchmark times."""
import math

import numpy as np
import pytest

import oracle as O
import oracle.dispersion as D
import workloads as W

pytestmark = pytest.mark.gpu
M = pytest.importorskip("paper_2508_18205_gb300")


def _fields(nx, ny, seed):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((ny, nx)) for _ in range(3)]


def _yee(ctx, nx, ny, prec, S, fields):
    dt, eps0, mu0, c0, eta0 = W.units(S)
    y = M.Yee(ctx, nx, ny, prec, dt, 1.0, eps0, mu0)
    for comp, v in zip((M.MFD_EZ, M.MFD_HX, M.MFD_HY), fields):
        y.set_field(comp, v)
    return y, dt, eps0, mu0


@pytest.mark.parametrize("nx,ny,steps", [(40, 32, 100), (10, 6, 67), (33, 17, 1), (64, 64, 130), (70, 45, 66)])
def test_yee_fp64_bit_exact(nx, ny, steps):
    """Ragged tiles (40 = 32 + 8), a grid smaller than one tile, one step,
    and runs long enough to replay the graph from both buffer parities."""
    ctx = M.Ctx(0)
    f = _fields(nx, ny, nx * ny)
    y, dt, eps0, mu0 = _yee(ctx, nx, ny, M.MFD_FP64, 0.5, f)
    y.step(3)
    y.step(steps)
    ref = O.run_yee(nx, ny, dt / mu0, dt / eps0, dt, *f, steps + 3)
    for comp, r in zip((M.MFD_EZ, M.MFD_HX, M.MFD_HY), ref[:3]):
        assert np.array_equal(y.get_field(comp), r), comp


def test_yee_fp32_and_sources_probes():
    ctx = M.Ctx(0)
    nx, ny, S, steps = 96, 40, 0.6, 300
    f = _fields(nx, ny, 3)
    src = W.Sources(node=np.array([5 * nx + 7, 20 * nx + 50, 5 * nx + 7]), rhs=np.zeros(3, np.int32),
                    amp=np.array([2.0, -1.0, 0.5]), f0=np.array([0.05, 0.04, 0.06]),
                    t0=np.array([30.0, 37.5, 25.0]))
    probes = np.array([0, 5 * nx + 8, ny * nx - 1, 20 * nx + 50])
    # FP32: the scheme neither damps nor amplifies its rounding errors, so they
    # may grow linearly: steps x 4 roundings x 2^-24 bounds the relative error
    f32 = [a.astype(np.float32).astype(np.float64) for a in f]
    for prec, tol, f0 in ((M.MFD_FP64, 1e-13, f), (M.MFD_FP32, steps * 4 * 2.0 ** -24, f32)):
        y, dt, eps0, mu0 = _yee(ctx, nx, ny, prec, S, f0)
        y.set_sources(src.node, src.amp, src.f0, src.t0)
        y.set_probes(probes, steps)
        y.step(steps)
        ez, hx, hy, pr = O.run_yee(nx, ny, dt / mu0, dt / eps0, dt, *f0, steps, sources=src, probes=probes)
        got = np.concatenate([y.get_field(c).ravel() for c in (M.MFD_EZ, M.MFD_HX, M.MFD_HY)])
        want = np.concatenate([ez.ravel(), hx.ravel(), hy.ravel()])
        assert np.linalg.norm(got - want) <= tol * np.linalg.norm(want), prec
        assert np.linalg.norm(y.read_probes() - pr) <= tol * np.linalg.norm(pr), prec


def test_yee_benchmark_size_fp32():
    """8192 x 8192 cells, the size the benchmark's roofline line uses: three
    steps against the oracle on every cell."""
    ctx = M.Ctx(0)
    nx = ny = 8192
    f = [a.astype(np.float32).astype(np.float64) for a in _fields(nx, ny, 9)]
    y, dt, eps0, mu0 = _yee(ctx, nx, ny, M.MFD_FP32, 0.5, f)
    y.step(3)
    ref = O.run_yee(nx, ny, dt / mu0, dt / eps0, dt, *f, 3)
    for comp, r in zip((M.MFD_EZ, M.MFD_HX, M.MFD_HY), ref[:3]):
        g = y.get_field(comp)
        assert np.linalg.norm(g - r) <= 1e-6 * np.linalg.norm(r), comp


def test_yee_dispersion_follows_eq6():
    """A modulated pulse along x on the Yee grid, analysed by mfd_dispersion:
    at the carrier the measured phase speed is the one Eq. 6 predicts, to
    within one wavenumber bin."""
    ctx = M.Ctx(0)
    nx, ny, S, lam = 240, 8, 0.5, 8.0
    dt, eps0, mu0, c0, eta0 = W.units(S)
    xy = np.stack(np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float)), -1).reshape(-1, 2)
    ez, _, _ = W.gaussian_pulse(xy, nx, nx / 2, 3 * lam, c0, eta0, dt, lam)
    hxy = xy + np.array([0.5, 0.0])  # Hy sits at (i + 1/2, j)
    _, _, hy = W.gaussian_pulse(hxy, nx, nx / 2, 3 * lam, c0, eta0, dt, lam)
    y, dt, eps0, mu0 = _yee(ctx, nx, ny, M.MFD_FP64, S, [ez.reshape(ny, nx), np.zeros((ny, nx)), hy.reshape(ny, nx)])
    stride, nt = 2, 600
    y.set_probes(np.arange(nx) + (ny // 2) * nx, stride * nt)
    y.step(stride * nt)
    samples = y.read_probes()[stride - 1::stride]
    spec, kidx, c, _ = M.dispersion(ctx, samples, 1.0, stride * dt, c0, 10)
    k0 = 2 * math.pi / lam
    w0 = 2 * math.asin(S * math.sin(k0 / 2))  # Eq. 6 at phi = 0, h = dt = 1
    j0 = int(round(w0 * nt * stride / (2 * math.pi)))
    assert abs(kidx[j0] - nx / lam) <= 1
    c_eq6 = D.fdtd_phase_speed(2 * math.pi * j0 / (nt * stride), S, 0.0)
    assert abs(c[j0] - c_eq6) <= c_eq6 / (nx / lam - 1)


def test_yee_tallest_grid_and_the_bound():
    """The tallest grid mfd_yee_create accepts (65535 rows of blocks of the
    four-step kernel's 28-row tiles, here two columns wide) steps bit for bit
    with the oracle through four-step launches; one row more is refused."""
    ctx = M.Ctx(0)
    nx, ny = 2, 65535 * 28
    f = _fields(nx, ny, 11)
    y, dt, eps0, mu0 = _yee(ctx, nx, ny, M.MFD_FP64, 0.5, f)
    y.step(8)
    ref = O.run_yee(nx, ny, dt / mu0, dt / eps0, dt, *f, 8)
    for comp, r in zip((M.MFD_EZ, M.MFD_HX, M.MFD_HY), ref[:3]):
        assert np.array_equal(y.get_field(comp), r), comp
    with pytest.raises(M.MfdError):
        M.Yee(ctx, nx, ny + 1, M.MFD_FP64, dt, 1.0, eps0, mu0)
