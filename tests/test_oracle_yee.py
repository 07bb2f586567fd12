"""Pins of the FDTD (Yee) oracle, Eq. 5, against the scheme's exact discrete
plane waves (whose frequency is the numerical dispersion relation Eq. 6) and
against a source whose first-step response is known in closed form."""
import math

import numpy as np
import pytest

import oracle as O
import oracle.dispersion as D
import workloads as W


def yee_plane_wave(nx, ny, p, q, S, eta0, n):
    """The discrete TMz plane wave of Eq. 5 with wavevector k = 2 pi (p / nx,
    q / ny) / h at step n (h = dt = 1): Ez = cos(theta), theta = kx i + ky j -
    w n, with w from Eq. 6 and the H amplitudes that the H update implies."""
    kx, ky = 2 * math.pi * p / nx, 2 * math.pi * q / ny
    w = 2 * math.asin(S * math.sqrt(math.sin(kx / 2) ** 2 + math.sin(ky / 2) ** 2))
    i = np.arange(nx)[None, :]
    j = np.arange(ny)[:, None]
    ez = np.cos(kx * i + ky * j - w * n)
    ax = (S / eta0) * math.sin(ky / 2) / math.sin(w / 2)
    ay = -(S / eta0) * math.sin(kx / 2) / math.sin(w / 2)
    hx = ax * np.cos(kx * i + ky * (j + 0.5) - w * (n - 0.5))
    hy = ay * np.cos(kx * (i + 0.5) + ky * j - w * (n - 0.5))
    return ez, hx, hy, w


@pytest.mark.parametrize("p,q,S", [(3, 0, 0.5), (2, 5, 0.6), (7, 7, 1 / math.sqrt(2)), (1, 2, 0.25)])
def test_discrete_plane_wave_propagates_exactly(p, q, S):
    nx, ny, steps = 40, 32, 300
    dt, eps0, mu0, c0, eta0 = W.units(S)
    ez, hx, hy, w = yee_plane_wave(nx, ny, p, q, S, eta0, 0)
    out = O.run_yee(nx, ny, dt / mu0, dt / eps0, dt, ez, hx, hy, steps)
    ez1, hx1, hy1, _ = yee_plane_wave(nx, ny, p, q, S, eta0, steps)
    for got, want in ((out[0], ez1), (out[1], hx1), (out[2], hy1)):
        assert np.max(np.abs(got - want)) < 1e-11 * max(1.0, np.max(np.abs(want)))
    # its phase speed is the one of Eq. 6 at the wave's angle
    phi = math.atan2(q / ny, p / nx)
    kh = 2 * math.pi * math.hypot(p / nx, q / ny)
    assert abs(w / kh - D.fdtd_phase_speed(w, S, phi)) < 1e-12


def test_first_step_of_a_soft_source():
    nx, ny, S = 16, 12, 0.5
    dt, eps0, mu0, c0, eta0 = W.units(S)
    z = np.zeros((ny, nx))
    src = W.Sources(node=np.array([5 * nx + 7]), rhs=np.zeros(1, np.int32), amp=np.array([2.0]),
                    f0=np.array([0.05]), t0=np.array([1.5 / 0.05]))
    ez, hx, hy, pr = O.run_yee(nx, ny, dt / mu0, dt / eps0, dt, z, z, z, 2, sources=src, probes=[5 * nx + 7, 5 * nx + 8])
    a = 2.0 * O.ricker(dt, 0.05, 30.0)
    assert pr[0, 0] == a and pr[0, 1] == 0.0
    # second step: the source cell's neighbours see the curl of the first kick
    assert pr[1, 1] == pytest.approx(dt / eps0 * (dt / mu0) * a, rel=1e-12)
