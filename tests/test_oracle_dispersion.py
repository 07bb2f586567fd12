"""Pins of the dispersion oracle (Sec. 6, Eqs. 24-26; Eq. 6 for the Yee
scheme) against definitions, closed forms and physics, not against itself."""
import cmath
import math

import numpy as np
import pytest

import oracle as O
import oracle.dispersion as D
import workloads as W


def test_hann_window_values():
    assert np.allclose(D.hann(5), [0.0, 0.5, 1.0, 0.5, 0.0], atol=1e-15)
    for nt in (3, 7, 64, 129):  # (N - 1) / 2 holds for N >= 3
        w = D.hann(nt)
        assert w[0] == 0.0 and abs(w[-1]) < 1e-15
        assert np.allclose(w, w[::-1], atol=1e-15)
        # sum of the symmetric Hann window = (N - 1) / 2
        assert abs(w.sum() - (nt - 1) / 2) < 1e-12
    assert D.hann(1)[0] == 1.0


def test_spectrum_is_the_written_out_double_sum():
    rng = np.random.default_rng(3)
    s = rng.standard_normal((5, 6))
    nt, nx = s.shape
    w = [0.5 - 0.5 * math.cos(2 * math.pi * n / (nt - 1)) for n in range(nt)]
    ref = np.zeros((nt, nx))
    for j in range(nt):
        for i in range(nx):
            acc = 0j
            for n in range(nt):
                for m in range(nx):
                    acc += w[n] * s[n, m] * cmath.exp(-2j * math.pi * i * m / nx) * cmath.exp(2j * math.pi * j * n / nt)
            ref[j, i] = abs(acc)
    assert np.allclose(D.spectrum(s), ref, rtol=1e-12, atol=1e-12)


def _wave(nx, nt, h, dt, k, omega):
    x = np.arange(nx) * h
    t = np.arange(nt) * dt
    return np.cos(k * x[None, :] - omega * t[:, None])


def test_travelling_wave_speed_is_recovered():
    """A wave of speed v = 0.37 whose wavenumber and frequency sit on the
    transform grid: the largest component of row j0 is column i0 and
    c(w_j0) = v (v enters only through the samples)."""
    nx, nt, h = 64, 50, 1.5
    i0, j0, v = 5, 7, 0.37
    k = 2 * math.pi * i0 / (nx * h)
    dt = 2 * math.pi * j0 / (nt * v * k)  # puts w0 = v k on bin j0
    s = _wave(nx, nt, h, dt, k, v * k)
    spec, idx, c, _ = D.dispersion(s, h, dt, v, 10)
    assert idx[j0] == i0
    assert abs(c[j0] - v) < 1e-12
    # nothing of comparable size elsewhere in that row
    row = np.sort(spec[j0])
    assert row[-2] < 0.1 * row[-1]


def test_left_moving_wave_lands_on_negative_wavenumbers():
    nx, nt, h, dt = 32, 40, 1.0, 1.0
    i0, j0 = 3, 4
    k = 2 * math.pi * i0 / nx
    om = 2 * math.pi * j0 / nt
    s = _wave(nx, nt, h, dt, -k, om)  # cos(-k x - w t): travels towards -x
    spec = D.spectrum(s)
    assert np.argmax(spec[j0]) == nx - i0


def test_parseval_and_constant_signal():
    rng = np.random.default_rng(4)
    s = rng.standard_normal((24, 30))
    spec = D.spectrum(s)
    ws = D.hann(24)[:, None] * s
    assert abs((spec ** 2).sum() - 24 * 30 * (ws ** 2).sum()) < 1e-9 * (spec ** 2).sum()
    # constant in space: only k = 0; at w = 0 the window's sum times N_x
    spec = D.spectrum(np.ones((9, 12)))
    assert abs(spec[0, 0] - 12 * (9 - 1) / 2) < 1e-12
    assert spec[:, 1:].max() < 1e-12


def test_err_l1_sums_from_j_1():
    c = np.array([math.nan, 0.5, 0.5, 0.7, 0.5])
    assert D.err_l1(c, 0.5, 3) == pytest.approx(0.2)
    assert D.err_l1(c, 0.5, 2) == 0.0
    spec = np.zeros((3, 4))
    spec[1, 0] = 1.0
    spec[2, 2] = 1.0
    idx, cc = D.phase_speed(spec, 1.0, 1.0)
    assert math.isnan(cc[0]) and cc[1] == math.inf and cc[2] == pytest.approx(2 * 4 / (2 * 3))


def test_fdtd_relation_closed_forms():
    """Eq. 6: along an axis k h = 2 asin(sin(w dt / 2) / S); along the
    diagonal at S = 1/sqrt(2) the Yee scheme has no dispersion (phase speed
    S h/dt at every w); for small w every angle tends to the physical speed.
    Phase speeds are in h per dt, where the physical one is S."""
    for S in (0.3, 0.5, 0.7):
        for wdt in (0.05, 0.3, 0.6):
            kh = D.fdtd_wavenumber(wdt, S, 0.0)
            assert abs(kh - 2 * math.asin(math.sin(wdt / 2) / S)) < 1e-12
    for wdt in (0.1, 0.5, 1.0, 1.5):
        assert abs(D.fdtd_phase_speed(wdt, 1 / math.sqrt(2), math.pi / 4) - 1 / math.sqrt(2)) < 1e-12
    for phi in (0.0, 0.3, math.pi / 4):
        c = D.fdtd_phase_speed(1e-4 * 0.5, 0.5, phi)  # omega dt small: c -> S = 0.5
        assert abs(c - 0.5) < 1e-8
    # above the cut-off there is no real wavenumber
    assert math.isnan(D.fdtd_wavenumber(2.0, 0.5, 0.0))


def test_phase_speed_of_an_oracle_run_is_near_c0():
    """Physics check of the whole analysis on the method itself: a
    Gaussian-modulated pulse (carrier 12 h, S = 0.5) on a periodic jittered
    192 x 32 layout with an equispaced seed line; at the carrier's frequency
    the largest component is the physical wavenumber to within one bin."""
    nx, ny = 192, 32
    S = 0.5
    dt, eps0, mu0, c0, eta0 = W.units(S)
    nodes = W.periodic_box((nx, ny), 0.25, 21, seed_line_y=ny // 2)
    prob, _ = O.tmz_collocated(nodes, 12, 3, 2, 2, dt, eps0, mu0, -4e-3)
    lam = 12.0
    ez, hx, hy = W.gaussian_pulse(nodes.xyz, nx, nx / 2, 2 * lam, c0, eta0, dt, lam)
    line = np.nonzero(np.abs(nodes.xyz[:, 1] - ny // 2) < 1e-12)[0]
    line = line[np.argsort(nodes.xyz[line, 0])]
    assert len(line) == nx
    stride, nt = 4, 120
    out = O.run_tmz(prob, ez, hx, hy, stride * nt, probes=line)
    samples = out[3][stride - 1::stride]  # Ez after steps stride, 2 stride, ...
    spec, idx, c, _ = D.dispersion(samples, 1.0, stride * dt, c0, 30)
    j0 = int(round(c0 * (2 * math.pi / lam) * nt * stride * dt / (2 * math.pi)))  # carrier bin
    i0 = nx / lam
    assert abs(idx[j0] - i0) <= 1
    assert abs(c[j0] - c0) / c0 < 0.07
