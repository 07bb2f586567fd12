"""FP64 oracle of the numerical-dispersion analysis of Sec. 6 (test
infrastructure only; the same import rule as the rest of ``oracle/``).

Field samples s[n][m] of Ez at N_x equispaced nodes of a line (spacing h_line
along it), taken every dt_sample time units (N_t samples), are windowed in
time with a Hann window and transformed in both directions (Sec. 6); the
numerical propagation velocity of each temporal frequency is read off the
largest spectral component (Eq. 24), compared with the physical speed
(Eq. 25) and summed into an l1 error (Eq. 26). numpy's FFT is the transform;
everything else is written out.

Readings (where Sec. 6 is silent):
* sign convention: E(k_i, w_j) = sum_n sum_m w_n s[n][m] exp(-i k_i x_m)
  exp(+i w_j t_n), so that a wave travelling towards +x appears at positive
  k and w (the paper's spectra show the physical branch w = c0 k);
* Hann window, symmetric form: w_n = 1/2 - 1/2 cos(2 pi n / (N_t - 1));
* k_i = 2 pi i / (N_x h_line), w_j = 2 pi j / (N_t dt_sample), argmax over
  0 <= i < N_x as printed (ties: smallest i);
* Eq. 26 starts at j = 0, where w_0 = 0 leaves c undefined: the sum runs over
  1 <= j <= j_max; c(w_0) is reported as NaN and a maximum at k_0 = 0 for
  j >= 1 gives c = +inf.
"""
from __future__ import annotations

import math

import numpy as np


def hann(nt: int) -> np.ndarray:
    """Symmetric Hann window of nt points (1 for a single point)."""
    if nt == 1:
        return np.ones(1)
    n = np.arange(nt, dtype=np.float64)
    return 0.5 - 0.5 * np.cos(2.0 * math.pi * n / (nt - 1))


def spectrum(samples) -> np.ndarray:
    """|E(k_i, w_j)| as an (N_t, N_x) array, row j, column i (Sec. 6)."""
    s = np.asarray(samples, dtype=np.float64)
    nt, nx = s.shape
    ws = hann(nt)[:, None] * s
    e = np.fft.fft(ws, axis=1)              # exp(-i k_i x_m) along the line
    e = np.fft.ifft(e, axis=0) * nt         # exp(+i w_j t_n) in time
    return np.abs(e)


def phase_speed(spec, h_line: float, dt_sample: float):
    """Eq. 24: i(j) = argmax_i |E(k_i, w_j)| and c(w_j) = w_j / k_{i(j)}."""
    spec = np.asarray(spec)
    nt, nx = spec.shape
    idx = np.argmax(spec, axis=1)  # first maximum: smallest i on ties
    c = np.empty(nt)
    for j in range(nt):
        if j == 0:
            c[j] = math.nan
        elif idx[j] == 0:
            c[j] = math.inf
        else:
            # w_j / k_i = (2 pi j / (N_t dt)) / (2 pi i / (N_x h))
            c[j] = (j * nx * h_line) / (idx[j] * nt * dt_sample)
    return idx, c


def err_l1(c, c_ref: float, jmax: int) -> float:
    """Eqs. 25-26 over 1 <= j <= jmax."""
    return float(sum(abs(c[j] - c_ref) for j in range(1, jmax + 1)))


def dispersion(samples, h_line: float, dt_sample: float, c_ref: float, jmax: int):
    """The whole analysis: (spectrum, i(j), c(w_j), ||err||_1)."""
    spec = spectrum(samples)
    idx, c = phase_speed(spec, h_line, dt_sample)
    return spec, idx, c, err_l1(c, c_ref, jmax)


def fdtd_wavenumber(omega_dt: float, courant: float, phi: float) -> float:
    """k h of the Yee scheme on a square grid (Eq. 6) for the angular
    frequency omega (omega_dt = omega dt), Courant number S = c dt / h and
    propagation angle phi: the root of
        sin^2(k h cos(phi) / 2) + sin^2(k h sin(phi) / 2) = sin^2(omega dt / 2) / S^2
    on the branch that starts at k = 0, found by bisection. Returns nan when
    omega lies above the grid's cut-off (no real root on that branch)."""
    rhs = math.sin(0.5 * omega_dt) ** 2 / courant ** 2
    cp, sp = math.cos(phi), math.sin(phi)

    def f(kh):
        return math.sin(0.5 * kh * cp) ** 2 + math.sin(0.5 * kh * sp) ** 2 - rhs

    # the left side grows monotonically from 0 up to kh = pi / max(|cos|, |sin|)
    hi = math.pi / max(abs(cp), abs(sp))
    if f(hi) < 0.0:
        return math.nan
    lo = 0.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) < 0.0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def fdtd_phase_speed(omega_dt: float, courant: float, phi: float) -> float:
    """Phase speed (in h per dt) of the Yee scheme at omega and angle phi (Eq. 6)."""
    kh = fdtd_wavenumber(omega_dt, courant, phi)
    return omega_dt / kh if kh > 0 else math.nan
