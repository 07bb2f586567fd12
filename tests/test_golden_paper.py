"""The oracle against values the paper prints (tests/golden/paper_values.json,
each entry with its passage)."""
import json
import math
import os

import numpy as np

import oracle as O
import oracle.dispersion as D
import workloads as W

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _yee_growth(S, steps=3000, n=16):
    """max |Ez| after `steps` steps of the oracle's Yee scheme from a random
    field (every grid mode present), relative to the start."""
    dt, eps0, mu0, c0, eta0 = W.units(S)
    rng = np.random.default_rng(1)
    f = [rng.standard_normal((n, n)) for _ in range(3)]
    ez = O.run_yee(n, n, dt / mu0, dt / eps0, dt, *f, steps)[0]
    return np.max(np.abs(ez)) / np.max(np.abs(f[0]))


def test_yee_stability_limit():
    """Sec. 3: the FDTD step is stable for S_c <= sqrt(2)/2 and not above."""
    lim = GOLDEN["yee_stability_limit"]["value"]
    assert abs(lim - math.sqrt(2) / 2) < 1e-15
    assert _yee_growth(0.98 * lim) < 10.0
    g = _yee_growth(1.02 * lim)
    assert not np.isfinite(g) or g > 1e6


def test_units_give_the_printed_speed_of_light():
    """Sec. 6 quotes c0 = 1/(10 sqrt 2) "in our units" with h = 1: with dt = 1
    the Courant number is c0 itself (the reading of the units)."""
    c0 = GOLDEN["c0_in_units"]["value"]
    dt, eps0, mu0, cc, eta0 = W.units(c0)
    assert dt == 1.0 and abs(cc - c0) < 1e-16 and abs(1 / math.sqrt(eps0 * mu0) - c0) < 1e-16


def test_section6_transform_grid():
    """Sec. 6: 2820 steps with every 15th snapshot give N_t = 188 samples of
    N_x = 200 line nodes; on exactly that grid the analysis (Eqs. 24-26)
    recovers waves travelling at c0 (on transform-grid wavenumbers) to within
    one wavenumber bin at their frequencies, up to j = 45."""
    g = GOLDEN["section6_transform"]
    nx, nt, every, jmax = g["N_x"], g["N_t"], g["every"], g["j_max"]
    assert nt * every == g["steps"]
    c0 = GOLDEN["c0_in_units"]["value"]
    x = np.arange(nx)[None, :] * g["h"]
    t = (np.arange(nt)[:, None]) * every
    # waves at speed c0 with wavenumbers on the transform grid; each one's
    # frequency falls in row j = round(c0 i N_t every / N_x) <= 45
    waves = list(range(4, 46, 8))
    s = sum(np.cos(2 * math.pi * i / nx * (x - c0 * t)) for i in waves)
    spec, idx, c, _ = D.dispersion(s, g["h"], float(every), c0, jmax)
    for i in waves:
        j = int(round(c0 * i * nt * every / nx))
        assert 1 <= j <= jmax
        assert abs(idx[j] - i) <= 1, (i, j, idx[j])
        assert abs(c[j] - c0) <= c0 / (i - 1)


def test_energy_band_is_the_search_default():
    """Sec. 6 keeps u(t) in [0.99, 1.01]; the coefficient search's default
    tolerance is that band's upper side."""
    import inspect
    band = GOLDEN["energy_band"]
    import paper_2508_18205_gb300 as M
    assert abs(inspect.signature(M.hv_search).parameters["tol"].default - (band["hi"] - 1.0)) < 1e-12
