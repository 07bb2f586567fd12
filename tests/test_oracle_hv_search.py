"""Pins of the hyperviscosity search oracle: its interval logic against
synthetic stability maps with a known answer, and its runner against the
physics it relies on (energy growth without hyperviscosity, Appendix A)."""
import math

import numpy as np
import pytest

import oracle as O
import oracle.hv_search as S
import workloads as W


def _threshold_runner(t_lo, t_hi=math.inf):
    """Stable exactly on [t_lo, t_hi] (in log10 c)."""
    def run(lcs):
        return [(1.0 if t_lo <= lc <= t_hi else 5.0, 1.0) for lc in lcs]
    return run


@pytest.mark.parametrize("ncand,rounds", [(4, 3), (16, 2), (32, 1)])
def test_search_brackets_a_known_threshold(ncand, rounds):
    lo, hi, t = -6.0, -1.0, -3.2917
    c, hist = S.search(_threshold_runner(t), lo, hi, ncand, rounds, 0.01)
    width = (hi - lo) / ncand ** rounds
    assert t <= c < t + width + 1e-12
    assert len(hist) == rounds and all(len(h) == ncand for h in hist)
    assert hist[0][-1][0] == hi  # the last candidate of a round is the upper end


def test_search_finds_the_lower_edge_of_a_stable_window():
    """A coefficient too large is unstable too (the explicit HV step); the
    first stable candidate still marks the lower edge."""
    c, _ = S.search(_threshold_runner(-3.0, -1.5), -5.0, -1.6, 16, 3, 0.01)
    assert -3.0 <= c < -3.0 + 3.4 / 16 ** 3 + 1e-12


def test_search_reports_no_stable_candidate():
    c, hist = S.search(_threshold_runner(0.0), -5.0, -1.0, 8, 2, 0.01)
    assert math.isnan(c) and len(hist) == 1


def test_candidates_are_log_spaced_up_to_hi():
    assert S.candidates(-4.0, 0.0, 4) == [-3.0, -2.0, -1.0, 0.0]
    assert S.check_steps(250, 100) == [100, 200, 250]
    assert S.check_steps(200, 100) == [100, 200]


def test_tmz_runner_sees_growth_without_hyperviscosity_and_none_with_it():
    """At the paper's Courant number 1/(10 sqrt 2) (Sec. 6) on a jittered
    periodic layout (n = 30, PHS r^5, m = 4, alpha = 2, a sigma = 2 h pulse)
    the energy grows for a negligible coefficient (App. A: eigenvalues outside
    the unit circle on scattered nodes) and stays bounded, slightly
    dissipated, for c = 10^-2.5."""
    dt, eps0, mu0, c0, eta0 = W.units(1 / (10 * math.sqrt(2)))
    nodes = W.periodic_box((24, 24), 0.25, 41)
    prob, _ = O.tmz_collocated(nodes, 30, 5, 4, 2, dt, eps0, mu0, 0.0)
    ez, hx, hy = W.gaussian_pulse(nodes.xyz, 24, 12.0, 2.0, c0, eta0, dt, None)
    run = S.tmz_runner(prob, ez, hx, hy, 3000, 100, 2)
    (um_small, _), (um_ok, ue_ok) = run([-9.0, -2.5])
    assert um_small > 100.0
    assert um_ok <= 1.01 and 0.9 < ue_ok < 1.0
