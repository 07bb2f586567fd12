"""FP64 oracle of the hyperviscosity coefficient search (test
infrastructure only; the same import rule as the rest of ``oracle/``).

Sec. 5.1 shows that a usable coefficient c of gamma = c (-1)^(alpha-1)
h^(2 alpha) lies in an interval and that it is found by a search; Sec. 6 names
the search a bisection without giving its criterion. Reading taken: the
answer is the smallest stable c of [10^lo, 10^hi] (the least dissipative
stable choice), found by multisection on log10 c with ncand candidates per
round, log10 c_k = lo + (hi - lo) (k + 1) / ncand (the last one is hi); a
candidate is stable when u(t) = U(t)/U(0) of Eq. 20 stays <= 1 + tol and
finite at every check (every check_every steps and after the last step); the
next interval is [c_{k*-1}, c_{k*}] around the first stable candidate k*
(lo kept when k* = 0).

``search`` holds the logic and takes the candidate runner as an argument;
``tmz_runner`` runs each candidate with the oracle's leapfrog (``run_tmz``).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


def candidates(lo: float, hi: float, ncand: int):
    return [lo + (hi - lo) * (k + 1) / ncand for k in range(ncand)]


def search(run, lo: float, hi: float, ncand: int, rounds: int, tol: float):
    """run(list of log10 c) -> list of (max u, final u). Returns (log10 c of
    the answer, or nan when a round has no stable candidate; history)."""
    history = []
    for _ in range(rounds):
        lc = candidates(lo, hi, ncand)
        res = run(lc)
        history.append([(c, um, ue) for c, (um, ue) in zip(lc, res)])
        stable = [k for k, (um, _) in enumerate(res) if um <= 1.0 + tol]
        if not stable:
            return math.nan, history
        k = stable[0]
        lo, hi = (lc[k - 1] if k > 0 else lo), lc[k]
    return hi, history


def check_steps(nsteps: int, check_every: int):
    """The steps after which the energy is checked."""
    out = list(range(check_every, nsteps, check_every))
    out.append(nsteps)
    return out


def tmz_runner(prob, ez, hx, hy, nsteps: int, check_every: int, alpha: int):
    """Candidate runner over the oracle's TMz leapfrog: for each log10 c the
    whole run with gamma = c (-1)^(alpha-1); U(t) is Eq. 20 at step t
    (``run_tmz`` reports U at the start of every step, so it runs one step
    more than nsteps)."""
    from . import run_tmz
    sign = 1.0 if alpha % 2 == 1 else -1.0
    checks = check_steps(nsteps, check_every)

    def run(lcs):
        out = []
        for lc in lcs:
            p = dataclasses.replace(prob, gamma=sign * 10.0 ** lc)
            u = run_tmz(p, ez, hx, hy, nsteps + 1, energy=True)[4]
            r = np.array([u[t] / u[0] for t in checks])
            um = math.inf if np.any(~np.isfinite(r)) else max(1.0, float(r.max()))
            out.append((um, float(r[-1])))
        return out

    return run
