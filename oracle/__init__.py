"""FP64 CPU oracle of the meshless RBF leapfrog (test infrastructure only).

Only tests/, ``__graft_entry__.smoke()`` and bench.py's ``cpu_baseline`` /
``--impl reference`` legs may import this package. It never imports the CUDA
package and the CUDA package never imports it. The arithmetic lives in
``oracle.c`` (plain C, FP64, stencil sums in stencil order); this module only
marshals arrays and assembles problems from its functions. The dispersion
analysis of Sec. 6 is ``oracle/dispersion.py`` (numpy, with numpy's FFT as the
transform).

Pins that tie the oracle to the paper and to mathematics live in
``tests/test_oracle_*.py``. Every function here is pinned there.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")

OP_GRAD, OP_LAP_POW, OP_GRAD_VFD = 0, 1, 2


def build(force: bool = False) -> str:
    """Compiles oracle.c into oracle/_build/liboracle.so (gcc, FP64, no FMA contraction)."""
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
                           "-o", tmp, src, "-lm"])
    os.replace(tmp, _SO)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.orc_energy_tmz.restype = C.c_double
        _lib.orc_ricker.restype = C.c_double
        _lib.orc_ricker.argtypes = [C.c_double] * 3
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def _check(st, what):
    if st != 0:
        raise RuntimeError(f"oracle {what} failed with status {st}")


def threads(n: int = 0) -> int:
    """OpenMP threads of the oracle's parallel loops (OMP_NUM_THREADS, else all
    cores); n > 0 sets the count for the calls that follow."""
    return int(lib().orc_threads(int(n)))


# ------------------------------------------------------------------ O-1

def knn_brute(centres, sources, period, n):
    centres, sources = _f64(centres), _f64(sources)
    d = centres.shape[1]
    out = np.empty((centres.shape[0], n), dtype=np.int64)
    _check(lib().orc_knn_brute(C.c_int(d), C.c_int64(len(centres)), _p(centres),
                               C.c_int64(len(sources)), _p(sources), _p(_f64(period)),
                               C.c_int(n), _p(out)), "knn_brute")
    return out


def knn_cells(centres, sources, period, n, cell=1.0):
    centres, sources = _f64(centres), _f64(sources)
    d = centres.shape[1]
    out = np.empty((centres.shape[0], n), dtype=np.int64)
    _check(lib().orc_knn_cells(C.c_int(d), C.c_int64(len(centres)), _p(centres),
                               C.c_int64(len(sources)), _p(sources), _p(_f64(period)),
                               C.c_int(n), C.c_double(cell), _p(out)), "knn_cells")
    return out


def knn(centres, sources, period, n):
    """Brute force for small inputs, the cell list otherwise (same result)."""
    if len(centres) * len(sources) <= 4_000_000:
        return knn_brute(centres, sources, period, n)
    return knn_cells(centres, sources, period, n)


# ------------------------------------------------------------------ O-2

def monomials(dim, m):
    e = np.zeros((512, 3), dtype=np.int32)
    q = lib().orc_monomials(C.c_int(dim), C.c_int(m), _p(e))
    return e[:q, :dim].copy()


def stencil_weights(rel, phs_k, poly_m, op, alpha=0, delta=0.0):
    """Weights of one stencil from offsets rel (n x d) = x_j - x_c. Returns (nout, n)."""
    rel = _f64(rel)
    n, d = rel.shape
    nout = 1 if op == OP_LAP_POW else d
    w = np.empty((nout, n))
    _check(lib().orc_stencil_weights(C.c_int(d), C.c_int(n), _p(rel), C.c_int(phs_k),
                                     C.c_int(poly_m), C.c_int(op), C.c_int(alpha),
                                     C.c_double(delta), _p(w)), "stencil_weights")
    return w


def weights(xc, xs, period, idx, n_use, phs_k, poly_m, op, alpha=0, delta=0.0):
    """Weights for every centre on the first n_use entries of idx. Returns (nout, nc, n_use)."""
    xc, xs, idx = _f64(xc), _f64(xs), _i64(idx)
    nc, stride = idx.shape
    d = xc.shape[1]
    nout = 1 if op == OP_LAP_POW else d
    w = np.empty((nout, nc, n_use))
    _check(lib().orc_weights(C.c_int(d), C.c_int64(nc), _p(xc), _p(xs), _p(_f64(period)),
                             C.c_int(stride), C.c_int(n_use), _p(idx), C.c_int(phs_k),
                             C.c_int(poly_m), C.c_int(op), C.c_int(alpha), C.c_double(delta),
                             _p(w)), "weights")
    return w


def weights_sized(xc, xs, period, idx, n_per, phs_k, poly_m, op, alpha=0, delta=0.0):
    """Weights with a stencil size per centre: centre c uses the first n_per[c]
    entries of its row (Eq. 12 on that stencil). Rows are max(n_per) long,
    zero beyond each centre's own size (an entry with weight 0 is not in the
    stencil). Returns (nout, nc, max(n_per))."""
    xc, idx = _f64(xc), _i64(idx)
    n_per = _i64(n_per)
    nmax = int(n_per.max())
    d = xc.shape[1]
    nout = 1 if op == OP_LAP_POW else d
    w = np.zeros((nout, len(xc), nmax))
    for n_use in np.unique(n_per):
        sel = np.nonzero(n_per == n_use)[0]
        w[:, sel, :n_use] = weights(xc[sel], xs, period, idx[sel], int(n_use), phs_k, poly_m, op, alpha, delta)
    return w


def gepp(A, B):
    A = _f64(A).copy()
    B = _f64(B).reshape(A.shape[0], -1).copy()
    _check(lib().orc_gepp(C.c_int(A.shape[0]), _p(A), C.c_int(B.shape[1]), _p(B)), "gepp")
    return B


def ricker(t, f0, t0):
    return lib().orc_ricker(float(t), float(f0), float(t0))


# ------------------------------------------------------------------ problems

@dataclass
class Stencil:
    """Stencil of one operator family: idx (N x n, ids into the source set) and
    weights; code (N x n uint8, or None): image codes of the entries (PEC walls
    by images: bit a = the mirror image across the walls normal to axis a)."""

    idx: np.ndarray
    w: np.ndarray  # (nout, N, n)
    code: np.ndarray | None = None


@dataclass
class TMz:
    """A TMz problem: H node set, E node set (the same object when collocated)."""

    nh: int
    ne: int
    hc: Stencil  # H nodes <- E set, d/dx, d/dy
    hv: Stencil  # H nodes <- H set, Delta^alpha
    ec: Stencil  # E nodes <- H set, d/dx, d/dy
    ev: Stencil  # E nodes <- E set, Delta^alpha
    eps_r: np.ndarray
    pec: np.ndarray
    dt: float
    eps0: float
    mu0: float
    gamma: float


def _stencil(xc, xs, period, idx, n_use, phs_k, m, op, alpha=0, delta=0.0):
    idx = _i64(idx)
    w = weights(xc, xs, period, idx, n_use, phs_k, m, op, alpha, delta)
    return Stencil(idx=np.ascontiguousarray(idx[:, :n_use]), w=w)


def tmz_collocated(nodes, n, phs_k, m, alpha, dt, eps0, mu0, gamma, eps_r=None, vfd_delta=None,
                   nh_override=None):
    """Collocated TMz problem (the paper's layout): one kNN list serves both
    the curl stencil (its first n entries) and the HV stencil
    (n_HV = 2 M_{2 alpha} + 1 entries, PHS r^{2 alpha + 1}, monomials up to 2 alpha)."""
    import math
    d = nodes.dim
    nhv = nh_override or (2 * math.comb(2 * alpha + d, d) + 1)
    L = max(n, nhv)
    idx = knn(nodes.xyz, nodes.xyz, nodes.period, L)
    if vfd_delta is None:
        curl = _stencil(nodes.xyz, nodes.xyz, nodes.period, idx, n, phs_k, m, OP_GRAD)
    else:
        curl = _stencil(nodes.xyz, nodes.xyz, nodes.period, idx, n, phs_k, m, OP_GRAD_VFD, 0,
                        vfd_delta)
    hv = _stencil(nodes.xyz, nodes.xyz, nodes.period, idx, nhv, 2 * alpha + 1, 2 * alpha,
                  OP_LAP_POW, alpha)
    er = np.ones(nodes.n) if eps_r is None else _f64(eps_r)
    return TMz(nh=nodes.n, ne=nodes.n, hc=curl, hv=hv, ec=curl, ev=hv, eps_r=er,
               pec=np.ascontiguousarray(nodes.pec, dtype=np.uint8), dt=dt, eps0=eps0, mu0=mu0,
               gamma=gamma), idx


def tmz_staggered(e_nodes, h_nodes, n, phs_k, m, alpha, dt, eps0, mu0, gamma, eps_r=None):
    """Staggered TMz problem: curl stencils are the n nearest nodes of the other
    set; HV stencils are own-set (n_HV = 2 M_{2 alpha} + 1)."""
    import math
    d = e_nodes.dim
    nhv = 2 * math.comb(2 * alpha + d, d) + 1
    per = e_nodes.period
    i_he = knn(h_nodes.xyz, e_nodes.xyz, per, n)
    i_hh = knn(h_nodes.xyz, h_nodes.xyz, per, nhv)
    i_eh = knn(e_nodes.xyz, h_nodes.xyz, per, n)
    i_ee = knn(e_nodes.xyz, e_nodes.xyz, per, nhv)
    hc = _stencil(h_nodes.xyz, e_nodes.xyz, per, i_he, n, phs_k, m, OP_GRAD)
    hv = _stencil(h_nodes.xyz, h_nodes.xyz, per, i_hh, nhv, 2 * alpha + 1, 2 * alpha, OP_LAP_POW,
                  alpha)
    ec = _stencil(e_nodes.xyz, h_nodes.xyz, per, i_eh, n, phs_k, m, OP_GRAD)
    ev = _stencil(e_nodes.xyz, e_nodes.xyz, per, i_ee, nhv, 2 * alpha + 1, 2 * alpha, OP_LAP_POW,
                  alpha)
    er = np.ones(e_nodes.n) if eps_r is None else _f64(eps_r)
    return TMz(nh=h_nodes.n, ne=e_nodes.n, hc=hc, hv=hv, ec=ec, ev=ev, eps_r=er,
               pec=np.ascontiguousarray(e_nodes.pec, dtype=np.uint8), dt=dt, eps0=eps0, mu0=mu0,
               gamma=gamma)


def _tmz_args(p: TMz):
    hc, hv, ec, ev = p.hc, p.hv, p.ec, p.ev
    keep = []

    def st(s, k):
        a = np.ascontiguousarray(s.w[k])
        keep.append(a)
        return _p(a)

    args = [C.c_int64(p.nh), C.c_int(hc.idx.shape[1]), _p(hc.idx), st(hc, 0), st(hc, 1),
            C.c_int(hv.idx.shape[1]), _p(hv.idx), st(hv, 0),
            C.c_int64(p.ne), C.c_int(ec.idx.shape[1]), _p(ec.idx), st(ec, 0), st(ec, 1),
            C.c_int(ev.idx.shape[1]), _p(ev.idx), st(ev, 0),
            _p(p.eps_r), _p(p.pec), C.c_double(p.dt), C.c_double(p.eps0), C.c_double(p.mu0),
            C.c_double(p.gamma)]
    return args, keep


def run_tmz(p: TMz, ez, hx, hy, nsteps, step0=0, sources=None, probes=None, energy=False):
    """Runs nsteps of Eq. 19. Returns (ez, hx, hy, probe series (nsteps x P), energy or None)."""
    ez, hx, hy = _f64(ez).copy(), _f64(hx).copy(), _f64(hy).copy()
    args, keep = _tmz_args(p)
    if sources is None:
        sn = sa = sf = st0 = np.zeros(0)
        sn = np.zeros(0, np.int64)
    else:
        sn, sa, sf, st0 = _i64(sources.node), _f64(sources.amp), _f64(sources.f0), _f64(sources.t0)
    pr = np.zeros(0, np.int64) if probes is None else _i64(probes)
    pout = np.zeros((nsteps, len(pr)))
    eout = np.zeros(nsteps) if energy else None
    tail = [_p(ez), _p(hx), _p(hy), C.c_int64(step0), C.c_int64(nsteps), C.c_int(len(sn)), _p(sn), _p(sa),
            _p(sf), _p(st0), C.c_int(len(pr)), _p(pr), _p(pout), _p(eout)]
    if any(st.code is not None for st in (p.hc, p.hv, p.ec, p.ev)):
        codes = [None if st.code is None else np.ascontiguousarray(st.code, dtype=np.uint8)
                 for st in (p.hc, p.hv, p.ec, p.ev)]
        _check(lib().orc_run_tmz_img(*args, *tail, *[_p(c) for c in codes]), "run_tmz_img")
    else:
        _check(lib().orc_run_tmz(*args, *tail), "run_tmz")
    del keep
    return ez, hx, hy, pout, eout


def run_yee(nx, ny, ch, ce, dt, ez, hx, hy, nsteps, step0=0, sources=None, probes=None):
    """FDTD (Yee) TMz steps on a periodic nx x ny grid (Eq. 5); fields are
    (ny, nx) arrays (Ez at cell centres' nodes, Hx / Hy staggered, Eq. 4).
    Returns (ez, hx, hy, probe series (nsteps x P))."""
    ez, hx, hy = (np.ascontiguousarray(_f64(a).reshape(ny, nx)).copy() for a in (ez, hx, hy))
    if sources is None:
        sn, sa, sf, st0 = np.zeros(0, np.int64), np.zeros(0), np.zeros(0), np.zeros(0)
    else:
        sn, sa, sf, st0 = _i64(sources.node), _f64(sources.amp), _f64(sources.f0), _f64(sources.t0)
    pr = np.zeros(0, np.int64) if probes is None else _i64(probes)
    pout = np.zeros((nsteps, len(pr)))
    _check(lib().orc_run_yee(C.c_int64(nx), C.c_int64(ny), C.c_double(ch), C.c_double(ce), C.c_double(dt),
                             _p(ez), _p(hx), _p(hy), C.c_int64(step0), C.c_int64(nsteps), C.c_int(len(sn)),
                             _p(sn), _p(sa), _p(sf), _p(st0), C.c_int(len(pr)), _p(pr), _p(pout)), "run_yee")
    return ez, hx, hy, pout


def adjoint_step_tmz(p: TMz, lE, lHx, lHy):
    lE, lHx, lHy = _f64(lE).copy(), _f64(lHx).copy(), _f64(lHy).copy()
    args, keep = _tmz_args(p)
    _check(lib().orc_adjoint_step_tmz(*args, _p(lE), _p(lHx), _p(lHy)), "adjoint_step_tmz")
    del keep
    return lE, lHx, lHy


def grad_tmz(p: TMz, ez, hx, hy, nsteps, sources, probes):
    """J = dt sum_n sum_p Ez_p^2 and its gradient w.r.t. eps_r and source amplitudes."""
    args, keep = _tmz_args(p)
    ez, hx, hy = _f64(ez), _f64(hx), _f64(hy)
    sn, sa, sf, st0 = _i64(sources.node), _f64(sources.amp), _f64(sources.f0), _f64(sources.t0)
    pr = _i64(probes)
    J = C.c_double(0.0)
    ge = np.zeros(p.ne)
    ga = np.zeros(len(sn))
    _check(lib().orc_grad_tmz(*args, _p(ez), _p(hx), _p(hy), C.c_int64(nsteps), C.c_int(len(sn)),
                              _p(sn), _p(sa), _p(sf), _p(st0), C.c_int(len(pr)), _p(pr),
                              C.byref(J), _p(ge), _p(ga)), "grad_tmz")
    del keep
    return J.value, ge, ga


def energy_tmz(ez, eps_r, hxa, hya, hxb, hyb, eta0):
    ez, eps_r = _f64(ez), _f64(eps_r)
    hxa, hya, hxb, hyb = _f64(hxa), _f64(hya), _f64(hxb), _f64(hyb)
    return lib().orc_energy_tmz(C.c_int64(len(ez)), _p(ez), _p(eps_r), C.c_int64(len(hxa)),
                                _p(hxa), _p(hya), _p(hxb), _p(hyb), C.c_double(eta0))


@dataclass
class Max3D:
    """A collocated 3D problem."""

    n: int
    c: Stencil
    v: Stencil
    eps_r: np.ndarray
    wall: np.ndarray
    dt: float
    eps0: float
    mu0: float
    gamma: float


def max3d_collocated(nodes, n, phs_k, m, alpha, dt, eps0, mu0, gamma, eps_r=None, nh_override=None, n_per=None):
    """The 3D collocated problem; n_per: a curl stencil size per node (weights_sized) instead of n."""
    import math
    nhv = nh_override or (2 * math.comb(2 * alpha + 3, 3) + 1)
    L = max(n, nhv) if n_per is None else max(int(np.max(n_per)), nhv)
    idx = knn(nodes.xyz, nodes.xyz, nodes.period, L)
    if n_per is None:
        c = _stencil(nodes.xyz, nodes.xyz, nodes.period, idx, n, phs_k, m, OP_GRAD)
    else:
        w = weights_sized(nodes.xyz, nodes.xyz, nodes.period, idx, n_per, phs_k, m, OP_GRAD)
        c = Stencil(idx=np.ascontiguousarray(idx[:, :w.shape[2]]), w=w)
    v = _stencil(nodes.xyz, nodes.xyz, nodes.period, idx, nhv, 2 * alpha + 1, 2 * alpha,
                 OP_LAP_POW, alpha)
    er = np.ones(nodes.n) if eps_r is None else _f64(eps_r)
    return Max3D(n=nodes.n, c=c, v=v, eps_r=er,
                 wall=np.ascontiguousarray(nodes.normal_axes, dtype=np.uint8), dt=dt, eps0=eps0,
                 mu0=mu0, gamma=gamma), idx


def run_3d(p: Max3D, E, H, nsteps, step0=0, sources=None, probes=None, energy=False):
    """E, H: (3, N). Returns (E, H, probes, energy)."""
    E, H = _f64(E).copy(), _f64(H).copy()
    w = [np.ascontiguousarray(p.c.w[k]) for k in range(3)]
    wv = np.ascontiguousarray(p.v.w[0])
    if sources is None:
        sn = np.zeros(0, np.int64)
        sa = sf = st0 = np.zeros(0)
    else:
        sn, sa, sf, st0 = _i64(sources.node), _f64(sources.amp), _f64(sources.f0), _f64(sources.t0)
    pr = np.zeros(0, np.int64) if probes is None else _i64(probes)
    pout = np.zeros((nsteps, len(pr)))
    eout = np.zeros(nsteps) if energy else None
    args = [C.c_int64(p.n), C.c_int(p.c.idx.shape[1]), _p(p.c.idx), _p(w[0]), _p(w[1]), _p(w[2]),
            C.c_int(p.v.idx.shape[1]), _p(p.v.idx), _p(wv), _p(p.eps_r), _p(p.wall), C.c_double(p.dt),
            C.c_double(p.eps0), C.c_double(p.mu0), C.c_double(p.gamma), _p(E), _p(H), C.c_int64(step0),
            C.c_int64(nsteps), C.c_int(len(sn)), _p(sn), _p(sa), _p(sf), _p(st0), C.c_int(len(pr)), _p(pr),
            _p(pout), _p(eout)]
    if p.c.code is not None or p.v.code is not None:
        codes = [None if st.code is None else np.ascontiguousarray(st.code, dtype=np.uint8) for st in (p.c, p.v)]
        _check(lib().orc_run_3d_img(*args, *[_p(c) for c in codes]), "run_3d_img")
    else:
        _check(lib().orc_run_3d(*args), "run_3d")
    return E, H, pout, eout


def tmz_sample_step(e_nodes, h_nodes, e_ids, n, phs_k, m, alpha, dt, eps0, mu0, gamma, ez, hx, hy,
                    h_ids=(), collocated=False):
    """One Eq. 19 step evaluated at the E nodes e_ids (and H nodes h_ids) only.

    Builds the oracle's own stencils and weights for exactly the centres the
    result depends on (the sampled E nodes, the H nodes in their curl stencils
    and the sampled H nodes) by the cell-list kNN, then steps them.
    Returns (ez1 at e_ids, hx1 and hy1 at the H subset, the H subset ids).
    """
    import math
    d = e_nodes.dim
    nhv = 2 * math.comb(2 * alpha + d, d) + 1
    per = e_nodes.period
    e_ids = _i64(e_ids)
    xe = e_nodes.xyz[e_ids]
    L = max(n, nhv) if collocated else None
    if collocated:
        i_e = knn_cells(xe, e_nodes.xyz, per, L)
        ec_idx, ev_idx = i_e[:, :n], i_e[:, :nhv]
    else:
        ec_idx = knn_cells(xe, h_nodes.xyz, per, n)
        ev_idx = knn_cells(xe, e_nodes.xyz, per, nhv)
    hs = np.unique(np.concatenate([ec_idx.reshape(-1), _i64(h_ids)]))
    xh = h_nodes.xyz[hs]
    if collocated:
        i_h = knn_cells(xh, h_nodes.xyz, per, L)
        hc_idx, hv_idx = i_h[:, :n], i_h[:, :nhv]
    else:
        hc_idx = knn_cells(xh, e_nodes.xyz, per, n)
        hv_idx = knn_cells(xh, h_nodes.xyz, per, nhv)
    hc = weights(xh, e_nodes.xyz, per, hc_idx, n, phs_k, m, OP_GRAD)
    hv = weights(xh, h_nodes.xyz, per, hv_idx, nhv, 2 * alpha + 1, 2 * alpha, OP_LAP_POW, alpha)
    ec = weights(xe, h_nodes.xyz, per, ec_idx, n, phs_k, m, OP_GRAD)
    ev = weights(xe, e_nodes.xyz, per, ev_idx, nhv, 2 * alpha + 1, 2 * alpha, OP_LAP_POW, alpha)
    hpos = np.full(h_nodes.n, -1, dtype=np.int64)
    hpos[hs] = np.arange(len(hs))
    hx1 = np.empty(len(hs))
    hy1 = np.empty(len(hs))
    ez1 = np.empty(len(e_ids))
    c = [np.ascontiguousarray(a) for a in (hc_idx, hc[0], hc[1], hv_idx, hv[0], ec_idx, ec[0], ec[1],
                                           ev_idx, ev[0])]
    ez, hx, hy = _f64(ez), _f64(hx), _f64(hy)
    _check(lib().orc_tmz_sample_step(C.c_int64(len(hs)), _p(hs), C.c_int(n), _p(c[0]), _p(c[1]),
                                     _p(c[2]), C.c_int(nhv), _p(c[3]), _p(c[4]),
                                     C.c_int64(len(e_ids)), _p(e_ids), C.c_int(n), _p(c[5]),
                                     _p(c[6]), _p(c[7]), C.c_int(nhv), _p(c[8]), _p(c[9]), _p(hpos),
                                     None, C.c_double(dt), C.c_double(eps0), C.c_double(mu0),
                                     C.c_double(gamma), _p(ez), _p(hx), _p(hy), _p(hx1), _p(hy1),
                                     _p(ez1)), "tmz_sample_step")
    return ez1, hx1, hy1, hs


def max3d_sample_step(nodes, e_ids, n, phs_k, m, alpha, dt, eps0, mu0, gamma, E, H, eps_r=None, h_ids=()):
    """One 3D collocated step evaluated at the nodes e_ids (E') and at the H nodes
    they depend on plus h_ids (H'), with the oracle's own stencils and weights
    for exactly those centres. Returns (E1 (3 x len(e_ids)), H1 (3 x nhs), H subset ids)."""
    import math
    nhv = 2 * math.comb(2 * alpha + 3, 3) + 1
    L = max(n, nhv)
    per = nodes.period
    e_ids = _i64(e_ids)
    ie = knn_cells(nodes.xyz[e_ids], nodes.xyz, per, L)
    hs = np.unique(np.concatenate([ie[:, :n].reshape(-1), _i64(h_ids)]))
    ih = knn_cells(nodes.xyz[hs], nodes.xyz, per, L)

    def w(xc, idx):
        c = weights(xc, nodes.xyz, per, idx, n, phs_k, m, OP_GRAD)
        v = weights(xc, nodes.xyz, per, idx, nhv, 2 * alpha + 1, 2 * alpha, OP_LAP_POW, alpha)
        return c, v

    hc, hv = w(nodes.xyz[hs], ih)
    ec, ev = w(nodes.xyz[e_ids], ie)
    hpos = np.full(nodes.n, -1, dtype=np.int64)
    hpos[hs] = np.arange(len(hs))
    arr = [np.ascontiguousarray(a) for a in (ih[:, :n], hc[0], hc[1], hc[2], ih[:, :nhv], hv[0],
                                             ie[:, :n], ec[0], ec[1], ec[2], ie[:, :nhv], ev[0])]
    er = None if eps_r is None else _f64(np.asarray(eps_r)[e_ids])
    wall = np.ascontiguousarray(nodes.normal_axes[e_ids], dtype=np.uint8)
    E, H = _f64(E), _f64(H)
    H1 = np.empty((3, len(hs)))
    E1 = np.empty((3, len(e_ids)))
    _check(lib().orc_3d_sample_step(C.c_int64(len(hs)), _p(hs), C.c_int(n), _p(arr[0]), _p(arr[1]), _p(arr[2]),
                                    _p(arr[3]), C.c_int(nhv), _p(arr[4]), _p(arr[5]), C.c_int64(len(e_ids)),
                                    _p(e_ids), _p(arr[6]), _p(arr[7]), _p(arr[8]), _p(arr[9]), _p(arr[10]),
                                    _p(arr[11]), _p(hpos), _p(er), _p(wall), C.c_int64(nodes.n),
                                    C.c_double(dt), C.c_double(eps0), C.c_double(mu0), C.c_double(gamma),
                                    _p(E), _p(H), _p(H1), _p(E1)), "3d_sample_step")
    return E1, H1, hs


# ------------------------------------------------------------------ PEC walls by images

def mirror_doubled(nodes, axes=None):
    """The PEC box as a periodic box of twice its size (image theory of a perfect
    conductor): every node of `nodes` (a pec_box on [0, L] per axis) and, for
    every non-empty subset r of the mirrored axes (bit a = axis a), its image
    with x_a -> 2 L - x_a for a in r, skipping the images that fall on the node
    itself (a wall node is its own image). The period is 2 L on the mirrored
    axes. Nodes come first in their own order, then the images by (r, node id).
    Returns (NodeSet of the doubled box, orig (node id of each entry), code (r of
    each entry))."""
    import workloads as W
    d = nodes.dim
    L = np.asarray(nodes.box_hi, dtype=np.float64) - np.asarray(nodes.box_lo, dtype=np.float64)
    if axes is None:
        axes = (1 << d) - 1
    x = _f64(nodes.xyz)
    n = len(x)
    pts, orig, code = [x], [np.arange(n)], [np.zeros(n, np.int64)]
    for r in range(1, 1 << d):
        if r & ~axes:
            continue
        keep = np.ones(n, bool)
        y = x.copy()
        for a in range(d):
            if (r >> a) & 1:
                keep &= (x[:, a] > 0.0) & (x[:, a] < L[a])
                y[:, a] = 2.0 * L[a] - x[:, a]
        pts.append(y[keep])
        orig.append(np.nonzero(keep)[0])
        code.append(np.full(int(keep.sum()), r, np.int64))
    per = np.array([2.0 * L[a] if (axes >> a) & 1 else 0.0 for a in range(d)])
    xyz = np.concatenate(pts)
    # no component is held at the walls: the mirror symmetry of the extension is
    # the boundary condition (holding the tangential E of the wall nodes at 0 on
    # top of it makes the scheme grow)
    ns = W.NodeSet(xyz=xyz, pec=np.zeros(len(xyz), np.uint8), period=per, box_lo=np.zeros(d),
                   box_hi=np.where(per > 0, per, L), normal_axes=np.zeros(len(xyz), np.uint8))
    return ns, np.concatenate(orig), np.concatenate(code)


def image_sign_tmz(code, comp):
    """Sign of an image of TMz field `comp` ('ez', 'hx', 'hy') across the walls of
    code r: Ez is tangential to every wall (odd across each), Hx normal to the x
    walls (odd across them, even across the y walls), Hy normal to the y walls."""
    code = np.asarray(code)
    if comp == "ez":
        k = (code & 1) + ((code >> 1) & 1)
    elif comp == "hx":
        k = code & 1
    else:
        k = (code >> 1) & 1
    return 1.0 - 2.0 * (k & 1)


def image_sign_3d(code, field, b):
    """Sign of an image of component b of E or H across the walls of code r:
    E_b is odd across every wall it is tangential to (axes a != b), H_b across
    the wall it is normal to (axis b)."""
    code = np.asarray(code)
    if field == "e":
        m = code & ~(1 << b) & 7
        k = (m & 1) + ((m >> 1) & 1) + ((m >> 2) & 1)
    else:
        k = (code >> b) & 1
    return 1.0 - 2.0 * (k & 1)


def image_stencils(nodes, L_use):
    """The L_use nearest of every node of a PEC box among the nodes and their
    mirror images (the doubled box of mirror_doubled). Returns (doubled box,
    ids into it, node id and image code of every doubled entry)."""
    dbl, orig, code = mirror_doubled(nodes)
    ids = knn(nodes.xyz, dbl.xyz, dbl.period, L_use)
    return dbl, ids, orig, code


def _image_stencil(nodes, dbl, ids, orig, code, n_use, phs_k, m, op, alpha=0, n_per=None):
    if n_per is None:
        w = weights(nodes.xyz, dbl.xyz, dbl.period, ids, n_use, phs_k, m, op, alpha)
    else:
        w = weights_sized(nodes.xyz, dbl.xyz, dbl.period, ids, n_per, phs_k, m, op, alpha)
        n_use = w.shape[2]
    sub = ids[:, :n_use]
    return Stencil(idx=np.ascontiguousarray(orig[sub]), w=w, code=np.ascontiguousarray(code[sub], dtype=np.uint8))


def wall_sizes(nodes, n, n_wall, band=1.0):
    """Stencil size per node of a PEC box: n_wall for the nodes closer than
    `band` to a wall (the layer next to the walls), n elsewhere. Next to a
    mirror plane the n nearest of the nodes and their images are a set with
    mirror-paired nodes, and at n = 2 M_m (the fewest the rule of Sec. 4.1
    allows) some of these stencils give the collocated curl an eigenvalue
    with a large positive real part that the hyperviscosity does not
    outweigh; a few more nodes in that layer remove it."""
    x = _f64(nodes.xyz)
    lo = np.asarray(nodes.box_lo, dtype=np.float64)
    hi = np.asarray(nodes.box_hi, dtype=np.float64)
    dw = np.minimum(x - lo, hi - x).min(axis=1)
    return np.where(dw < band, n_wall, n).astype(np.int64)


def tmz_images(nodes, n, phs_k, m, alpha, dt, eps0, mu0, gamma, eps_r=None, nh_override=None):
    """Collocated TMz problem of a PEC box with image stencils: every stencil
    entry is a node of the box or its mirror image (node id and code); the
    weights are those of the image positions; no component is held at the
    walls (the symmetry is the boundary condition)."""
    import math
    nhv = nh_override or (2 * math.comb(2 * alpha + 2, 2) + 1)
    dbl, ids, orig, code = image_stencils(nodes, max(n, nhv))
    curl = _image_stencil(nodes, dbl, ids, orig, code, n, phs_k, m, OP_GRAD)
    hv = _image_stencil(nodes, dbl, ids, orig, code, nhv, 2 * alpha + 1, 2 * alpha, OP_LAP_POW, alpha)
    er = np.ones(nodes.n) if eps_r is None else _f64(eps_r)
    return TMz(nh=nodes.n, ne=nodes.n, hc=curl, hv=hv, ec=curl, ev=hv, eps_r=er,
               pec=np.zeros(nodes.n, np.uint8), dt=dt, eps0=eps0, mu0=mu0, gamma=gamma)


def max3d_images(nodes, n, phs_k, m, alpha, dt, eps0, mu0, gamma, eps_r=None, nh_override=None, n_wall=None,
                 wall_band=1.0):
    """The 3D collocated problem of a PEC box with image stencils (see
    tmz_images). With n_wall, the curl stencils of the nodes closer than
    wall_band to a wall take n_wall entries (wall_sizes)."""
    import math
    nhv = nh_override or (2 * math.comb(2 * alpha + 3, 3) + 1)
    n_per = None if n_wall is None else wall_sizes(nodes, n, n_wall, wall_band)
    dbl, ids, orig, code = image_stencils(nodes, max(n, nhv, n_wall or 0))
    c = _image_stencil(nodes, dbl, ids, orig, code, n, phs_k, m, OP_GRAD, n_per=n_per)
    v = _image_stencil(nodes, dbl, ids, orig, code, nhv, 2 * alpha + 1, 2 * alpha, OP_LAP_POW, alpha)
    er = np.ones(nodes.n) if eps_r is None else _f64(eps_r)
    return Max3D(n=nodes.n, c=c, v=v, eps_r=er, wall=np.zeros(nodes.n, np.uint8), dt=dt, eps0=eps0, mu0=mu0,
                 gamma=gamma)


def run_tmz_images(nodes, n, phs_k, m, alpha, dt, eps0, mu0, gamma, ez, hx, hy, nsteps, eps_r=None,
                   sources=None, probes=None, energy=False, nh_override=None):
    """Eq. 19 on a PEC box with image stencils (tmz_images): (ez, hx, hy, probes, energy)."""
    prob = tmz_images(nodes, n, phs_k, m, alpha, dt, eps0, mu0, gamma, eps_r, nh_override)
    return run_tmz(prob, ez, hx, hy, nsteps, sources=sources, probes=probes, energy=energy)


def run_3d_images(nodes, n, phs_k, m, alpha, dt, eps0, mu0, gamma, E, H, nsteps, eps_r=None, energy=False,
                  nh_override=None, n_wall=None, wall_band=1.0):
    """The 3D step on a PEC box with image stencils (max3d_images): (E, H, energy)."""
    prob = max3d_images(nodes, n, phs_k, m, alpha, dt, eps0, mu0, gamma, eps_r, nh_override, n_wall, wall_band)
    E1, H1, _, en = run_3d(prob, E, H, nsteps, energy=energy)
    return E1, H1, en
