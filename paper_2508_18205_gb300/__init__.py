"""Python binding of libmfd (include/mfd.h): the GB300 meshless RBF-FD Maxwell leapfrog.

Argument marshalling only: every step of the method (Morton reordering, kNN
stencils, weight solves, the fused leapfrog half steps, sources, probes,
energy) runs in the CUDA library. The functions mirror the C ABI names
(``mfd_nodes_create`` ...); the small classes below own the handles.

The library must be built (``paper_2508_18205_gb300.build.build()``); there
is no fallback: importing the handles without the built library, or using them
without a CUDA device, raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# MFD_LIB selects another build of the library (the bounds-checked one of build.build(bounds=True))
LIB_PATH = os.environ.get("MFD_LIB") or os.path.join(_HERE, "_build", "libmfd.so")

MFD_OK = 0
MFD_ERR_ARG, MFD_ERR_OOM, MFD_ERR_CUDA, MFD_ERR_SINGULAR = -1, -2, -3, -4
MFD_ERR_UNSTABLE, MFD_ERR_TIMEOUT, MFD_ERR_STATE = -5, -6, -7
MFD_OP_GRAD, MFD_OP_LAP_POW, MFD_OP_GRAD_VFD = 0, 1, 2
MFD_FP32, MFD_FP64 = 0, 1
MFD_INDEX_Q16, MFD_INDEX_I32 = 0, 1
MFD_EX, MFD_EY, MFD_EZ, MFD_HX, MFD_HY, MFD_HZ = range(6)
MFD_BUILD_BOUNDS_CHECK = 1


class MfdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"mfd status {status}: {msg}")
        self.status = status


class mfd_sim_desc(C.Structure):
    _fields_ = [("dim", C.c_int), ("precision", C.c_int), ("nrhs", C.c_int), ("compensated", C.c_int),
                ("dt", C.c_double), ("eps0", C.c_double), ("mu0", C.c_double), ("gamma", C.c_double),
                ("h_curl", C.c_void_p), ("h_hv", C.c_void_p), ("e_curl", C.c_void_p), ("e_hv", C.c_void_p)]


_VP, _I, _I64, _D = C.c_void_p, C.c_int, C.c_int64, C.c_double
_SIGS = {
    "mfd_last_error": (C.c_char_p, []),
    "mfd_version": (C.c_int, []),
    "mfd_ctx_create": (_I, [_I, _VP, C.POINTER(_VP)]),
    "mfd_ctx_stream": (_VP, [_VP]),
    "mfd_ctx_sync": (_I, [_VP]),
    "mfd_ctx_destroy": (None, [_VP]),
    "mfd_nodes_create": (_I, [_VP, _I, _I64, _VP, _VP, C.POINTER(_VP)]),
    "mfd_nodes_count": (_I64, [_VP]),
    "mfd_nodes_permutation": (_I, [_VP, _VP]),
    "mfd_nodes_destroy": (None, [_VP]),
    "mfd_stencils_build": (_I, [_VP, _VP, _I, C.POINTER(_VP)]),
    "mfd_stencils_read": (_I, [_VP, _VP]),
    "mfd_stencils_destroy": (None, [_VP]),
    "mfd_weights_compute": (_I, [_VP, _I, _I, _I, _I, _I, _D, C.POINTER(_VP)]),
    "mfd_weights_compute_sized": (_I, [_VP, _VP, _I, _I, _I, _I, _D, C.POINTER(_VP)]),
    "mfd_weights_read": (_I, [_VP, _VP]),
    "mfd_weights_destroy": (None, [_VP]),
    "mfd_sim_create": (_I, [_VP, C.POINTER(mfd_sim_desc), C.POINTER(_VP)]),
    "mfd_set_materials": (_I, [_VP, _VP, _VP]),
    "mfd_set_field": (_I, [_VP, _I, _I, _VP]),
    "mfd_get_field": (_I, [_VP, _I, _I, _VP]),
    "mfd_set_field_device": (_I, [_VP, _I, _I, _VP, _VP]),
    "mfd_get_field_device": (_I, [_VP, _I, _I, _VP, _VP]),
    "mfd_set_sources": (_I, [_VP, _I, _VP, _VP, _VP, _VP, _VP]),
    "mfd_set_probes": (_I, [_VP, _I, _VP, _I64]),
    "mfd_step": (_I, [_VP, _I64]),
    "mfd_step_timed": (_I, [_VP, _I64, _VP]),
    "mfd_read_probes": (_I, [_VP, _VP, C.POINTER(_I64)]),
    "mfd_energy": (_I, [_VP, _VP]),
    "mfd_sim_steps": (_I64, [_VP]),
    "mfd_grad": (_I, [_VP, _I64, _I64, _VP, _VP, _VP]),
    "mfd_fma_peak": (_I, [_I, _VP, _VP]),
    "mfd_sim_set_blocks": (_I, [_VP, _I, _I]),
    "mfd_set_watchdog": (_I, [_VP, _I64, _D]),
    "mfd_sim_autotune": (_I, [_VP, _I, _VP]),
    "mfd_sim_launch_config": (_I, [_VP, _VP, _VP]),
    "mfd_sim_set_lanes": (_I, [_VP, _I, _I]),
    "mfd_set_probe_component": (_I, [_VP, _I]),
    "mfd_sim_set_index_format": (_I, [_VP, _I]),
    "mfd_sim_index_stats": (_I, [_VP, _VP]),
    "mfd_sim_set_l2_keep": (_I, [_VP, _D]),
    "mfd_sim_l2_keep": (_D, [_VP]),
    "mfd_sim_destroy": (None, [_VP]),
    "mfd_knn_static": (_I, [_I, _I64, _VP, _I64, _VP, _VP, _I, _VP, _VP]),
    "mfd_yee_create": (_I, [_VP, _I64, _I64, _I, _D, _D, _D, _D, C.POINTER(_VP)]),
    "mfd_yee_set_field": (_I, [_VP, _I, _VP]),
    "mfd_yee_get_field": (_I, [_VP, _I, _VP]),
    "mfd_yee_set_sources": (_I, [_VP, _I, _VP, _VP, _VP, _VP]),
    "mfd_yee_set_probes": (_I, [_VP, _I, _VP, _I64]),
    "mfd_yee_step": (_I, [_VP, _I64]),
    "mfd_yee_step_timed": (_I, [_VP, _I64, _VP]),
    "mfd_yee_read_probes": (_I, [_VP, _VP, C.POINTER(_I64)]),
    "mfd_yee_steps_per_launch": (_I, [_VP]),
    "mfd_yee_destroy": (None, [_VP]),
    "mfd_dispersion": (_I, [_VP, _I, _I, _VP, _D, _D, _D, _I, _VP, _VP, _VP, _VP]),
    "mfd_sim_dispersion": (_I, [_VP, _I, _I, _D, _D, _I, _VP, _VP, _VP, _VP]),
    "mfd_fdtd_phase_speed": (_I, [_D, _D, _D, _VP]),
    "mfd_partition_create": (_I, [_I64, _VP, _I, C.POINTER(_VP)]),
    "mfd_partition_owner": (_I, [_VP, _VP]),
    "mfd_partition_owned": (_I, [_VP, _I, C.POINTER(_I64), _VP]),
    "mfd_partition_destroy": (None, [_VP]),
    "mfd_halo_create": (_I, [_VP, _I, _VP, _VP, _VP, C.POINTER(_VP)]),
    "mfd_halo_nodes": (_I, [_VP, _I, C.POINTER(_I64), _VP]),
    "mfd_halo_send": (_I, [_VP, _I, _I, C.POINTER(_I64), _VP]),
    "mfd_halo_local_idx": (_I, [_VP, _I, _I, _VP]),
    "mfd_halo_destroy": (None, [_VP]),
    "mfd_batch_create": (_I, [_VP, _I, _VP, _I, C.POINTER(_VP)]),
    "mfd_batch_set_materials": (_I, [_VP, _I, _VP, _VP]),
    "mfd_batch_set_field": (_I, [_VP, _I, _I, _I, _VP]),
    "mfd_batch_get_field": (_I, [_VP, _I, _I, _I, _VP]),
    "mfd_batch_set_field_device": (_I, [_VP, _I, _I, _I, _VP, _VP]),
    "mfd_batch_get_field_device": (_I, [_VP, _I, _I, _I, _VP, _VP]),
    "mfd_batch_set_sources": (_I, [_VP, _I, _I, _VP, _VP, _VP, _VP, _VP]),
    "mfd_batch_set_probes": (_I, [_VP, _I, _I, _VP, _I64]),
    "mfd_batch_step": (_I, [_VP, _I64]),
    "mfd_batch_read_probes": (_I, [_VP, _I, _VP, C.POINTER(_I64)]),
    "mfd_batch_nodes": (_I64, [_VP]),
    "mfd_batch_uses_graph": (_I, [_VP]),
    "mfd_batch_set_gamma": (_I, [_VP, _I, _VP]),
    "mfd_batch_energy": (_I, [_VP, _I, _VP]),
    "mfd_batch_destroy": (None, [_VP]),
    "mfd_batch_set_spin_limit": (_I, [_VP, C.c_uint64]),
    "mfd_batch_set_variant": (_I, [_VP, _I]),
    "mfd_batch_variant": (_I, [_VP]),
    "mfd_batch_autotune": (_I, [_VP, _I, _VP, _VP]),
    "mfd_build_flags": (_I, []),
    "mfd_nodes_set_mirror": (_I, [_VP, C.c_uint32, _VP]),
    "mfd_grad_forward": (_I, [_VP, _I64, _I64, _VP, _VP]),
    "mfd_grad_backward": (_I, [_VP, _VP, _VP, _I, _VP]),
    "mfd_tape_destroy": (None, [_VP]),
    "mfd_probe_objective": (_I, [_VP, _VP]),
    "mfd_sim_adjoint_sweeps": (_I64, [_VP]),
    "mfd_set_materials_device": (_I, [_VP, _VP, _VP, _VP]),
    "mfd_set_source_amps_device": (_I, [_VP, _VP, _VP]),
    "mfd_sim_state_size": (_I, [_VP, _VP]),
    "mfd_sim_save_state": (_I, [_VP, _VP, C.c_size_t]),
    "mfd_sim_load_state": (_I, [_VP, _VP, C.c_size_t]),
    "mfd_batch_state_size": (_I, [_VP, _VP]),
    "mfd_batch_save_state": (_I, [_VP, _VP, C.c_size_t]),
    "mfd_batch_load_state": (_I, [_VP, _VP, C.c_size_t]),
    "mfd_debug_fail_alloc": (_I, [_I64]),
    "mfd_debug_alloc_pending": (_I64, []),
    "mfd_hv_search": (_I, [_VP, _VP, _VP, _D, _D, _D, _VP, _VP, _VP, _VP, _VP, _D, _D, _I, _I, _I64, _I64, _D, _VP,
                           _VP]),
}

_lib = None


def lib():
    """The loaded libmfd (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libmfd is not built ({LIB_PATH}); run paper_2508_18205_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _ck(status):
    if status != MFD_OK:
        raise MfdError(status, lib().mfd_last_error().decode())


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _is_cuda_tensor(a):
    return getattr(a, "is_cuda", False) and hasattr(a, "data_ptr")


def _dev_ptr(t):
    """Device pointer of a contiguous torch CUDA FP64 tensor (raises otherwise)."""
    import torch
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError("device field buffers are contiguous float64 CUDA tensors")
    return C.c_void_p(t.data_ptr())


def _torch_stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dispersion_out(nt, nx, want_spectrum):
    spec = np.empty((nt, nx)) if want_spectrum else None
    return spec, np.empty(nt, dtype=np.int32), np.empty(nt), np.zeros(1)


def dispersion(ctx, samples, h_line, dt_sample, c_ref, jmax, spectrum=True):
    """Numerical dispersion of line samples (mfd_dispersion, Sec. 6, Eqs. 24-26):
    (spectrum |E(k_i, w_j)| or None, argmax index i(j), c(w_j), ||err||_1)."""
    s = _f64(samples)
    nt, nx = s.shape
    spec, kidx, c, l1 = _dispersion_out(nt, nx, spectrum)
    _ck(lib().mfd_dispersion(ctx.h, nx, nt, _p(s), float(h_line), float(dt_sample), float(c_ref), int(jmax),
                             _p(spec), _p(kidx), _p(c), _p(l1)))
    return spec, kidx, c, float(l1[0])


def hv_search(ctx, curl, hv, dt, eps0, mu0, ez, hx, hy, log10_lo, log10_hi, ncand=16, rounds=2, nsteps=2000,
              check_every=100, tol=0.01, eps_r=None, pec=None):
    """Smallest stable hyperviscosity coefficient c by multisection (mfd_hv_search).
    Returns (c, history[rounds][ncand][3] = (log10 c, max u, final u)); raises
    MfdError (MFD_ERR_UNSTABLE) when a round has no stable candidate."""
    er = None if eps_r is None else _f64(eps_r)
    pc = None if pec is None else np.ascontiguousarray(pec, dtype=np.uint8)
    hist = np.full((rounds, ncand, 3), np.nan)
    c = np.zeros(1)
    _ck(lib().mfd_hv_search(ctx.h, curl.h, hv.h, float(dt), float(eps0), float(mu0), _p(er), _p(pc), _p(_f64(ez)),
                            _p(_f64(hx)), _p(_f64(hy)), float(log10_lo), float(log10_hi), int(ncand), int(rounds),
                            int(nsteps), int(check_every), float(tol), _p(c), _p(hist)))
    return float(c[0]), hist


# TEz mode (Sec. 2: TEz is TMz with the roles of E and H interchanged). The
# TMz step advances (Hx, Hy) at half steps with dt/mu0 and Ez at whole steps
# with dt/(eps0 eps_r); under (Ez, Hx, Hy, eps0, mu0) <- (Hz, -Ex, -Ey, mu0, eps0)
# the same step advances TEz: (Ex, Ey) at half steps with dt/eps0 and Hz at
# whole steps with dt/(mu0 mu_r). So a Sim or Yee created with the constants
# tez_constants(eps0, mu0) steps TEz fields stored through tez_set / tez_get;
# its per-node material (set_materials) is then mu_r, the permittivity is
# uniform, and a wall held at zero holds Hz (a magnetic wall).
TEZ_FIELDS = {"Hz": (MFD_EZ, 1.0), "Ex": (MFD_HX, -1.0), "Ey": (MFD_HY, -1.0)}


def tez_constants(eps0, mu0):
    """(eps0, mu0) to create a TMz Sim or Yee that steps the TEz mode."""
    return mu0, eps0


def tez_set(obj, name, values):
    """Sets TEz field `name` ("Hz", "Ex" or "Ey") of a Sim or Yee created with tez_constants."""
    comp, sign = TEZ_FIELDS[name]
    obj.set_field(comp, sign * np.asarray(values, dtype=np.float64))


def tez_get(obj, name):
    comp, sign = TEZ_FIELDS[name]
    return sign * obj.get_field(comp)


def fdtd_phase_speed(omega_dt, courant, phi):
    """Phase speed of the Yee scheme in h per dt (mfd_fdtd_phase_speed, Eq. 6)."""
    c = np.zeros(1)
    _ck(lib().mfd_fdtd_phase_speed(float(omega_dt), float(courant), float(phi), _p(c)))
    return float(c[0])


def _save_state(size_fn, save_fn, h):
    n = C.c_size_t(0)
    _ck(size_fn(h, C.byref(n)))
    buf = C.create_string_buffer(n.value)
    _ck(save_fn(h, buf, n.value))
    return buf.raw


def debug_fail_alloc(after):
    """Makes the device allocation after the next `after` ones fail with MFD_ERR_OOM (-1: off)."""
    _ck(lib().mfd_debug_fail_alloc(int(after)))


def debug_alloc_pending():
    """Allocations left before the injected failure fires (-1: none pending)."""
    return int(lib().mfd_debug_alloc_pending())


def fma_peak(device=0):
    """(FP64, FP32) FMA throughput of the device in GFLOP/s (mfd_fma_peak)."""
    a, b = np.zeros(1), np.zeros(1)
    _ck(lib().mfd_fma_peak(device, _p(a), _p(b)))
    return float(a[0]), float(b[0])


# ------------------------------------------------------------------ handles

class Ctx:
    """A library context on CUDA device `device` (its own non-blocking stream unless one is given)."""

    def __init__(self, device: int = 0, stream: int | None = None):
        h = C.c_void_p()
        _ck(lib().mfd_ctx_create(device, stream, C.byref(h)))
        self.h = h
        self.device = device

    @property
    def stream(self) -> int:
        return lib().mfd_ctx_stream(self.h) or 0

    def torch_stream(self):
        import torch
        return torch.cuda.ExternalStream(self.stream, device=f"cuda:{self.device}")

    def sync(self):
        _ck(lib().mfd_ctx_sync(self.h))

    def close(self):
        if self.h:
            lib().mfd_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Nodes:
    def __init__(self, ctx: Ctx, xyz, period=None):
        xyz = _f64(xyz)
        n, dim = xyz.shape
        per = _f64(np.zeros(dim) if period is None else period)
        h = C.c_void_p()
        _ck(lib().mfd_nodes_create(ctx.h, dim, n, _p(xyz), _p(per), C.byref(h)))
        self.h, self.ctx, self.n, self.dim = h, ctx, n, dim

    def set_mirror(self, axes, hi):
        """PEC walls by images at 0 and hi[a] on the axes of bit mask `axes` (mfd_nodes_set_mirror)."""
        h = _f64(hi)
        _ck(lib().mfd_nodes_set_mirror(self.h, int(axes), _p(h)))

    def permutation(self):
        out = np.empty(self.n, dtype=np.int64)
        _ck(lib().mfd_nodes_permutation(self.h, _p(out)))
        return out

    def __del__(self):
        try:
            if self.h:
                lib().mfd_nodes_destroy(self.h)
                self.h = None
        except Exception:
            pass


class Stencils:
    def __init__(self, centres: Nodes, sources: Nodes, n: int):
        h = C.c_void_p()
        _ck(lib().mfd_stencils_build(centres.h, sources.h, n, C.byref(h)))
        self.h, self.centres, self.sources, self.n = h, centres, sources, n

    def read(self):
        out = np.empty((self.centres.n, self.n), dtype=np.int64)
        _ck(lib().mfd_stencils_read(self.h, _p(out)))
        return out

    def __del__(self):
        try:
            if self.h:
                lib().mfd_stencils_destroy(self.h)
                self.h = None
        except Exception:
            pass


def wall_layer_sizes(xyz, box_lo, box_hi, n, n_wall, band=1.0):
    """Stencil size per node for mfd_weights_compute_sized: n_wall for the nodes
    closer than `band` to a face of the box [box_lo, box_hi] (the layer next to
    mirror walls), n elsewhere."""
    x = np.asarray(xyz, dtype=np.float64)
    d = np.minimum(x - np.asarray(box_lo, dtype=np.float64), np.asarray(box_hi, dtype=np.float64) - x).min(axis=1)
    return np.where(d < band, int(n_wall), int(n)).astype(np.int32)


class Weights:
    """Stencil weights (mfd_weights_compute). n_use: one stencil size, or an
    array with the size of every centre (caller order;
    mfd_weights_compute_sized), the rows then being max(n_use) long."""

    def __init__(self, st: Stencils, n_use, phs_k: int, poly_m: int, op: int, alpha: int = 0,
                 delta: float = 0.0):
        h = C.c_void_p()
        if np.ndim(n_use) == 0:
            _ck(lib().mfd_weights_compute(st.h, int(n_use), phs_k, poly_m, op, alpha, float(delta), C.byref(h)))
            n = int(n_use)
        else:
            sizes = np.ascontiguousarray(n_use, dtype=np.int32)
            if sizes.shape != (st.centres.n,):
                raise ValueError("one stencil size per centre expected")
            _ck(lib().mfd_weights_compute_sized(st.h, _p(sizes), phs_k, poly_m, op, alpha, float(delta),
                                                C.byref(h)))
            n = int(sizes.max()) if sizes.size else 1
        self.h, self.st, self.n_use, self.op = h, st, n, op
        self.nout = 1 if op == MFD_OP_LAP_POW else st.centres.dim

    def read(self):
        out = np.empty((self.nout, self.st.centres.n, self.n_use))
        _ck(lib().mfd_weights_read(self.h, _p(out)))
        return out

    def __del__(self):
        try:
            if self.h:
                lib().mfd_weights_destroy(self.h)
                self.h = None
        except Exception:
            pass


class Yee:
    """FDTD (Yee) TMz on a periodic nx x ny grid (mfd_yee_*, Eq. 5)."""

    def __init__(self, ctx: Ctx, nx, ny, precision, dt, h, eps0, mu0):
        hd = C.c_void_p()
        _ck(lib().mfd_yee_create(ctx.h, int(nx), int(ny), precision, float(dt), float(h), float(eps0), float(mu0),
                                 C.byref(hd)))
        self.h, self.ctx, self.nx, self.ny, self.nprobe = hd, ctx, int(nx), int(ny), 0

    def set_field(self, comp, values):
        v = _f64(values).reshape(self.ny, self.nx)
        _ck(lib().mfd_yee_set_field(self.h, comp, _p(np.ascontiguousarray(v))))

    def get_field(self, comp):
        out = np.empty((self.ny, self.nx))
        _ck(lib().mfd_yee_get_field(self.h, comp, _p(out)))
        return out

    def set_sources(self, cell, amp, f0, t0):
        cell = np.ascontiguousarray(cell, dtype=np.int64)
        _ck(lib().mfd_yee_set_sources(self.h, len(cell), _p(cell), _p(_f64(amp)), _p(_f64(f0)), _p(_f64(t0))))

    def set_probes(self, cell, capacity):
        cell = np.ascontiguousarray(cell, dtype=np.int64)
        _ck(lib().mfd_yee_set_probes(self.h, len(cell), _p(cell), int(capacity)))
        self.nprobe = len(cell)

    def step(self, n):
        _ck(lib().mfd_yee_step(self.h, int(n)))

    def step_timed(self, n):
        ms = np.zeros(1)
        _ck(lib().mfd_yee_step_timed(self.h, int(n), _p(ms)))
        return float(ms[0])

    @property
    def steps_per_launch(self):
        return int(lib().mfd_yee_steps_per_launch(self.h))

    def read_probes(self):
        steps = C.c_int64(0)
        _ck(lib().mfd_yee_read_probes(self.h, None, C.byref(steps)))
        out = np.zeros((steps.value, self.nprobe))
        if steps.value and self.nprobe:
            _ck(lib().mfd_yee_read_probes(self.h, _p(out), C.byref(steps)))
        return out

    def __del__(self):
        try:
            if self.h:
                lib().mfd_yee_destroy(self.h)
                self.h = None
        except Exception:
            pass


class Partition:
    """A node set of n nodes cut into nshards contiguous ranges of `order`
    (mfd_partition_create; host only, no GPU needed)."""

    def __init__(self, n: int, nshards: int, order=None):
        o = None if order is None else np.ascontiguousarray(order, dtype=np.int64)
        if o is not None and o.shape != (n,):
            raise ValueError("order must hold n caller ids")
        h = C.c_void_p()
        _ck(lib().mfd_partition_create(int(n), _p(o), int(nshards), C.byref(h)))
        self.h, self.n, self.nshards = h, int(n), int(nshards)

    def owner(self):
        out = np.empty(self.n, dtype=np.int32)
        _ck(lib().mfd_partition_owner(self.h, _p(out)))
        return out

    def owned(self, shard: int):
        c = C.c_int64()
        _ck(lib().mfd_partition_owned(self.h, shard, C.byref(c), None))
        out = np.empty(c.value, dtype=np.int64)
        _ck(lib().mfd_partition_owned(self.h, shard, C.byref(c), _p(out)))
        return out

    def __del__(self):
        try:
            if self.h:
                lib().mfd_partition_destroy(self.h)
                self.h = None
        except Exception:
            pass


class HaloPlan:
    """Halo plan of one source set for the stencil sets that read it
    (mfd_halo_create). sets: sequence of (centre Partition, idx [rows][ncols]
    caller ids into the source set)."""

    def __init__(self, src: Partition, sets):
        parts = [c for c, _ in sets]
        idxs = [np.ascontiguousarray(i, dtype=np.int64) for _, i in sets]
        for c, i in zip(parts, idxs):
            if i.ndim != 2 or i.shape[0] != c.n:
                raise ValueError("each stencil set needs idx of shape (centres, ncols)")
        cp = (C.c_void_p * len(sets))(*[c.h.value for c in parts])
        nc = (C.c_int * len(sets))(*[i.shape[1] for i in idxs])
        ip = (C.c_void_p * len(sets))(*[i.ctypes.data for i in idxs])
        h = C.c_void_p()
        _ck(lib().mfd_halo_create(src.h, len(sets), C.cast(cp, C.c_void_p), C.cast(nc, C.c_void_p),
                                  C.cast(ip, C.c_void_p), C.byref(h)))
        self.h, self.src, self.parts = h, src, parts
        self.ncols = [i.shape[1] for i in idxs]

    def nodes(self, shard: int):
        c = C.c_int64()
        _ck(lib().mfd_halo_nodes(self.h, shard, C.byref(c), None))
        out = np.empty(c.value, dtype=np.int64)
        _ck(lib().mfd_halo_nodes(self.h, shard, C.byref(c), _p(out)))
        return out

    def send(self, frm: int, to: int):
        c = C.c_int64()
        _ck(lib().mfd_halo_send(self.h, frm, to, C.byref(c), None))
        out = np.empty(c.value, dtype=np.int64)
        _ck(lib().mfd_halo_send(self.h, frm, to, C.byref(c), _p(out)))
        return out

    def local_idx(self, shard: int, k: int):
        rows = len(self.parts[k].owned(shard))
        out = np.empty((rows, self.ncols[k]), dtype=np.int32)
        _ck(lib().mfd_halo_local_idx(self.h, shard, k, _p(out)))
        return out

    def __del__(self):
        try:
            if self.h:
                lib().mfd_halo_destroy(self.h)
                self.h = None
        except Exception:
            pass


class Sim:
    """A stepped problem (see mfd_sim_desc in include/mfd.h)."""

    def __init__(self, ctx: Ctx, dim, precision, dt, eps0, mu0, gamma, h_curl: Weights, h_hv: Weights,
                 e_curl: Weights = None, e_hv: Weights = None, compensated=False, nrhs=1):
        e_curl = e_curl or h_curl
        e_hv = e_hv or h_hv
        d = mfd_sim_desc(dim, precision, nrhs, int(bool(compensated)), dt, eps0, mu0, gamma,
                         h_curl.h, h_hv.h, e_curl.h, e_hv.h)
        h = C.c_void_p()
        _ck(lib().mfd_sim_create(ctx.h, C.byref(d), C.byref(h)))
        self.h, self.ctx = h, ctx
        self._keep = (h_curl, h_hv, e_curl, e_hv)
        self.ne = e_curl.st.centres.n
        self.nh = h_curl.st.centres.n
        self.nprobe = 0

    def set_materials(self, eps_r=None, pec=None):
        er = None if eps_r is None else _f64(eps_r)
        pc = None if pec is None else np.ascontiguousarray(pec, dtype=np.uint8)
        _ck(lib().mfd_set_materials(self.h, _p(er), _p(pc)))

    def set_field(self, comp, values, rhs=0):
        if _is_cuda_tensor(values):  # zero copy: torch CUDA FP64 tensor on the current stream
            _ck(lib().mfd_set_field_device(self.h, comp, rhs, _dev_ptr(values), _torch_stream()))
            return
        _ck(lib().mfd_set_field(self.h, comp, rhs, _p(_f64(values))))

    def get_field(self, comp, rhs=0, out=None):
        """Host FP64 array, or, with `out` a torch CUDA FP64 tensor, into it (zero copy)."""
        if out is not None and _is_cuda_tensor(out):
            _ck(lib().mfd_get_field_device(self.h, comp, rhs, _dev_ptr(out), _torch_stream()))
            return out
        n = self.ne if comp <= MFD_EZ else self.nh
        out = np.empty(n)
        _ck(lib().mfd_get_field(self.h, comp, rhs, _p(out)))
        return out

    def set_sources(self, node, amp, f0, t0, rhs=None):
        node = np.ascontiguousarray(node, dtype=np.int64)
        r = None if rhs is None else np.ascontiguousarray(rhs, dtype=np.int32)
        _ck(lib().mfd_set_sources(self.h, len(node), _p(node), _p(r), _p(_f64(amp)), _p(_f64(f0)),
                                  _p(_f64(t0))))

    def set_probes(self, node, capacity):
        node = np.ascontiguousarray(node, dtype=np.int64)
        _ck(lib().mfd_set_probes(self.h, len(node), _p(node), int(capacity)))
        self.nprobe = len(node)

    def step(self, n):
        _ck(lib().mfd_step(self.h, int(n)))

    def step_timed(self, n):
        ms = np.zeros(2)
        _ck(lib().mfd_step_timed(self.h, int(n), _p(ms)))
        return ms

    def read_probes(self):
        steps = C.c_int64(0)
        _ck(lib().mfd_read_probes(self.h, None, C.byref(steps)))
        out = np.zeros((steps.value, self.nprobe))
        if steps.value and self.nprobe:
            _ck(lib().mfd_read_probes(self.h, _p(out), C.byref(steps)))
        return out

    def energy(self):
        u = np.zeros(1)
        _ck(lib().mfd_energy(self.h, _p(u)))
        return float(u[0])

    def dispersion(self, stride, nt, h_line, c_ref, jmax, spectrum=True):
        """mfd_sim_dispersion: the analysis of the probe series (probes = the line)."""
        spec, kidx, c, l1 = _dispersion_out(nt, self.nprobe, spectrum)
        _ck(lib().mfd_sim_dispersion(self.h, int(stride), int(nt), float(h_line), float(c_ref), int(jmax),
                                     _p(spec), _p(kidx), _p(c), _p(l1)))
        return spec, kidx, c, float(l1[0])

    @property
    def adjoint_sweeps(self):
        """Adjoint sweeps this simulation has run (mfd_sim_adjoint_sweeps)."""
        return int(lib().mfd_sim_adjoint_sweeps(self.h))

    @property
    def steps(self):
        return int(lib().mfd_sim_steps(self.h))

    def set_watchdog(self, every, max_ratio=1.5):
        _ck(lib().mfd_set_watchdog(self.h, int(every), float(max_ratio)))

    def set_blocks(self, block_h, block_e):
        _ck(lib().mfd_sim_set_blocks(self.h, int(block_h), int(block_e)))

    def set_l2_keep(self, keep):
        """Fraction of the stencil streams' L2 lines kept from step to step (mfd_sim_set_l2_keep);
        negative: sized from the device's L2."""
        _ck(lib().mfd_sim_set_l2_keep(self.h, float(keep)))

    @property
    def l2_keep(self):
        """The fraction the step kernels use (mfd_sim_l2_keep)."""
        return float(lib().mfd_sim_l2_keep(self.h))

    def set_index_format(self, fmt):
        """MFD_INDEX_Q16 (default) or MFD_INDEX_I32 indices in the staggered kernels (mfd_sim_set_index_format)."""
        _ck(lib().mfd_sim_set_index_format(self.h, int(fmt)))

    def index_stats(self):
        """{"h"|"e": (slices, 32-bit curl slices, 32-bit HV slices)} (mfd_sim_index_stats)."""
        out = np.zeros(6, dtype=np.int64)
        _ck(lib().mfd_sim_index_stats(self.h, _p(out)))
        return {"h": tuple(int(x) for x in out[:3]), "e": tuple(int(x) for x in out[3:])}

    def autotune(self, reps=20):
        """Times 64/128/256/512 threads per block (and, collocated 2D, 1/2/4 threads
        per node) for each half-step kernel and keeps the fastest: the blocks."""
        ch = np.zeros(2, dtype=np.int32)
        _ck(lib().mfd_sim_autotune(self.h, int(reps), _p(ch)))
        return int(ch[0]), int(ch[1])

    def set_probe_component(self, comp):
        """The component the probes record (mfd_set_probe_component; MFD_EZ by default)."""
        _ck(lib().mfd_set_probe_component(self.h, int(comp)))

    def set_lanes(self, lanes_h, lanes_e):
        """Threads per node of the H and E passes (collocated 2D, mfd_sim_set_lanes)."""
        _ck(lib().mfd_sim_set_lanes(self.h, int(lanes_h), int(lanes_e)))

    def launch_config(self):
        """((block H, block E), (lanes H, lanes E)) in use (mfd_sim_launch_config)."""
        b = np.zeros(2, dtype=np.int32)
        ln = np.zeros(2, dtype=np.int32)
        _ck(lib().mfd_sim_launch_config(self.h, _p(b), _p(ln)))
        return (int(b[0]), int(b[1])), (int(ln[0]), int(ln[1]))

    def save_state(self):
        """Checkpoint of the fields, the step index and the probe records (bytes, mfd_sim_save_state)."""
        return _save_state(lib().mfd_sim_state_size, lib().mfd_sim_save_state, self.h)

    def load_state(self, blob):
        """Resumes from a checkpoint of save_state (a simulation built the same way)."""
        _ck(lib().mfd_sim_load_state(self.h, blob, len(blob)))

    def grad(self, nsteps, every=0, nsrc=0):
        """(J, dJ/deps_r per E node, dJ/d amplitude per source) over the next nsteps (mfd_grad)."""
        J = np.zeros(1)
        ge = np.zeros(self.ne)
        ga = np.zeros(max(nsrc, 1))
        _ck(lib().mfd_grad(self.h, int(nsteps), int(every), _p(J), _p(ge), _p(ga)))
        return float(J[0]), ge, ga[:nsrc]

    def __del__(self):
        try:
            if self.h:
                lib().mfd_sim_destroy(self.h)
                self.h = None
        except Exception:
            pass


class Batch:
    """Many collocated TMz domains x nrhs right-hand sides, stepped by one persistent kernel."""

    def __init__(self, ctx: Ctx, domains, nrhs=16):
        """domains: list of (curl Weights, hv Weights, dt, eps0, mu0, gamma)."""
        descs = (mfd_sim_desc * len(domains))()
        for d, (cw, hw, dt, eps0, mu0, gamma) in enumerate(domains):
            descs[d] = mfd_sim_desc(2, MFD_FP32, nrhs, 0, dt, eps0, mu0, gamma, cw.h, hw.h, cw.h, hw.h)
        h = C.c_void_p()
        _ck(lib().mfd_batch_create(ctx.h, len(domains), C.cast(descs, C.c_void_p), nrhs, C.byref(h)))
        self.h, self.ctx, self.nrhs = h, ctx, nrhs
        self._keep = list(domains)
        self.n = [cw.st.centres.n for cw, *_ in domains]
        self.nprobe = [0] * len(domains)

    def set_materials(self, dom, eps_r=None, pec=None):
        er = None if eps_r is None else _f64(eps_r)
        pc = None if pec is None else np.ascontiguousarray(pec, dtype=np.uint8)
        _ck(lib().mfd_batch_set_materials(self.h, dom, _p(er), _p(pc)))

    def set_field(self, dom, comp, values, rhs=-1):
        if _is_cuda_tensor(values):
            _ck(lib().mfd_batch_set_field_device(self.h, dom, comp, rhs, _dev_ptr(values), _torch_stream()))
            return
        _ck(lib().mfd_batch_set_field(self.h, dom, comp, rhs, _p(_f64(values))))

    def get_field(self, dom, comp, rhs=-1, out=None):
        if out is not None and _is_cuda_tensor(out):
            _ck(lib().mfd_batch_get_field_device(self.h, dom, comp, rhs, _dev_ptr(out), _torch_stream()))
            return out
        out = np.empty((self.n[dom], self.nrhs) if rhs < 0 else self.n[dom])
        _ck(lib().mfd_batch_get_field(self.h, dom, comp, rhs, _p(out)))
        return out

    def set_gamma(self, dom, gamma):
        """Per right-hand side hyperviscosity coefficients (mfd_batch_set_gamma)."""
        g = _f64(gamma)
        if g.shape != (self.nrhs,):
            raise ValueError("one gamma per right-hand side")
        _ck(lib().mfd_batch_set_gamma(self.h, dom, _p(g)))

    def energy(self, dom):
        """Eq. 20 energy of every right-hand side of domain dom (mfd_batch_energy)."""
        u = np.empty(self.nrhs)
        _ck(lib().mfd_batch_energy(self.h, dom, _p(u)))
        return u

    def set_sources(self, dom, node, rhs, amp, f0, t0):
        node = np.ascontiguousarray(node, dtype=np.int64)
        r = np.ascontiguousarray(rhs, dtype=np.int32)
        _ck(lib().mfd_batch_set_sources(self.h, dom, len(node), _p(node), _p(r), _p(_f64(amp)), _p(_f64(f0)),
                                        _p(_f64(t0))))

    def set_probes(self, dom, node, capacity):
        node = np.ascontiguousarray(node, dtype=np.int64)
        _ck(lib().mfd_batch_set_probes(self.h, dom, len(node), _p(node), int(capacity)))
        self.nprobe[dom] = len(node)

    def step(self, n):
        _ck(lib().mfd_batch_step(self.h, int(n)))

    def save_state(self):
        """Checkpoint of every domain's fields, the step index and the probe records (bytes)."""
        return _save_state(lib().mfd_batch_state_size, lib().mfd_batch_save_state, self.h)

    def load_state(self, blob):
        """Resumes from a checkpoint of save_state (a batch built the same way)."""
        _ck(lib().mfd_batch_load_state(self.h, blob, len(blob)))

    def set_variant(self, variant):
        """Variant of the batched kernel (mfd_batch_set_variant): bit 0 = no next-chunk stream
        prefetch (four resident blocks per SM instead of three); bit 1 = the H row's HV term
        summed in the E pass of the step before (H* kept beside the state)."""
        _ck(lib().mfd_batch_set_variant(self.h, int(variant)))

    @property
    def variant(self):
        return int(lib().mfd_batch_variant(self.h))

    def autotune(self, reps=20):
        """Times the four variants on this batch and keeps the fastest (mfd_batch_autotune):
        (chosen variant, ms per step of each)."""
        chosen = C.c_int(-1)
        ms = np.zeros(4)
        _ck(lib().mfd_batch_autotune(self.h, int(reps), C.byref(chosen), _p(ms)))
        return chosen.value, ms

    def set_spin_limit(self, limit):
        """Polls a waiting block makes at a grid barrier before the call gives up (mfd_batch_set_spin_limit)."""
        _ck(lib().mfd_batch_set_spin_limit(self.h, int(limit)))

    def read_probes(self, dom):
        steps = C.c_int64(0)
        _ck(lib().mfd_batch_read_probes(self.h, dom, None, C.byref(steps)))
        out = np.zeros((steps.value, self.nprobe[dom], self.nrhs))
        if steps.value and self.nprobe[dom]:
            _ck(lib().mfd_batch_read_probes(self.h, dom, _p(out), C.byref(steps)))
        return out

    @property
    def uses_graph(self):
        return bool(lib().mfd_batch_uses_graph(self.h))

    @property
    def nodes(self):
        return int(lib().mfd_batch_nodes(self.h))

    def __del__(self):
        try:
            if self.h:
                lib().mfd_batch_destroy(self.h)
                self.h = None
        except Exception:
            pass


def _host_f64(x):
    if hasattr(x, "detach"):  # a torch tensor
        x = x.detach().cpu().double().numpy()
    return np.ascontiguousarray(x, dtype=np.float64)


class ProbeObjective:
    """A collocated TMz run whose probe objective J(eps_r, amp) = dt sum_n sum_p Ez_p^n^2
    is differentiable through ``ProbeEnergy``: the forward pass runs the steps
    (recording a tape only when a gradient may be asked for), the backward pass
    runs the adjoint sweep over that tape (mfd_grad_forward / mfd_grad_backward).
    eps_r and amp may be torch CUDA tensors (zero copy) or host arrays."""

    def __init__(self, sim: Sim, pec, fields, sources, probes, nsteps, every=0):
        self.sim, self.pec, self.fields = sim, pec, fields
        self.src, self.probes, self.nsteps, self.every = sources, probes, nsteps, every
        self._pec_dev = None
        self.last_forward_taped = None

    def _setup(self, eps_r, amp):
        s = self.sim
        if _is_cuda_tensor(eps_r):
            import torch
            eps = eps_r.detach().to(torch.float64).contiguous()
            if self.pec is not None and self._pec_dev is None:
                self._pec_dev = torch.as_tensor(np.ascontiguousarray(self.pec, dtype=np.uint8), device=eps.device)
            pec = C.c_void_p(self._pec_dev.data_ptr()) if self.pec is not None else None
            _ck(lib().mfd_set_materials_device(s.h, _dev_ptr(eps), pec, _torch_stream()))
        else:
            s.set_materials(_host_f64(eps_r), self.pec)
        for comp, v in self.fields.items():
            s.set_field(comp, v)
        if _is_cuda_tensor(amp):
            import torch
            a = amp.detach().to(torch.float64).contiguous()
            s.set_sources(self.src.node, np.ones(len(self.src.node)), self.src.f0, self.src.t0)
            _ck(lib().mfd_set_source_amps_device(s.h, _dev_ptr(a), _torch_stream()))
        else:
            s.set_sources(self.src.node, _host_f64(amp), self.src.f0, self.src.t0)
        s.set_probes(self.probes, self.nsteps)

    def run(self, eps_r, amp):
        """J and its gradient in one call (mfd_grad): (J, dJ/deps_r, dJ/d amplitude) on the host."""
        self._setup(eps_r, amp)
        return self.sim.grad(self.nsteps, self.every, len(self.src.node))

    def forward(self, eps_r, amp, taped):
        """The forward run and J; with taped, also the tape of mfd_grad_forward (else None)."""
        self._setup(eps_r, amp)
        self.last_forward_taped = bool(taped)
        J = C.c_double(0.0)
        if not taped:
            self.sim.step(self.nsteps)
            _ck(lib().mfd_probe_objective(self.sim.h, C.byref(J)))
            return J.value, None
        tape = C.c_void_p()
        _ck(lib().mfd_grad_forward(self.sim.h, int(self.nsteps), int(self.every), C.byref(J), C.byref(tape)))
        return J.value, tape

    def backward(self, tape, device):
        """The adjoint sweep over a tape: (dJ/deps_r, dJ/d amplitude) as float64 tensors on `device`."""
        import torch
        try:
            ns = len(self.src.node)
            ge = torch.empty(self.sim.ne, dtype=torch.float64, device=device)
            ga = torch.empty(max(ns, 1), dtype=torch.float64, device=device)
            if ge.is_cuda:
                _ck(lib().mfd_grad_backward(tape, _dev_ptr(ge), _dev_ptr(ga), 1, _torch_stream()))
            else:
                _ck(lib().mfd_grad_backward(tape, C.c_void_p(ge.data_ptr()), C.c_void_p(ga.data_ptr()), 0, None))
            return ge, ga[:ns]
        finally:
            lib().mfd_tape_destroy(tape)


def _probe_energy_function():
    import torch

    class ProbeEnergy(torch.autograd.Function):
        """J(eps_r, amp) of a ProbeObjective. forward runs the steps (and records a
        tape when a gradient may follow); backward runs the adjoint sweep."""

        @staticmethod
        def forward(ctx, eps_r, amp, obj, taped):
            J, tape = obj.forward(eps_r, amp, taped)
            ctx.obj, ctx.tape = obj, tape
            ctx.dtypes = (eps_r.dtype, amp.dtype)
            ctx.device = eps_r.device
            return torch.tensor(J, dtype=torch.float64, device=eps_r.device)

        @staticmethod
        def backward(ctx, gJ):
            if ctx.tape is None:
                raise RuntimeError("ProbeEnergy: the forward pass recorded no tape")
            ge, ga = ctx.obj.backward(ctx.tape, ctx.device)
            ctx.tape = None
            g = gJ.to(torch.float64)
            return (g * ge).to(ctx.dtypes[0]), (g * ga).to(ctx.dtypes[1]), None, None

    return ProbeEnergy


def probe_energy(eps_r, amp, obj: ProbeObjective):
    """Differentiable J(eps_r, amp) (torch tensors in, 0-d tensor out). Under
    torch.no_grad(), or when neither input requires a gradient, only the
    forward run is made (no tape, no adjoint)."""
    import torch
    taped = torch.is_grad_enabled() and (eps_r.requires_grad or amp.requires_grad)
    return _probe_energy_function().apply(eps_r, amp, obj, taped)
