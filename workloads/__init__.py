"""Seeded synthetic inputs shared by the oracle tests, the CUDA-path tests and the benchmark.

This module draws node sets, material fields, source/probe placements and
initial fields. It holds none of the method's arithmetic (no stencil
selection, no weights, no time stepping): everything here is input data.

Units: every workload is expressed in units of the mean node spacing h
(h = 1) and the time step (dt = 1). Then c0 = S_c (the Courant number),
and with the vacuum impedance eta0 = 1 one has eps0 = mu0 = 1 / S_c, so that
dt/mu0 = dt/eps0 = S_c.

Random numbers come from splitmix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): the i-th draw of stream
`seed` is mix(seed + (i + 1) * 0x9E3779B97F4A7C15), mapped to a double in
[0, 1) as (z >> 11) * 2^-53.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws `offset .. offset+count-1` of the splitmix64 stream `seed` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the splitmix64 stream `seed`."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, count: int) -> np.ndarray:
    """Standard normal draws (Box-Muller on two interleaved uniform draws)."""
    u = uniform(seed, 2 * count)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


@dataclass
class NodeSet:
    """A scattered node set in `dim` dimensions (user order).

    xyz    : (N, dim) float64 coordinates.
    pec    : (N,) uint8, 1 on perfectly conducting boundary nodes.
    normal_axes: (N,) uint8 bit mask, bit a set when the node sits on a wall
             normal to axis a (3D PEC: tangential E components are zeroed).
    period : (dim,) float64, the period along each axis (0 = not periodic).
    box_lo, box_hi: bounding box used for Morton keys.
    """

    xyz: np.ndarray
    pec: np.ndarray
    period: np.ndarray
    box_lo: np.ndarray
    box_hi: np.ndarray
    normal_axes: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def dim(self) -> int:
        return int(self.xyz.shape[1])


def _grid(shape):
    axes = [np.arange(s, dtype=np.float64) for s in shape]
    mesh = np.meshgrid(*axes, indexing="ij")
    # user order: axis 0 fastest
    return np.stack([m.transpose().reshape(-1) for m in mesh], axis=1)


def pec_box(shape, jitter: float, seed: int) -> NodeSet:
    """Regular grid of `shape` nodes over [0, shape[a]-1] per axis, PEC walls.

    Interior nodes are moved by U(-jitter, jitter) per axis. Wall nodes move
    only along the wall (tangential jitter); edges and corners keep the
    coordinates they share with more than one wall fixed.
    """
    shape = tuple(int(s) for s in shape)
    d = len(shape)
    xyz = _grid(shape)
    n = xyz.shape[0]
    u = uniform(seed, n * d).reshape(n, d)
    jit = (2.0 * u - 1.0) * jitter
    on_wall = np.zeros((n, d), dtype=bool)
    for a in range(d):
        on_wall[:, a] = (xyz[:, a] == 0) | (xyz[:, a] == shape[a] - 1)
    jit[on_wall] = 0.0
    xyz = xyz + jit
    pec = on_wall.any(axis=1).astype(np.uint8)
    normal_axes = np.zeros(n, dtype=np.uint8)
    for a in range(d):
        normal_axes |= (on_wall[:, a].astype(np.uint8) << a)
    hi = np.array([s - 1 for s in shape], dtype=np.float64)
    return NodeSet(xyz=xyz, pec=pec, period=np.zeros(d), box_lo=np.zeros(d), box_hi=hi,
                   normal_axes=normal_axes, meta={"kind": "pec_box", "shape": shape})


def pec_box_cells(shape, jitter: float, seed: int) -> NodeSet:
    """Regular grid of `shape` nodes at the cell centres (i + 1/2) of the box
    [0, shape[a]] per axis, every node moved by U(-jitter, jitter) per axis;
    the PEC walls are the box faces, half a spacing beyond the outer layers, so
    no node sits on a wall (the layout of PEC walls by images)."""
    shape = tuple(int(s) for s in shape)
    d = len(shape)
    xyz = _grid(shape) + 0.5
    n = xyz.shape[0]
    u = uniform(seed, n * d).reshape(n, d)
    xyz = xyz + (2.0 * u - 1.0) * jitter
    hi = np.array(shape, dtype=np.float64)
    return NodeSet(xyz=xyz, pec=np.zeros(n, np.uint8), period=np.zeros(d), box_lo=np.zeros(d), box_hi=hi,
                   normal_axes=np.zeros(n, np.uint8), meta={"kind": "pec_box_cells", "shape": shape})


def periodic_box(shape, jitter: float, seed: int, offset=None, seed_line_y=None,
                 seed_diagonal: bool = False) -> NodeSet:
    """Regular grid of `shape` nodes on the periodic box [0, shape[a]) per axis.

    Every node is moved by U(-jitter, jitter) per axis and wrapped into the
    box. `offset` shifts the whole lattice (the H set of the staggered layout
    sits at +(1/2, 1/2)). Nodes whose unshifted y equals `seed_line_y` keep
    their y coordinate (an equispaced line for Fourier sampling); with
    seed_diagonal, the nodes whose unshifted x equals y are not moved (an
    equispaced diagonal, spacing sqrt(2), for sampling at 45 degrees).
    """
    shape = tuple(int(s) for s in shape)
    d = len(shape)
    xyz = _grid(shape)
    n = xyz.shape[0]
    u = uniform(seed, n * d).reshape(n, d)
    jit = (2.0 * u - 1.0) * jitter
    if seed_line_y is not None:
        line = xyz[:, 1] == seed_line_y
        jit[line, 1] = 0.0
        jit[line, 0] = 0.0
    if seed_diagonal:
        jit[xyz[:, 0] == xyz[:, 1]] = 0.0
    if offset is not None:
        xyz = xyz + np.asarray(offset, dtype=np.float64)
    xyz = xyz + jit
    period = np.array(shape, dtype=np.float64)
    xyz = np.mod(xyz, period)
    xyz = np.where(xyz >= period, xyz - period, xyz)
    return NodeSet(xyz=xyz, pec=np.zeros(n, dtype=np.uint8), period=period,
                   box_lo=np.zeros(d), box_hi=period.copy(),
                   normal_axes=np.zeros(n, dtype=np.uint8),
                   meta={"kind": "periodic", "shape": shape})


def disk(radius: float, jitter: float, seed: int) -> NodeSet:
    """Disk of `radius` (in h) centred at (radius, radius), PEC rim.

    Interior: the jittered unit grid clipped to distance < radius - 0.5.
    Rim: round(2*pi*radius) equispaced PEC nodes on the circle.
    """
    m = int(math.ceil(2 * radius)) + 1
    g = _grid((m, m))
    n = g.shape[0]
    u = uniform(seed, 2 * n).reshape(n, 2)
    g = g + (2.0 * u - 1.0) * jitter
    c = np.array([radius, radius])
    keep = np.linalg.norm(g - c, axis=1) < radius - 0.5
    inner = g[keep]
    k = int(round(2 * math.pi * radius))
    th = 2 * math.pi * np.arange(k) / k
    rim = c + radius * np.stack([np.cos(th), np.sin(th)], axis=1)
    xyz = np.concatenate([inner, rim], axis=0)
    pec = np.concatenate([np.zeros(len(inner), np.uint8), np.ones(k, np.uint8)])
    return NodeSet(xyz=xyz, pec=pec, period=np.zeros(2), box_lo=np.zeros(2),
                   box_hi=np.array([2 * radius, 2 * radius]),
                   normal_axes=pec.copy(), meta={"kind": "disk", "radius": radius})


def interior_nodes(nodes: NodeSet, count: int, seed: int, margin: float = 0.0) -> np.ndarray:
    """`count` distinct non-PEC node ids drawn with splitmix64 (ascending draw order)."""
    ok = nodes.pec == 0
    if margin > 0:
        lo = nodes.box_lo + margin
        hi = nodes.box_hi - margin
        ok &= np.all((nodes.xyz >= lo) & (nodes.xyz <= hi), axis=1)
    cand = np.nonzero(ok)[0]
    if count > len(cand):
        raise ValueError("not enough interior nodes")
    keys = splitmix64(seed, len(cand))
    order = np.argsort(keys, kind="stable")
    return np.sort(cand[order[:count]])


def eps_r_smooth_3d(xyz: np.ndarray, box_hi: np.ndarray, seed: int, grid: int = 128,
                    blur: float = 0.1, contrast: float = 3.0) -> np.ndarray:
    """Relative permittivity 1 + contrast * g from a smoothed Gaussian random field.

    White noise N(0,1) on a periodic `grid`^3 lattice over the unit cube is
    blurred by a Gaussian of standard deviation `blur` (unit-cube length),
    min-max scaled to [0, 1] and interpolated trilinearly at the nodes
    (node coordinates divided by `box_hi`).
    """
    w = normal(seed, grid ** 3).reshape(grid, grid, grid)
    k = np.fft.fftfreq(grid) * 2.0 * np.pi  # radians per cell
    s = blur * grid  # standard deviation in cells
    k2 = k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2
    g = np.real(np.fft.ifftn(np.fft.fftn(w) * np.exp(-0.5 * s * s * k2)))
    g = (g - g.min()) / (g.max() - g.min())
    p = np.clip(xyz / box_hi, 0.0, 1.0) * (grid - 1)
    i0 = np.minimum(np.floor(p).astype(np.int64), grid - 2)
    t = p - i0
    out = np.zeros(len(xyz))
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                wgt = ((t[:, 0] if dx else 1 - t[:, 0]) * (t[:, 1] if dy else 1 - t[:, 1])
                       * (t[:, 2] if dz else 1 - t[:, 2]))
                out += wgt * g[i0[:, 0] + dx, i0[:, 1] + dy, i0[:, 2] + dz]
    return 1.0 + contrast * out


def eps_r_uniform(n: int, seed: int, lo: float = 1.0, span: float = 0.5) -> np.ndarray:
    """Per-node relative permittivity lo + span * U[0, 1)."""
    return lo + span * uniform(seed, n)


@dataclass
class Sources:
    """Soft Ricker point sources: node id, right-hand side, amplitude, centre frequency, delay."""

    node: np.ndarray
    rhs: np.ndarray
    amp: np.ndarray
    f0: np.ndarray
    t0: np.ndarray


def ricker_sources(nodes: NodeSet, count: int, seed: int, c0: float, nrhs: int = 1,
                   ppw=(10.0, 20.0), one_per_rhs: bool = False) -> Sources:
    """`count` Ricker sources at random interior nodes.

    The wavelength c0/f0 is drawn from U[ppw[0], ppw[1]) (points per
    wavelength, h = 1); the delay is t0 = 1.5 / f0 and the amplitude 1.
    With one_per_rhs, source k drives right-hand side k.
    """
    node = interior_nodes(nodes, count, seed)
    u = uniform(seed + 1, count)
    lam = ppw[0] + (ppw[1] - ppw[0]) * u
    f0 = c0 / lam
    rhs = np.arange(count) % max(nrhs, 1) if one_per_rhs else np.zeros(count, np.int64)
    return Sources(node=node.astype(np.int64), rhs=rhs.astype(np.int64),
                   amp=np.ones(count), f0=f0, t0=1.5 / f0)


# ---------------------------------------------------------------- initial fields

def tm11_fields(xyz: np.ndarray, L: float, c0: float, mu0: float, t_e: float, t_h: float):
    """TM11 mode of the PEC square [0, L]^2 (closed form of Maxwell's TMz equations).

    Ez = sin(pi x/L) sin(pi y/L) cos(w t_e), w = sqrt(2) pi c0 / L, and the H
    fields that satisfy dH/dt = -(1/mu0) curl E at time t_h:
    Hx = -(pi/(L mu0 w)) sin(pi x/L) cos(pi y/L) sin(w t_h),
    Hy = +(pi/(L mu0 w)) cos(pi x/L) sin(pi y/L) sin(w t_h).
    """
    x, y = xyz[:, 0], xyz[:, 1]
    k = math.pi / L
    w = math.sqrt(2.0) * k * c0
    a = k / (mu0 * w)
    ez = np.sin(k * x) * np.sin(k * y) * math.cos(w * t_e)
    hx = -a * np.sin(k * x) * np.cos(k * y) * math.sin(w * t_h)
    hy = a * np.cos(k * x) * np.sin(k * y) * math.sin(w * t_h)
    return ez, hx, hy


def tm110_fields_3d(xyz: np.ndarray, L: float, c0: float, mu0: float, t_e: float, t_h: float):
    """TM110 mode of the PEC cube [0, L]^3: the TM11 square mode, constant in z."""
    ez, hx, hy = tm11_fields(xyz[:, :2], L, c0, mu0, t_e, t_h)
    z = np.zeros_like(ez)
    return (z, z.copy(), ez), (hx, hy, z.copy())


def gaussian_pulse(xyz: np.ndarray, period_x: float, x0: float, sigma: float, c0: float,
                   eta0: float, dt: float, wavelength: float | None = None, direction=(1, 0)):
    """Plane pulse on a periodic square box of side period_x (d'Alembert data).

    Along +x (direction (1, 0)): Ez(x, 0) = f(x - x0); Hx(-dt/2) = 0;
    Hy(-dt/2) = -f(x - x0 + c0 dt/2)/eta0, with f(s) = exp(-s^2/(2 sigma^2))
    [times cos(2 pi s / wavelength) for a modulated pulse], s the minimum
    image on the period. For an integer direction (p, q) at angle phi the
    coordinate is d = x cos(phi) + y sin(phi), periodic with period
    period_x / sqrt(p^2 + q^2) on the box, and (Eq. 27)
    Hx = sin(phi) f(d - x0 + c0 dt/2)/eta0, Hy = -cos(phi) f(...)/eta0.
    """
    p, q = direction
    norm = math.hypot(p, q)
    cp, sp = p / norm, q / norm
    period = period_x / norm

    def f(s):
        s = s - period * np.round(s / period)
        v = np.exp(-s * s / (2.0 * sigma * sigma))
        if wavelength is not None:
            v = v * np.cos(2.0 * np.pi * s / wavelength)
        return v

    d = xyz[:, 0] * cp + xyz[:, 1] * sp
    ez = f(d - x0)
    g = f(d - x0 + 0.5 * c0 * dt) / eta0
    hx = sp * g if q != 0 else np.zeros_like(ez)
    hy = -cp * g
    return ez, hx, hy


def pulse_exact(xyz: np.ndarray, period_x: float, x0: float, sigma: float, c0: float,
                eta0: float, t_e: float, t_h: float, wavelength: float | None = None):
    """d'Alembert solution of the plane pulse: E at time t_e, H at time t_h."""
    ez, _, _ = gaussian_pulse(xyz, period_x, x0 + c0 * t_e, sigma, c0, eta0, 0.0, wavelength)
    e2, _, _ = gaussian_pulse(xyz, period_x, x0 + c0 * t_h, sigma, c0, eta0, 0.0, wavelength)
    return ez, np.zeros_like(ez), -e2 / eta0


# ---------------------------------------------------------------- named workloads

def units(courant: float):
    """(dt, eps0, mu0, c0, eta0) in h-normalised units for Courant number S_c."""
    return 1.0, 1.0 / courant, 1.0 / courant, courant, 1.0


def n_monomials(m: int, d: int) -> int:
    """M_m = C(m + d, d): the number of monomials of total degree <= m in d variables."""
    return math.comb(m + d, d)


def batch_domains(count: int, seed: int, n_min: int = 2000, n_max: int = 60000,
                  stencils=(12, 20, 30, 40), jitter: float = 0.25):
    """`count` domains for the batched workload: squares and disks (alternating
    draws), node counts log-uniform in [n_min, n_max], stencil size drawn
    uniformly from `stencils`. Returns a list of (NodeSet, n)."""
    u = uniform(seed, 3 * count).reshape(count, 3)
    out = []
    for d in range(count):
        target = math.exp(math.log(n_min) + (math.log(n_max) - math.log(n_min)) * u[d, 0])
        n = stencils[min(int(u[d, 1] * len(stencils)), len(stencils) - 1)]
        if u[d, 2] < 0.5:
            side = max(8, int(round(math.sqrt(target))))
            ns = pec_box((side, side), jitter, seed * 1000 + d)
        else:
            ns = disk(max(6.0, math.sqrt(target / math.pi)), jitter, seed * 1000 + d)
        out.append((ns, n))
    return out


def poly_degree_for(n: int) -> int:
    """The largest augmentation degree m with 2 M_m <= n in 2D (n = 12, 20, 30, 40 -> 2, 3, 4, 4)."""
    m = 0
    while 2 * n_monomials(m + 1, 2) <= n:
        m += 1
    return m
