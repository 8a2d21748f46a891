"""Seeded synthetic inputs for the staggered-grid Stokes smoothers.

This module only builds input fields; it holds none of the solver's arithmetic
and is shared by the tests (GPU path and oracle alike) and the benchmark.

Every generator point-samples each material property at its own grid location
(eta_c at cell centres, eta_n at nodes, rho at vy points, which is where the
staggered grid of Sec. 2.1 / Fig. 1 keeps density).  Later inclusions overwrite
earlier ones.  The body force is f_x = 0, f_y = -rho * g_y (gravity pulls
toward -y for g_y < 0), zero on the wall entries.  Arrays are float64 in the
natural layouts: vx-like ny x (nx+1), vy-like (ny+1) x nx, cell ny x nx,
node (ny+1) x (nx+1).

Workloads (the paper's sinker of Sec. 6.1 and the synthetic grids of Sec. 7.1
stand in; no external dataset is involved):
  sinker_problem     centred circular inclusion (64^2 and 1024^2 cases)
  multi_sinker       20 seeded inclusions (4096^2 multigrid case)
  layered_sinker     10 seeded horizontal layers plus a sinker (8192^2 case)
  batch_specs        256 seeded sinker instances of uneven sizes (batched case)
"""
from dataclasses import dataclass, field
from typing import List

import numpy as np


@dataclass
class Problem:
    nx: int
    ny: int
    lx: float
    ly: float
    eta_c: np.ndarray
    eta_n: np.ndarray
    rho: np.ndarray  # at vy points, (ny+1) x nx
    fx: np.ndarray
    fy: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def hx(self):
        return self.lx / self.nx

    @property
    def hy(self):
        return self.ly / self.ny


def _coords(nx, ny, lx, ly):
    hx, hy = lx / nx, ly / ny
    xc = (np.arange(nx) + 0.5) * hx
    yc = (np.arange(ny) + 0.5) * hy
    xn = np.arange(nx + 1) * hx
    yn = np.arange(ny + 1) * hy
    return xc, yc, xn, yn


class _Painter:
    """Point-samples circles and bands into the three material arrays."""

    def __init__(self, nx, ny, lx, ly, eta_bg, rho_bg):
        self.nx, self.ny, self.lx, self.ly = nx, ny, lx, ly
        self.xc, self.yc, self.xn, self.yn = _coords(nx, ny, lx, ly)
        self.eta_c = np.full((ny, nx), float(eta_bg))
        self.eta_n = np.full((ny + 1, nx + 1), float(eta_bg))
        self.rho = np.full((ny + 1, nx), float(rho_bg))

    @staticmethod
    def _disc(arr, xs, ys, cx, cy, r, value):
        ilo, ihi = np.searchsorted(xs, cx - r), np.searchsorted(xs, cx + r, side="right")
        jlo, jhi = np.searchsorted(ys, cy - r), np.searchsorted(ys, cy + r, side="right")
        if ilo >= ihi or jlo >= jhi:
            return
        dx = xs[ilo:ihi][None, :] - cx
        dy = ys[jlo:jhi][:, None] - cy
        m = dx * dx + dy * dy < r * r
        arr[jlo:jhi, ilo:ihi][m] = value

    def circle(self, cx, cy, r, eta, rho):
        self._disc(self.eta_c, self.xc, self.yc, cx, cy, r, eta)
        self._disc(self.eta_n, self.xn, self.yn, cx, cy, r, eta)
        self._disc(self.rho, self.xc, self.yn, cx, cy, r, rho)

    def band(self, y0, y1, eta, rho=None):
        """Horizontal band y0 <= y < y1."""
        self.eta_c[(self.yc >= y0) & (self.yc < y1), :] = eta
        self.eta_n[(self.yn >= y0) & (self.yn < y1), :] = eta
        if rho is not None:
            self.rho[(self.yn >= y0) & (self.yn < y1), :] = rho

    def finish(self, g_y, meta):
        nx, ny = self.nx, self.ny
        fx = np.zeros((ny, nx + 1))
        fy = -self.rho * g_y
        fy[0, :] = 0.0
        fy[ny, :] = 0.0
        return Problem(nx, ny, self.lx, self.ly, self.eta_c, self.eta_n, self.rho, fx, fy, meta)


def sinker_problem(nx, ny=None, eta_in=1e3, eta_out=1.0, rho_in=2.0, rho_out=1.0, radius=0.1, center=(0.5, 0.5),
                   lx=1.0, ly=1.0, g_y=-1.0):
    """Centred circular sinker (Sec. 6.1 geometry, scaled to the unit square)."""
    ny = nx if ny is None else ny
    p = _Painter(nx, ny, lx, ly, eta_out, rho_out)
    p.circle(center[0] * lx, center[1] * ly, radius * min(lx, ly), eta_in, rho_in)
    return p.finish(g_y, dict(kind="sinker", eta_in=eta_in, eta_out=eta_out))


def multi_sinker(n, seed=3, count=20, lx=1.0, ly=1.0, g_y=-1.0):
    """`count` inclusions drawn in order: r ~ U[0.02, 0.08], cx, cy ~ U[r, 1-r],
    log10 eta ~ U[-3, 3], rho ~ U[0.9, 1.1]; background eta = rho = 1."""
    rng = np.random.default_rng(seed)
    p = _Painter(n, n, lx, ly, 1.0, 1.0)
    incl = []
    for _ in range(count):
        r = rng.uniform(0.02, 0.08)
        cx = rng.uniform(r, 1.0 - r)
        cy = rng.uniform(r, 1.0 - r)
        eta = 10.0 ** rng.uniform(-3.0, 3.0)
        rho = rng.uniform(0.9, 1.1)
        p.circle(cx * lx, cy * ly, r * min(lx, ly), eta, rho)
        incl.append((cx, cy, r, eta, rho))
    return p.finish(g_y, dict(kind="multi_sinker", seed=seed, inclusions=incl))


def layered_sinker(n, seed=4, layers=10, lx=1.0, ly=1.0, g_y=-1.0, sinker_eta=1e3, sinker_rho=2.0, radius=0.1):
    """`layers` horizontal layers of equal height with log10 eta ~ U[-3, 3]
    (drawn bottom to top), background rho = 1, plus a centred sinker."""
    rng = np.random.default_rng(seed)
    p = _Painter(n, n, lx, ly, 1.0, 1.0)
    etas = []
    for q in range(layers):
        eta = 10.0 ** rng.uniform(-3.0, 3.0)
        y0, y1 = q * ly / layers, (q + 1) * ly / layers
        if q == layers - 1:
            y1 = 2.0 * ly  # the top node row belongs to the last layer
        p.band(y0, y1, eta)
        etas.append(eta)
    p.circle(0.5 * lx, 0.5 * ly, radius * min(lx, ly), sinker_eta, sinker_rho)
    return p.finish(g_y, dict(kind="layered_sinker", seed=seed, layer_eta=etas))


@dataclass
class BatchSpec:
    n: int
    contrast: float
    radius: float
    cx: float
    cy: float


def batch_specs(seed=5, count=256):
    """Instance table of the batched workload: side n = 64 round(2^U(6,10) / 64)
    (cells log-uniform between 64^2 and 1024^2; a multiple of 64, so that
    halving reaches a coarsest level of at most 16 x 16 cells), contrast
    c = 10^U(2,6), one sinker r ~ U[0.05, 0.2], centre ~ U[0.3, 0.7]^2."""
    rng = np.random.default_rng(seed)
    out: List[BatchSpec] = []
    for _ in range(count):
        n = int(64 * round(2.0 ** rng.uniform(6.0, 10.0) / 64.0))
        c = 10.0 ** rng.uniform(2.0, 6.0)
        r = rng.uniform(0.05, 0.2)
        cx = rng.uniform(0.3, 0.7)
        cy = rng.uniform(0.3, 0.7)
        out.append(BatchSpec(n, c, r, cx, cy))
    return out


def batch_problem(spec: BatchSpec, g_y=-1.0):
    return sinker_problem(spec.n, eta_in=spec.contrast, eta_out=1.0, rho_in=2.0, rho_out=1.0, radius=spec.radius,
                          center=(spec.cx, spec.cy), g_y=g_y)


def random_velocity(nx, ny, seed, scale=1.0):
    """Seeded random velocity with zero wall entries (natural layouts)."""
    rng = np.random.default_rng(seed)
    vx = rng.standard_normal((ny, nx + 1)) * scale
    vy = rng.standard_normal((ny + 1, nx)) * scale
    vx[:, 0] = 0.0
    vx[:, nx] = 0.0
    vy[0, :] = 0.0
    vy[ny, :] = 0.0
    return vx, vy


def random_pressure(nx, ny, seed, scale=1.0):
    return np.random.default_rng(seed).standard_normal((ny, nx)) * scale


def random_viscosity(nx, ny, seed, log10_range=(-2.0, 2.0)):
    """Seeded log-uniform random viscosity at centres and nodes."""
    rng = np.random.default_rng(seed)
    eta_c = 10.0 ** rng.uniform(*log10_range, size=(ny, nx))
    eta_n = 10.0 ** rng.uniform(*log10_range, size=(ny + 1, nx + 1))
    return eta_c, eta_n


def random_shifts(n_outer, ti, tj, seed):
    """Explicit tile-shift list (s_i, s_j) per outer iteration, s_i in [0, ti)."""
    rng = np.random.default_rng(seed)
    s = np.empty((n_outer, 2), dtype=np.int32)
    s[:, 0] = rng.integers(0, ti, size=n_outer)
    s[:, 1] = rng.integers(0, tj, size=n_outer)
    return s


# ---------------------------------------------------------------------------
# 3D staggered grid: nx x ny x nz cells, arrays indexed [k][j][i]
#   vx-like nz x ny x (nx+1), vy-like nz x (ny+1) x nx, vz-like (nz+1) x ny x nx,
#   cells nz x ny x nx, x-y edges nz x (ny+1) x (nx+1), x-z edges
#   (nz+1) x ny x (nx+1), y-z edges (nz+1) x (ny+1) x nx.
# Density sits with vz (gravity along -z); the body force is f_z = -rho g_z.
# ---------------------------------------------------------------------------
@dataclass
class Problem3:
    nx: int
    ny: int
    nz: int
    lx: float
    ly: float
    lz: float
    eta_c: np.ndarray
    eta_xy: np.ndarray
    eta_xz: np.ndarray
    eta_yz: np.ndarray
    rho: np.ndarray  # at vz points
    fx: np.ndarray
    fy: np.ndarray
    fz: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def hx(self):
        return self.lx / self.nx

    @property
    def hy(self):
        return self.ly / self.ny

    @property
    def hz(self):
        return self.lz / self.nz


def _axes3(nx, ny, nz, lx, ly, lz):
    hx, hy, hz = lx / nx, ly / ny, lz / nz
    c = [(np.arange(n) + 0.5) * h for n, h in ((nx, hx), (ny, hy), (nz, hz))]
    e = [np.arange(n + 1) * h for n, h in ((nx, hx), (ny, hy), (nz, hz))]
    return c, e


def _ball(xs, ys, zs, cx, cy, cz, r):
    """Mask [k][j][i] of the points (xs[i], ys[j], zs[k]) strictly inside the ball."""
    return ((xs[None, None, :] - cx) ** 2 + (ys[None, :, None] - cy) ** 2 + (zs[:, None, None] - cz) ** 2) < r * r


def sinker3d_problem(nx, ny=None, nz=None, eta_in=1e3, eta_out=1.0, rho_in=2.0, rho_out=1.0, radius=0.1,
                     center=(0.5, 0.5, 0.5), lx=1.0, ly=1.0, lz=1.0, g_z=-1.0):
    """A spherical sinker in a box (the 3D counterpart of the Sec. 6.1
    sinker): every material property point-sampled at its own location."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    (xc, yc, zc), (xn, yn, zn) = _axes3(nx, ny, nz, lx, ly, lz)
    cx, cy, cz = center[0] * lx, center[1] * ly, center[2] * lz
    r = radius * min(lx, ly, lz)
    eta_c = np.where(_ball(xc, yc, zc, cx, cy, cz, r), eta_in, eta_out).astype(np.float64)
    eta_xy = np.where(_ball(xn, yn, zc, cx, cy, cz, r), eta_in, eta_out).astype(np.float64)
    eta_xz = np.where(_ball(xn, yc, zn, cx, cy, cz, r), eta_in, eta_out).astype(np.float64)
    eta_yz = np.where(_ball(xc, yn, zn, cx, cy, cz, r), eta_in, eta_out).astype(np.float64)
    rho = np.where(_ball(xc, yc, zn, cx, cy, cz, r), rho_in, rho_out).astype(np.float64)
    fx = np.zeros((nz, ny, nx + 1))
    fy = np.zeros((nz, ny + 1, nx))
    fz = -rho * g_z
    fz[0] = 0.0
    fz[nz] = 0.0
    return Problem3(nx, ny, nz, lx, ly, lz, eta_c, eta_xy, eta_xz, eta_yz, rho, fx, fy, fz,
                    dict(kind="sinker3d", eta_in=eta_in))


def layered3d_problem(n, seed=6, layers=10, eta_range=(-3.0, 3.0), sinker_eta=1e3, sinker_rho=2.0, radius=0.1):
    """The 3D counterpart of the layered sinker: `layers` horizontal layers
    (along z, drawn bottom to top) with log10 eta ~ U[eta_range] plus a
    centred spherical sinker, on the unit cube."""
    rng = np.random.default_rng(seed)
    prob = sinker3d_problem(n, eta_in=sinker_eta, eta_out=1.0, rho_in=sinker_rho, radius=radius)
    (xc, yc, zc), (xn, yn, zn) = _axes3(n, n, n, 1.0, 1.0, 1.0)
    etas = 10.0 ** rng.uniform(*eta_range, size=layers)
    lay_c = np.minimum((zc * layers).astype(int), layers - 1)
    lay_n = np.minimum((zn * layers).astype(int), layers - 1)
    r = radius
    for arr, zs, xs, ys in ((prob.eta_c, lay_c, xc, yc), (prob.eta_xy, lay_c, xn, yn),
                            (prob.eta_xz, lay_n, xn, yc), (prob.eta_yz, lay_n, xc, yn)):
        zz = zc if zs is lay_c else zn
        inside = _ball(xs, ys, zz, 0.5, 0.5, 0.5, r)
        arr[...] = np.where(inside, sinker_eta, etas[zs][:, None, None])
    prob.meta = dict(kind="layered3d", seed=seed, layer_eta=etas.tolist())
    return prob


def random_viscosity3d(nx, ny, nz, seed, log10_range=(-2.0, 2.0)):
    """Seeded log-uniform viscosity at the cells and the three edge sets."""
    rng = np.random.default_rng(seed)
    u = lambda shape: 10.0 ** rng.uniform(*log10_range, size=shape)
    return (u((nz, ny, nx)), u((nz, ny + 1, nx + 1)), u((nz + 1, ny, nx + 1)), u((nz + 1, ny + 1, nx)))


def random_velocity3d(nx, ny, nz, seed, scale=1.0):
    """Seeded random velocity with zero wall entries."""
    rng = np.random.default_rng(seed)
    vx = rng.standard_normal((nz, ny, nx + 1)) * scale
    vy = rng.standard_normal((nz, ny + 1, nx)) * scale
    vz = rng.standard_normal((nz + 1, ny, nx)) * scale
    vx[:, :, 0] = vx[:, :, nx] = 0.0
    vy[:, 0, :] = vy[:, ny, :] = 0.0
    vz[0] = vz[nz] = 0.0
    return vx, vy, vz


def random_pressure3d(nx, ny, nz, seed, scale=1.0):
    return np.random.default_rng(seed).standard_normal((nz, ny, nx)) * scale
