"""ctypes front end of the 3D C oracle (test infrastructure only).

Arrays are float64 numpy arrays in the natural 3D staggered layouts of
stokes3d_oracle.c, indexed [k][j][i]: vx nz x ny x (nx+1), vy nz x (ny+1) x nx,
vz (nz+1) x ny x nx, p and eta_c nz x ny x nx, eta_xy nz x (ny+1) x (nx+1),
eta_xz (nz+1) x ny x (nx+1), eta_yz (nz+1) x (ny+1) x nx.  Functions return new
arrays and never modify their inputs.
"""
import ctypes
from dataclasses import dataclass

import numpy as np

from . import oracle as _o2

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_i, _d, _u64 = ctypes.c_int, ctypes.c_double, ctypes.c_uint64
_H = [_i, _i, _i, _d, _d, _d, _D, _D, _D, _D]

_SIGS = {
    "o3_apply_M": (None, _H + [_D] * 6),
    "o3_diag_M": (None, _H + [_D] * 3),
    "o3_apply_D": (None, [_i, _i, _i, _d, _d, _d] + [_D] * 4),
    "o3_rhs": (None, [_i, _i, _i, _d, _d, _d] + [_D] * 7),
    "o3_jacobi": (None, _H + [_D] * 3 + [_d, _i] + [_D] * 3),
    "o3_ras_shift": (None, [_i, _u64, _I, _i, _i, _i, _i, _I]),
    "o3_ras": (_i, _H + [_D] * 3 + [_d, _i, _i, _i, _i, _i, _i, _i, _u64, _I, _u64] + [_D] * 3 + [_I]),
    "o3_energy": (None, _H + [_D] * 7 + [_D]),
}
_bound = False


def lib():
    global _bound
    h = _o2.lib()
    if not _bound:
        for name, (res, args) in _SIGS.items():
            f = getattr(h, name)
            f.restype = res
            f.argtypes = args
        _bound = True
    return h


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


@dataclass
class Grid3:
    """A 3D staggered grid with its viscosity fields (natural layouts)."""
    nx: int
    ny: int
    nz: int
    hx: float
    hy: float
    hz: float
    eta_c: np.ndarray
    eta_xy: np.ndarray
    eta_xz: np.ndarray
    eta_yz: np.ndarray

    def __post_init__(self):
        self.eta_c, self.eta_xy = _f64(self.eta_c), _f64(self.eta_xy)
        self.eta_xz, self.eta_yz = _f64(self.eta_xz), _f64(self.eta_yz)
        nx, ny, nz = self.nx, self.ny, self.nz
        assert self.eta_c.shape == (nz, ny, nx)
        assert self.eta_xy.shape == (nz, ny + 1, nx + 1)
        assert self.eta_xz.shape == (nz + 1, ny, nx + 1)
        assert self.eta_yz.shape == (nz + 1, ny + 1, nx)

    @property
    def head(self):
        return (self.nx, self.ny, self.nz, self.hx, self.hy, self.hz, _p(self.eta_c), _p(self.eta_xy),
                _p(self.eta_xz), _p(self.eta_yz))

    @property
    def dims(self):
        return (self.nx, self.ny, self.nz, self.hx, self.hy, self.hz)

    def zeros(self):
        nx, ny, nz = self.nx, self.ny, self.nz
        return np.zeros((nz, ny, nx + 1)), np.zeros((nz, ny + 1, nx)), np.zeros((nz + 1, ny, nx))


def apply_M(g: Grid3, vx, vy, vz):
    out = g.zeros()
    lib().o3_apply_M(*g.head, _p(_f64(vx)), _p(_f64(vy)), _p(_f64(vz)), *map(_p, out))
    return out


def diag_M(g: Grid3):
    out = g.zeros()
    lib().o3_diag_M(*g.head, *map(_p, out))
    return out


def apply_D(g: Grid3, vx, vy, vz):
    out = np.zeros((g.nz, g.ny, g.nx))
    lib().o3_apply_D(*g.dims, _p(_f64(vx)), _p(_f64(vy)), _p(_f64(vz)), _p(out))
    return out


def rhs(g: Grid3, fx, fy, fz, p=None):
    out = g.zeros()
    p = None if p is None else _f64(p)
    lib().o3_rhs(*g.dims, _p(_f64(fx)), _p(_f64(fy)), _p(_f64(fz)), _p(p), *map(_p, out))
    return out


def jacobi(g: Grid3, b, omega, sweeps, v):
    v = tuple(_f64(a).copy() for a in v)
    lib().o3_jacobi(*g.head, *(_p(_f64(a)) for a in b), omega, sweeps, *map(_p, v))
    return v


def ras_shift(shift_mode, seed, t, ti, tj, tk, shifts=None):
    out = (ctypes.c_int * 3)()
    sh = None
    if shifts is not None:
        arr = np.ascontiguousarray(np.asarray(shifts, dtype=np.int32).reshape(-1))
        sh = arr.ctypes.data_as(_I)
    lib().o3_ras_shift(shift_mode, seed & (2**64 - 1), sh, t, ti, tj, tk, out)
    return int(out[0]), int(out[1]), int(out[2])


def ras(g: Grid3, b, omega, sweeps, tile, k, overlap, shift_mode=1, seed=0, shifts=None, order_seed=0, v=None,
        return_counts=False):
    """RAS-Jacobi on 3D tiles (Algorithm 2 in 3D).  Returns (vx, vy, vz) or
    (vx, vy, vz, counts_x, counts_y, counts_z)."""
    v = g.zeros() if v is None else tuple(_f64(a).copy() for a in v)
    sh = None
    if shifts is not None:
        arr = np.ascontiguousarray(np.asarray(shifts, dtype=np.int32).reshape(-1))
        sh = arr.ctypes.data_as(_I)
    n = [a.size for a in v]
    counts = np.zeros(sum(n), dtype=np.int32) if return_counts else None
    st = lib().o3_ras(*g.head, *(_p(_f64(a)) for a in b), omega, sweeps, tile[0], tile[1], tile[2], k, overlap,
                      shift_mode, seed & (2**64 - 1), sh, order_seed & (2**64 - 1), *map(_p, v),
                      None if counts is None else counts.ctypes.data_as(_I))
    if st != 0:
        raise ValueError("o3_ras: bad arguments")
    if return_counts:
        cx = counts[:n[0]].reshape(v[0].shape)
        cy = counts[n[0]:n[0] + n[1]].reshape(v[1].shape)
        cz = counts[n[0] + n[1]:].reshape(v[2].shape)
        return v + (cx, cy, cz)
    return v


def energy(g: Grid3, f, p, v):
    """(sum r_v^2/(-diag M), sum (D v)^2 eta_c/(2/hx^2+2/hy^2+2/hz^2), sum f^2/(-diag M))."""
    out = (ctypes.c_double * 3)()
    p = None if p is None else _f64(p)
    lib().o3_energy(*g.head, *(_p(_f64(a)) for a in f), _p(p), *(_p(_f64(a)) for a in v), out)
    return float(out[0]), float(out[1]), float(out[2])
