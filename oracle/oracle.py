"""ctypes front end of the C oracle (test infrastructure only).

Every array is a float64 numpy array in the natural staggered layout
(see stokes_oracle.c): vx, fx, bx are ny x (nx+1); vy, fy, by are
(ny+1) x nx; p and eta_c are ny x nx; eta_n is (ny+1) x (nx+1).
Functions return new arrays and never modify their inputs.
"""
import ctypes
from dataclasses import dataclass

import numpy as np

from .build import build_oracle

_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_i, _d, _u64 = ctypes.c_int, ctypes.c_double, ctypes.c_uint64

_SIGS = {
    "ora_apply_M": (None, [_i, _i, _d, _d, _D, _D, _D, _D, _D, _D]),
    "ora_apply_G": (None, [_i, _i, _d, _d, _D, _D, _D]),
    "ora_apply_D": (None, [_i, _i, _d, _d, _D, _D, _D]),
    "ora_diag_M": (None, [_i, _i, _d, _d, _D, _D, _D, _D]),
    "ora_rhs": (None, [_i, _i, _d, _d, _D, _D, _D, _D, _D]),
    "ora_jacobi": (None, [_i, _i, _d, _d, _D, _D, _D, _D, _d, _i, _D, _D]),
    "ora_rbgs": (None, [_i, _i, _d, _d, _D, _D, _D, _D, _d, _i, _D, _D]),
    "ora_splitmix64": (ctypes.c_uint64, [_u64, _u64]),
    "ora_ras": (_i, [_i, _i, _d, _d, _D, _D, _D, _D, _d, _i, _i, _i, _i, _i, _i, _u64, _I, _u64, _D, _D, _I]),
    "ora_ras_shift": (None, [_i, _u64, _i, _i, _i, _I]),
    "ora_energy": (None, [_i, _i, _d, _d, _D, _D, _D, _D, _D, _D, _D, _D]),
    "ora_ras_tiles": (_i, [_i, _i, _d, _d, _D, _D, _D, _D, _d, _i, _i, _i, _i, _i, _i, _I, _i, _D, _D, _D, _D]),
    "ora_tile_count": (_i, [_i, _i, _i]),
    "ora_mg_levels": (_i, [_i, _i, _i, _i]),
    "ora_mg_sweeps": (_i, [_i, _d, _i, _i]),
    "ora_mg_prolong_add": (None, [_i, _i, _D, _D, _D, _D]),
    "ora_mg_restrict": (None, [_i, _i, _D, _D, _D, _D]),
    "ora_dense_solve": (_i, [_i, _i, _d, _d, _D, _D, _D, _D, _D, _D]),
    "ora_vcycle": (_i, [_i, _i, _d, _d, _D, _D, _D, _D, _i, _i, _i, _i, _d, _i, _i, _d, _i, _i, _i, _i, _u64, _D,
                        _D]),
    "ora_mg_fcg": (_i, [_i, _i, _d, _d, _D, _D, _D, _D, _D, _i, _i, _i, _i, _d, _i, _i, _d, _i, _i, _i, _i, _u64,
                        _d, _i, _D, _D, _D, _D]),
    "ora_mg_solve": (_i, [_i, _i, _d, _d, _D, _D, _D, _D, _D, _i, _i, _i, _i, _d, _i, _i, _d, _i, _i, _i, _i, _u64,
                          _d, _i, _D, _D, _D, _D]),
}


def _bind(h):
    for name, (res, args) in _SIGS.items():
        f = getattr(h, name)
        f.restype = res
        f.argtypes = args
    return h


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build_oracle()))
    return _lib





def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous float64"
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Grid:
    """A staggered grid with its viscosity fields (natural layouts)."""
    nx: int
    ny: int
    hx: float
    hy: float
    eta_c: np.ndarray  # ny x nx
    eta_n: np.ndarray  # (ny+1) x (nx+1)

    def __post_init__(self):
        self.eta_c = _f64(self.eta_c)
        self.eta_n = _f64(self.eta_n)
        assert self.eta_c.shape == (self.ny, self.nx)
        assert self.eta_n.shape == (self.ny + 1, self.nx + 1)

    @property
    def head(self):
        return (self.nx, self.ny, self.hx, self.hy, _p(self.eta_c), _p(self.eta_n))

    def zeros_vx(self):
        return np.zeros((self.ny, self.nx + 1))

    def zeros_vy(self):
        return np.zeros((self.ny + 1, self.nx))


def apply_M(g: Grid, vx, vy):
    vx, vy = _f64(vx), _f64(vy)
    ox, oy = g.zeros_vx(), g.zeros_vy()
    lib().ora_apply_M(*g.head, _p(vx), _p(vy), _p(ox), _p(oy))
    return ox, oy


def apply_G(g: Grid, p):
    p = _f64(p)
    ox, oy = g.zeros_vx(), g.zeros_vy()
    lib().ora_apply_G(g.nx, g.ny, g.hx, g.hy, _p(p), _p(ox), _p(oy))
    return ox, oy


def apply_D(g: Grid, vx, vy):
    vx, vy = _f64(vx), _f64(vy)
    out = np.zeros((g.ny, g.nx))
    lib().ora_apply_D(g.nx, g.ny, g.hx, g.hy, _p(vx), _p(vy), _p(out))
    return out


def diag_M(g: Grid):
    ox, oy = g.zeros_vx(), g.zeros_vy()
    lib().ora_diag_M(*g.head, _p(ox), _p(oy))
    return ox, oy


def rhs(g: Grid, fx, fy, p=None):
    fx, fy = _f64(fx), _f64(fy)
    p = None if p is None else _f64(p)
    bx, by = g.zeros_vx(), g.zeros_vy()
    lib().ora_rhs(g.nx, g.ny, g.hx, g.hy, _p(fx), _p(fy), _p(p), _p(bx), _p(by))
    return bx, by


def jacobi(g: Grid, bx, by, omega, sweeps, vx, vy):
    vx, vy = _f64(vx).copy(), _f64(vy).copy()
    lib().ora_jacobi(*g.head, _p(_f64(bx)), _p(_f64(by)), omega, sweeps, _p(vx), _p(vy))
    return vx, vy


def rbgs(g: Grid, bx, by, omega, sweeps, vx, vy):
    vx, vy = _f64(vx).copy(), _f64(vy).copy()
    lib().ora_rbgs(*g.head, _p(_f64(bx)), _p(_f64(by)), omega, sweeps, _p(vx), _p(vy))
    return vx, vy


def splitmix64(seed: int, c: int) -> int:
    return int(lib().ora_splitmix64(seed & (2**64 - 1), c & (2**64 - 1)))


def ras_shift(shift_mode, seed, t, ti, tj):
    out = (ctypes.c_int * 2)()
    lib().ora_ras_shift(shift_mode, seed & (2**64 - 1), t, ti, tj, out)
    return int(out[0]), int(out[1])


def ras(g: Grid, bx, by, omega, sweeps, ti, tj, k, overlap, shift_mode=1, seed=0, shifts=None, order_seed=0,
        vx=None, vy=None, return_counts=False):
    """RAS-Jacobi (Algorithm 2).  Returns (vx, vy) or (vx, vy, counts_x, counts_y)."""
    vx = g.zeros_vx() if vx is None else _f64(vx).copy()
    vy = g.zeros_vy() if vy is None else _f64(vy).copy()
    sh = None
    if shifts is not None:
        arr = np.ascontiguousarray(np.asarray(shifts, dtype=np.int32).reshape(-1))
        sh = arr.ctypes.data_as(_I)
    counts = np.zeros(vx.size + vy.size, dtype=np.int32) if return_counts else None
    st = lib().ora_ras(*g.head, _p(_f64(bx)), _p(_f64(by)), omega, sweeps, ti, tj, k, overlap, shift_mode,
                       seed & (2**64 - 1), sh, order_seed & (2**64 - 1), _p(vx), _p(vy),
                       None if counts is None else counts.ctypes.data_as(_I))
    if st != 0:
        raise ValueError("ora_ras: bad arguments")
    if return_counts:
        return vx, vy, counts[:vx.size].reshape(vx.shape), counts[vx.size:].reshape(vy.shape)
    return vx, vy


def ras_tiles(g: Grid, bx, by, omega, ti, tj, ksweeps, overlap, si, sj, tiles, vx, vy, out_x, out_y):
    """One RAS outer iteration on the listed tiles [(bx, by), ...] only; the
    owned unknowns of those tiles are written into copies of out_x/out_y."""
    vx, vy = _f64(vx), _f64(vy)
    ox, oy = _f64(out_x).copy(), _f64(out_y).copy()
    t = np.ascontiguousarray(np.asarray(tiles, dtype=np.int32).reshape(-1))
    st = lib().ora_ras_tiles(*g.head, _p(_f64(bx)), _p(_f64(by)), omega, ti, tj, ksweeps, overlap, si, sj,
                             t.ctypes.data_as(_I), len(t) // 2, _p(vx), _p(vy), _p(ox), _p(oy))
    if st != 0:
        raise ValueError("ora_ras_tiles: bad arguments")
    return ox, oy


def tile_count(n, T, s):
    return int(lib().ora_tile_count(n, T, s))


def energy(g: Grid, fx, fy, p, vx, vy):
    """(sum r_v^2/(-diag M), sum r_p^2 eta_c/(2/hx^2+2/hy^2), sum f^2/(-diag M))."""
    out = (ctypes.c_double * 3)()
    p = None if p is None else _f64(p)
    lib().ora_energy(*g.head, _p(_f64(fx)), _p(_f64(fy)), _p(p), _p(_f64(vx)), _p(_f64(vy)), out)
    return float(out[0]), float(out[1]), float(out[2])


def mg_levels(nx, ny, max_levels, coarsest):
    return int(lib().ora_mg_levels(nx, ny, max_levels, coarsest))


def mg_sweeps(nu0, growth, level, nu_max=0):
    return int(lib().ora_mg_sweeps(nu0, growth, level, nu_max))


def mg_prolong_add(nxf, nyf, cx, cy, fx, fy):
    fx, fy = _f64(fx).copy(), _f64(fy).copy()
    lib().ora_mg_prolong_add(nxf, nyf, _p(_f64(cx)), _p(_f64(cy)), _p(fx), _p(fy))
    return fx, fy


def mg_restrict(nxf, nyf, fx, fy):
    cx = np.zeros((nyf // 2, nxf // 2 + 1))
    cy = np.zeros((nyf // 2 + 1, nxf // 2))
    lib().ora_mg_restrict(nxf, nyf, _p(_f64(fx)), _p(_f64(fy)), _p(cx), _p(cy))
    return cx, cy


def dense_solve(g: Grid, bx, by):
    vx, vy = g.zeros_vx(), g.zeros_vy()
    st = lib().ora_dense_solve(*g.head, _p(_f64(bx)), _p(_f64(by)), _p(vx), _p(vy))
    if st != 0:
        raise ValueError("ora_dense_solve: -M is not positive definite")
    return vx, vy


@dataclass
class MG:
    """Multigrid settings (Sec. 6.2 defaults: 5 pre / 5 post sweeps, growth 2.5)."""
    max_levels: int = 16
    coarsest: int = 16
    nu_pre: int = 5
    nu_post: int = 5
    growth: float = 2.5
    nu_max: int = 0
    variant: int = 0
    omega: float = 0.3
    ti: int = 32
    tj: int = 32
    k: int = 4
    overlap: int = 3
    seed: int = 0

    def args(self):
        return (self.max_levels, self.coarsest, self.nu_pre, self.nu_post, self.growth, self.nu_max, self.variant,
                self.omega, self.ti, self.tj, self.k, self.overlap, self.seed & (2**64 - 1))


def vcycle(g: Grid, bx, by, mg: MG, vx=None, vy=None):
    vx = g.zeros_vx() if vx is None else _f64(vx).copy()
    vy = g.zeros_vy() if vy is None else _f64(vy).copy()
    st = lib().ora_vcycle(*g.head, _p(_f64(bx)), _p(_f64(by)), *mg.args(), _p(vx), _p(vy))
    if st != 0:
        raise ValueError("ora_vcycle failed")
    return vx, vy


def mg_solve(g: Grid, fx, fy, p, mg: MG, tol, max_cycles, vx=None, vy=None):
    """Defect-correction multigrid solve.  Returns (vx, vy, cycles, final_E, history)."""
    vx = g.zeros_vx() if vx is None else _f64(vx).copy()
    vy = g.zeros_vy() if vy is None else _f64(vy).copy()
    fe = ctypes.c_double(0.0)
    hist = np.zeros(max_cycles + 1)
    p = None if p is None else _f64(p)
    c = lib().ora_mg_solve(*g.head, _p(_f64(fx)), _p(_f64(fy)), _p(p), *mg.args(), tol, max_cycles, _p(vx), _p(vy),
                           ctypes.byref(fe), _p(hist))
    if c < 0:
        raise ValueError("ora_mg_solve failed")
    return vx, vy, c, fe.value, hist[:c + 1].copy()


def mg_fcg(g: Grid, fx, fy, p, mg: MG, tol, max_its, vx=None, vy=None):
    """Flexible CG preconditioned by one V-cycle.  Returns (vx, vy, its, final_E, history)."""
    vx = g.zeros_vx() if vx is None else _f64(vx).copy()
    vy = g.zeros_vy() if vy is None else _f64(vy).copy()
    fe = ctypes.c_double(0.0)
    hist = np.zeros(max_its + 1)
    p = None if p is None else _f64(p)
    c = lib().ora_mg_fcg(*g.head, _p(_f64(fx)), _p(_f64(fy)), _p(p), *mg.args(), tol, max_its, _p(vx), _p(vy),
                         ctypes.byref(fe), _p(hist))
    if c < 0:
        raise ValueError("ora_mg_fcg failed")
    return vx, vy, c, fe.value, hist[:c + 1].copy()


# ---------------------------------------------------------------------------
# inexact Uzawa iteration around the multigrid velocity solve (Sec. 3.1-3.2;
# solver configuration of Sec. 6.2)
# ---------------------------------------------------------------------------
def eta_min(eta_c, eta_n):
    """Smallest viscosity of the domain (Sec. 6.2): over the cells and the
    interior nodes (boundary nodes carry no shear stress and are ignored by
    the operator)."""
    return float(min(np.min(eta_c), np.min(np.asarray(eta_n)[1:-1, 1:-1])))


def blend_eta(eta_c, eta_n, theta, emin):
    """Viscosity continuation of Sec. 6.2: eta_comp = (1 - theta) eta_min +
    theta eta, at the cells and at the nodes."""
    return (1.0 - theta) * emin + theta * _f64(eta_c), (1.0 - theta) * emin + theta * _f64(eta_n)


def continuation_theta(cycle, interval, stages):
    """theta of Uzawa cycle `cycle` (from 0): 0, 1/(stages-1), ..., 1, one
    stage per `interval` cycles (Sec. 6.2: 0, 0.25, ..., 1 every 25 cycles);
    interval 0 means no continuation (theta = 1)."""
    if interval <= 0 or stages <= 1:
        return 1.0
    return min(cycle // interval, stages - 1) / (stages - 1)


def lithostatic(g: Grid, fy):
    """Initial pressure of Sec. 6.2, p = integral of rho g_y dy from the bottom,
    written discretely at the cell centres as p[0][i] = 0 and
    p[j][i] = p[j-1][i] + hy rho g_y at the vy face between them, with
    rho g_y = -f_y (reading: so that G p balances f_y exactly at every interior
    vy face), then shifted to zero mean."""
    fy = _f64(fy)
    p = np.zeros((g.ny, g.nx))
    for j in range(1, g.ny):
        p[j] = p[j - 1] - g.hy * fy[j]
    return p - p.mean()


def uzawa(g: Grid, fx, fy, mg: MG, cycles, omega_p=0.6, theta_interval=25, theta_stages=5, krylov=True, vel_its=1,
          p=None, vx=None, vy=None):
    """Inexact Uzawa iteration (Sec. 3.1-3.2, configuration of Sec. 6.2).

    Each cycle: the momentum solve M_theta v = f - G p from the current v
    (viscosity eta_theta of the continuation stage), with `vel_its`
    applications of the V-cycle: flexible-CG iterations preconditioned by it
    (krylov, the default: its first step is preconditioned steepest descent,
    which stays stable where the V-cycle is not a convergent splitting at
    high contrast) or defect-correction cycles (the paper's "single
    multigrid iteration" taken literally); the pressure update
    p <- p - omega_p eta_c,theta D v
    (reading: the paper's p + alpha eta D v with D taken with the sign that
    makes D M^-1 G positive, M being negative definite in the sign
    convention of Eq. (1)-(3); here D is the divergence); the pressure is
    shifted to zero mean (Sec. 6.2).  After every cycle the relative energy
    residual of Sec. 6.4 (velocity and pressure parts, true viscosity) is
    recorded.  Returns (vx, vy, p, history)."""
    vx = g.zeros_vx() if vx is None else _f64(vx).copy()
    vy = g.zeros_vy() if vy is None else _f64(vy).copy()
    p = lithostatic(g, fy) if p is None else _f64(p).copy()
    emin = eta_min(g.eta_c, g.eta_n)
    hist = []
    for c in range(cycles):
        theta = continuation_theta(c, theta_interval, theta_stages)
        ec, en = blend_eta(g.eta_c, g.eta_n, theta, emin)
        gc = Grid(g.nx, g.ny, g.hx, g.hy, ec, en)
        vx, vy, _, _, _ = (mg_fcg if krylov else mg_solve)(gc, fx, fy, p, mg, 0.0, vel_its, vx, vy)
        p = p - omega_p * ec * apply_D(g, vx, vy)
        p = p - p.mean()
        rv, rp, ff = energy(g, fx, fy, p, vx, vy)
        hist.append(float(np.sqrt((rv + rp) / ff)))
    return vx, vy, p, np.array(hist)


# ---------------------------------------------------------------------------
# Anderson acceleration of the inexact Uzawa iteration (Algorithm 1, Sec. 3.3)
# ---------------------------------------------------------------------------
def anderson_coefficients(R, reg=1e-14):
    """alpha = argmin ||R alpha||_2 subject to sum(alpha) = 1 for the columns of
    R (Algorithm 1), from the normal equations of the constrained problem:
    H y = 1 with H = R^T R (plus reg * max diag H on the diagonal, reading:
    keeps H invertible when residuals are nearly dependent), alpha = y / sum y."""
    R = np.asarray(R, dtype=np.float64)
    H = R.T @ R
    H = H + reg * max(float(np.max(np.diag(H))), 1e-300) * np.eye(H.shape[0])
    y = np.linalg.solve(H, np.ones(H.shape[0]))
    return y / y.sum()


def uzawa_map(g: Grid, fx, fy, mg: MG, vx, vy, p, theta, emin, omega_p=0.6, krylov=True, vel_its=1):
    """F(x) of Algorithm 1: one inexact Uzawa cycle (see uzawa) from
    x = (vx, vy, p) at continuation parameter theta."""
    ec, en = blend_eta(g.eta_c, g.eta_n, theta, emin)
    gc = Grid(g.nx, g.ny, g.hx, g.hy, ec, en)
    vx, vy, _, _, _ = (mg_fcg if krylov else mg_solve)(gc, fx, fy, p, mg, 0.0, vel_its, vx, vy)
    p = p - omega_p * ec * apply_D(g, vx, vy)
    return vx, vy, p - p.mean()


def anderson_uzawa(g: Grid, fx, fy, mg: MG, cycles, depth=5, omega_p=0.6, theta_interval=25, theta_stages=5,
                   krylov=True, vel_its=1, p=None, vx=None, vy=None, reg=1e-14):
    """Algorithm 1 on the inexact Uzawa map F over x = [v, p]: x1 = F(x0);
    then r_k = F(x_k) - x_k over the last min(depth, k) + 1 iterates,
    alpha = argmin ||R alpha||_2 with sum(alpha) = 1, and
    x_{k+1} = sum_i alpha_i F(x_i).  The 2-norm runs over every entry of vx,
    vy and p (walls and their residuals are zero).  Reading: F changes with
    the continuation stage, so the history restarts when theta changes.
    depth 0 is the plain iteration.  Returns (vx, vy, p, history of the
    relative energy residual after every cycle)."""
    vx = g.zeros_vx() if vx is None else _f64(vx).copy()
    vy = g.zeros_vy() if vy is None else _f64(vy).copy()
    p = lithostatic(g, fy) if p is None else _f64(p).copy()
    emin = eta_min(g.eta_c, g.eta_n)
    Fs, Rs, hist, stage = [], [], [], None
    for c in range(cycles):
        theta = continuation_theta(c, theta_interval, theta_stages)
        if theta != stage:
            Fs, Rs, stage = [], [], theta
        F = uzawa_map(g, fx, fy, mg, vx, vy, p, theta, emin, omega_p, krylov, vel_its)
        x = (vx, vy, p)
        Fs.append(F)
        Rs.append(np.concatenate([(a - b).ravel() for a, b in zip(F, x)]))
        Fs, Rs = Fs[-(depth + 1):], Rs[-(depth + 1):]
        if len(Rs) == 1 or depth == 0:
            vx, vy, p = F
        else:
            alpha = anderson_coefficients(np.stack(Rs, axis=1), reg)
            vx = sum(a * f[0] for a, f in zip(alpha, Fs))
            vy = sum(a * f[1] for a, f in zip(alpha, Fs))
            p = sum(a * f[2] for a, f in zip(alpha, Fs))
        rv, rp, ff = energy(g, fx, fy, p, vx, vy)
        hist.append(float(np.sqrt((rv + rp) / ff)))
    return vx, vy, p, np.array(hist)


def mg_refine(g: Grid, fx, fy, p, mg: MG, tol, max_cycles, inner_its, vx=None, vy=None):
    """Defect correction around inner flexible-CG solves (the outer loop of
    the precision pattern of Sec. 3.2 with FP32 sweeps): r = f - G p - M v;
    stop when E_v <= tol or max_cycles V-cycles were applied; else solve
    M e = r approximately by `inner_its` flexible-CG iterations from e = 0,
    each preconditioned by one V-cycle, and set v += e.  All FP64 here; the
    library runs the inner iterations in the V-cycle's precision.  Returns
    (vx, vy, V-cycles, final E_v, history of E_v per outer step)."""
    vx = g.zeros_vx() if vx is None else _f64(vx).copy()
    vy = g.zeros_vy() if vy is None else _f64(vy).copy()
    bx, by = rhs(g, fx, fy, p)
    dx, dy = diag_M(g)
    mx = np.zeros_like(dx, dtype=bool)
    mx[:, 1:g.nx] = True
    my = np.zeros_like(dy, dtype=bool)
    my[1:g.ny, :] = True
    den = np.sum(_f64(fx)[mx] ** 2 / -dx[mx]) + np.sum(_f64(fy)[my] ** 2 / -dy[my])
    hist, cycles = [], 0
    while True:
        ax, ay = apply_M(g, vx, vy)
        rx = np.where(mx, bx - ax, 0.0)
        ry = np.where(my, by - ay, 0.0)
        e = float(np.sqrt((np.sum(rx[mx] ** 2 / -dx[mx]) + np.sum(ry[my] ** 2 / -dy[my])) / den))
        hist.append(e)
        if e <= tol or cycles >= max_cycles:
            return vx, vy, cycles, e, np.array(hist)
        ex, ey, _, _, _ = mg_fcg(g, rx, ry, None, mg, 0.0, inner_its)
        vx = vx + ex
        vy = vy + ey
        cycles += inner_its


_lib_omp = None


def ras_all_cores(g: Grid, bx, by, omega, sweeps, ti, tj, k, overlap, shift_mode=1, seed=0):
    """ras() from the OpenMP build of the same source (the tiles of an outer
    iteration in parallel on every core the OpenMP runtime is given); the
    same result as ras().  For the all-cores CPU baseline only."""
    global _lib_omp
    if _lib_omp is None:
        from .build import build_oracle_omp
        _lib_omp = _bind(ctypes.CDLL(build_oracle_omp()))
    vx, vy = g.zeros_vx(), g.zeros_vy()
    st = _lib_omp.ora_ras(*g.head, _p(_f64(bx)), _p(_f64(by)), omega, sweeps, ti, tj, k, overlap, shift_mode,
                          seed & (2**64 - 1), None, 0, _p(vx), _p(vy), None)
    if st != 0:
        raise ValueError("ora_ras: bad arguments")
    return vx, vy
