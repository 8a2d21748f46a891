"""Thin Python binding of libstokes (include/stokes.h).

Functions carry the C names and only marshal arguments: device pointers come
from torch tensors, scalars are passed through, status codes become
StokesError.  Every step of the computation runs in the library's CUDA
kernels; there is no fallback, and a missing library raises.

Field tensors use the library layout: a (ny+1) x pitch array of the context's
dtype for every field (see stokes_get_layout); ``StokesContext.pack`` and
``unpack`` convert from and to the natural staggered shapes.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libstokes.so")

STOKES_OK = 0
STOKES_ERR_ARG = -1
STOKES_ERR_CUDA = -2
STOKES_ERR_OOM = -3
STOKES_ERR_DIVERGED = -4
STOKES_ERR_TIMEOUT = -5
STOKES_ERR_NOT_CONVERGED = -6
STOKES_ERR_STATE = -7

STOKES_F32, STOKES_F64 = 0, 1
STOKES_JACOBI, STOKES_JACOBI_FUSED, STOKES_JACOBI_BLOCKED, STOKES_RBGS, STOKES_RAS, STOKES_MIXED = 0, 1, 2, 3, 4, 5
STOKES_FIELD_VX, STOKES_FIELD_VY, STOKES_FIELD_P, STOKES_FIELD_ETA_C, STOKES_FIELD_ETA_N = 0, 1, 2, 3, 4
STOKES_SHIFT_NONE, STOKES_SHIFT_SPLITMIX, STOKES_SHIFT_LIST = 0, 1, 2
STOKES_OPT_USE_TMA, STOKES_OPT_WAIT_LIMIT_CYCLES, STOKES_OPT_PAIRED = 0, 1, 2
KERNEL_CLASSES = ["ras", "jacobi", "rbgs", "rhs", "energy", "copy", "apply", "mg"]

VARIANTS = {"jacobi": STOKES_JACOBI, "fused": STOKES_JACOBI_FUSED, "blocked": STOKES_JACOBI_BLOCKED,
            "rbgs": STOKES_RBGS, "ras": STOKES_RAS, "mixed": STOKES_MIXED}


class StokesError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = "%s: %s" % (where, _lib().stokes_strerror(status).decode())
        if status in (STOKES_ERR_CUDA, STOKES_ERR_OOM):
            msg += " (%s)" % _lib().stokes_last_cuda_error().decode()
        super().__init__(msg)


class stokes_smooth_params(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("sweeps", ctypes.c_int), ("tile_i", ctypes.c_int),
                ("tile_j", ctypes.c_int), ("k", ctypes.c_int), ("overlap", ctypes.c_int),
                ("omega", ctypes.c_double), ("seed", ctypes.c_uint64), ("shift_mode", ctypes.c_int),
                ("shifts", ctypes.POINTER(ctypes.c_int32))]


class stokes_mg_params(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("coarsest", ctypes.c_int), ("nu_pre", ctypes.c_int),
                ("nu_post", ctypes.c_int), ("nu_growth", ctypes.c_double), ("nu_max", ctypes.c_int),
                ("inner_dtype", ctypes.c_int), ("smoother", stokes_smooth_params), ("krylov", ctypes.c_int),
                ("tol", ctypes.c_double), ("max_cycles", ctypes.c_int), ("inner_its", ctypes.c_int)]


class stokes_uzawa_params(ctypes.Structure):
    _fields_ = [("mg", stokes_mg_params), ("omega_p", ctypes.c_double), ("cycles", ctypes.c_int),
                ("theta_interval", ctypes.c_int), ("theta_stages", ctypes.c_int), ("tol", ctypes.c_double),
                ("lithostatic_init", ctypes.c_int), ("anderson_depth", ctypes.c_int)]


class stokes3d_smooth_params(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("sweeps", ctypes.c_int), ("tile_i", ctypes.c_int),
                ("tile_j", ctypes.c_int), ("tile_k", ctypes.c_int), ("k", ctypes.c_int), ("overlap", ctypes.c_int),
                ("omega", ctypes.c_double), ("seed", ctypes.c_uint64), ("shift_mode", ctypes.c_int),
                ("shifts", ctypes.POINTER(ctypes.c_int32))]


_VP, _I, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
_SIGS = {
    "stokes_create": (_I, [_I, _I, _D, _D, _I, _VP, ctypes.POINTER(_VP)]),
    "stokes_get_layout": (_I, [_VP, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                               ctypes.POINTER(ctypes.c_size_t)]),
    "stokes_set_viscosity": (_I, [_VP, _VP, _VP]),
    "stokes_set_rhs": (_I, [_VP, _VP, _VP]),
    "stokes_apply_operator": (_I, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "stokes_smooth": (_I, [_VP, _VP, _VP, _VP, ctypes.POINTER(stokes_smooth_params)]),
    "stokes_residual_energy_norm": (_I, [_VP, _VP, _VP, _VP, ctypes.POINTER(_D)]),
    "stokes_vcycle": (_I, [_VP, _VP, _VP, _VP, ctypes.POINTER(stokes_mg_params), ctypes.POINTER(_D),
                           ctypes.POINTER(_I)]),
    "stokes_uzawa": (_I, [_VP, _VP, _VP, _VP, ctypes.POINTER(stokes_uzawa_params), ctypes.POINTER(_D),
                          ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "stokes_set_option": (_I, [_VP, _I, ctypes.c_longlong]),
    "stokes_synchronize": (_I, [_VP]),
    "stokes_tile_kernel_plan": (_I, [_I, _I, _I, _I, _I, _I, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_I),
                                     ctypes.POINTER(ctypes.c_size_t)]),
    "stokes_profile_reset": (_I, [_VP, _I]),
    "stokes_profile_read": (_I, [_VP, _I, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                                 ctypes.POINTER(_D)]),
    "stokes_energy_norm_noalloc": (_I, [_I, _I, _D, _D, _I, _I, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "stokes_batch_create": (_I, [_I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_D), ctypes.POINTER(_D),
                                 _I, _VP, ctypes.POINTER(_VP)]),
    "stokes_batch_get_layout": (_I, [_VP, _I, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_size_t),
                                     ctypes.POINTER(ctypes.c_size_t)]),
    "stokes_batch_set_viscosity": (_I, [_VP, _VP, _VP]),
    "stokes_batch_set_rhs": (_I, [_VP, _VP, _VP]),
    "stokes_batch_smooth": (_I, [_VP, _VP, _VP, _VP, ctypes.POINTER(stokes_smooth_params)]),
    "stokes_batch_residual_energy": (_I, [_VP, _VP, _VP, _VP, ctypes.POINTER(_D)]),
    "stokes_batch_solve": (_I, [_VP, _VP, _VP, _VP, ctypes.POINTER(stokes_mg_params), ctypes.POINTER(_D),
                                ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "stokes_batch_kernels": (_I, [_VP, ctypes.POINTER(ctypes.c_longlong)]),
    "stokes_batch_set_option": (_I, [_VP, _I, ctypes.c_longlong]),
    "stokes_batch_destroy": (_I, [_VP]),
    "stokes_slab_plan": (_I, [_I, _I, _I, _I, _I, ctypes.POINTER(_I)]),
    "stokes_slabs_create": (_I, [_I, _I, _D, _D, _I, _I, _VP, ctypes.POINTER(_VP)]),
    "stokes_slabs_set_viscosity": (_I, [_VP, _VP, _VP]),
    "stokes_slabs_set_rhs": (_I, [_VP, _VP, _VP]),
    "stokes_slabs_smooth": (_I, [_VP, _VP, _VP, _VP, ctypes.POINTER(stokes_smooth_params)]),
    "stokes_slabs_exchanges": (_I, [_VP, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
    "stokes_slabs_destroy": (_I, [_VP]),
    "stokes3d_create": (_I, [_I, _I, _I, _D, _D, _D, _I, _VP, ctypes.POINTER(_VP)]),
    "stokes3d_get_layout": (_I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_size_t)]),
    "stokes3d_set_viscosity": (_I, [_VP, _VP, _VP, _VP, _VP]),
    "stokes3d_set_rhs": (_I, [_VP, _VP, _VP, _VP]),
    "stokes3d_apply_operator": (_I, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "stokes3d_smooth": (_I, [_VP, _VP, _VP, _VP, _VP, ctypes.POINTER(stokes3d_smooth_params)]),
    "stokes3d_residual_energy_norm": (_I, [_VP, _VP, _VP, _VP, _VP, ctypes.POINTER(_D)]),
    "stokes3d_kernels": (_I, [_VP, ctypes.POINTER(ctypes.c_longlong)]),
    "stokes3d_destroy": (_I, [_VP]),
    "stokes_destroy": (_I, [_VP]),
    "stokes_strerror": (ctypes.c_char_p, [_I]),
    "stokes_last_cuda_error": (ctypes.c_char_p, []),
}

_handle = None


def _lib():
    """Load libstokes.so (built in place by paper_2509_19061_gb300.build)."""
    global _handle
    if _handle is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libstokes.so is not built (%s); run paper_2509_19061_gb300.build.build()" % LIB_PATH)
        h = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(h, name)
            fn.restype = res
            fn.argtypes = args
        _handle = h
    return _handle


def exported_symbols():
    return list(_SIGS)


def _check(status, where):
    if status != STOKES_OK:
        raise StokesError(status, where)
    return status


def _ptr(t):
    """Device pointer of a torch tensor (None -> NULL)."""
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


# --------------------------------------------------------------------------
# C-named entry points
# --------------------------------------------------------------------------
def stokes_create(nx, ny, lx, ly, dtype, cuda_stream=None):
    out = ctypes.c_void_p()
    stream = ctypes.c_void_p(cuda_stream) if cuda_stream else None
    _check(_lib().stokes_create(nx, ny, lx, ly, dtype, stream, ctypes.byref(out)), "stokes_create")
    return out


def stokes_get_layout(ctx, field):
    r, c, p = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    n = ctypes.c_size_t()
    _check(_lib().stokes_get_layout(ctx, field, ctypes.byref(r), ctypes.byref(c), ctypes.byref(p), ctypes.byref(n)),
           "stokes_get_layout")
    return r.value, c.value, p.value, n.value


def stokes_set_viscosity(ctx, eta_c, eta_n):
    _check(_lib().stokes_set_viscosity(ctx, _ptr(eta_c), _ptr(eta_n)), "stokes_set_viscosity")


def stokes_set_rhs(ctx, fx, fy):
    _check(_lib().stokes_set_rhs(ctx, _ptr(fx), _ptr(fy)), "stokes_set_rhs")


def stokes_apply_operator(ctx, vx, vy, p, out_x, out_y):
    _check(_lib().stokes_apply_operator(ctx, _ptr(vx), _ptr(vy), _ptr(p), _ptr(out_x), _ptr(out_y)),
           "stokes_apply_operator")


def smooth_params(variant="ras", sweeps=1, tile=(32, 32), k=4, overlap=None, omega=0.3, seed=0, shift_mode=None,
                  shifts=None):
    """Build a stokes_smooth_params.  overlap=None means k-1 (exact temporal
    blocking); shift_mode defaults to SplitMix64 shifts for RAS."""
    v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    if overlap is None:
        overlap = max(k - 1, 0)
    if shift_mode is None:
        shift_mode = STOKES_SHIFT_LIST if shifts is not None else STOKES_SHIFT_SPLITMIX
    p = stokes_smooth_params(v, sweeps, tile[0], tile[1], k, overlap, omega, seed & (2**64 - 1), shift_mode, None)
    if shifts is not None:
        arr = np.ascontiguousarray(np.asarray(shifts, dtype=np.int32).reshape(-1))
        p._shifts_keepalive = arr
        p.shifts = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    return p


def mg_params(levels=16, coarsest=16, nu_pre=5, nu_post=5, nu_growth=2.5, nu_max=0, inner="f32", krylov=True,
              tol=1e-8, max_cycles=100, inner_its=0, **smoother):
    """Build a stokes_mg_params (Sec. 6.2 defaults: 5/5 sweeps, growth 2.5).
    krylov: False / True (0 / 1) or 2 (defect correction around inner_its
    flexible-CG iterations in the inner precision)."""
    smoother.setdefault("variant", "ras")
    sm = smooth_params(**smoother)
    inner_code = STOKES_F64 if inner in ("f64", "float64") else STOKES_F32
    kr = int(krylov) if not isinstance(krylov, bool) else (1 if krylov else 0)
    return stokes_mg_params(levels, coarsest, nu_pre, nu_post, nu_growth, nu_max, inner_code, sm, kr, tol,
                            max_cycles, inner_its)


def stokes_smooth(ctx, vx, vy, p, params):
    _check(_lib().stokes_smooth(ctx, _ptr(vx), _ptr(vy), _ptr(p), ctypes.byref(params)), "stokes_smooth")


def stokes_residual_energy_norm(ctx, vx, vy, p=None):
    out = (ctypes.c_double * 3)()
    _check(_lib().stokes_residual_energy_norm(ctx, _ptr(vx), _ptr(vy), _ptr(p), out), "stokes_residual_energy_norm")
    return float(out[0]), float(out[1]), float(out[2])


def stokes_vcycle(ctx, vx, vy, p, params):
    """Returns (status, final_rel_resid, cycles); raises on errors other than
    STOKES_ERR_NOT_CONVERGED."""
    fr, cy = ctypes.c_double(0.0), ctypes.c_int(0)
    st = _lib().stokes_vcycle(ctx, _ptr(vx), _ptr(vy), _ptr(p), ctypes.byref(params), ctypes.byref(fr),
                              ctypes.byref(cy))
    if st not in (STOKES_OK, STOKES_ERR_NOT_CONVERGED):
        raise StokesError(st, "stokes_vcycle")
    return st, fr.value, cy.value


def uzawa_params(cycles=100, omega_p=0.6, theta_interval=25, theta_stages=5, tol=0.0, lithostatic_init=True,
                 vel_its=1, anderson=0, **mg):
    """Build a stokes_uzawa_params (Sec. 6.2 defaults: omega_p 0.6, continuation
    in 5 stages of 25 cycles); vel_its V-cycles (CG iterations) per cycle;
    anderson = depth of the Anderson acceleration (0 off)."""
    m = mg_params(max_cycles=vel_its, **mg)
    return stokes_uzawa_params(m, omega_p, cycles, theta_interval, theta_stages, tol, 1 if lithostatic_init else 0,
                               anderson)


def stokes_uzawa(ctx, vx, vy, p, params):
    """Returns (status, history, cycles, final E); raises on errors other than
    STOKES_ERR_NOT_CONVERGED."""
    hist = (_D * max(params.cycles, 1))()
    cy, fe = _I(0), _D(0.0)
    st = _lib().stokes_uzawa(ctx, _ptr(vx), _ptr(vy), _ptr(p), ctypes.byref(params), hist, ctypes.byref(cy),
                             ctypes.byref(fe))
    if st not in (STOKES_OK, STOKES_ERR_NOT_CONVERGED):
        raise StokesError(st, "stokes_uzawa")
    return st, np.array(hist[:cy.value]), cy.value, fe.value


def stokes_set_option(ctx, option, value):
    _check(_lib().stokes_set_option(ctx, option, int(value)), "stokes_set_option")


def stokes_synchronize(ctx):
    _check(_lib().stokes_synchronize(ctx), "stokes_synchronize")


TILE_KERNELS = {0: "tma", 1: "global", 2: "shared", 3: "pair"}


def stokes_tile_kernel_plan(nx, ny, tile, overlap, dtype="f32", use_tma=True, pair_mode=1):
    """(kernel name, CTA threads, dynamic shared bytes) of a tile-smoother launch."""
    kern, thr, smem = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
    code = STOKES_F64 if dtype in ("f64", "float64") else STOKES_F32
    _check(_lib().stokes_tile_kernel_plan(nx, ny, tile[0], tile[1], overlap, code, 1 if use_tma else 0,
                                          int(pair_mode), ctypes.byref(kern), ctypes.byref(thr),
                                          ctypes.byref(smem)), "stokes_tile_kernel_plan")
    return TILE_KERNELS[kern.value], thr.value, smem.value


def stokes_profile_reset(ctx, enable_timing):
    _check(_lib().stokes_profile_reset(ctx, 1 if enable_timing else 0), "stokes_profile_reset")


def stokes_profile_read(ctx, kind):
    """Returns (kernel launches, timed launch groups, total ms) of one class."""
    k, g, ms = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_double()
    _check(_lib().stokes_profile_read(ctx, kind, ctypes.byref(k), ctypes.byref(g), ctypes.byref(ms)),
           "stokes_profile_read")
    return k.value, g.value, ms.value


def stokes_energy_norm_noalloc(nx, ny, lx, ly, dtype, pitch, eta_c, eta_n, fx, fy, p, vx, vy, out_dev,
                               cuda_stream=None):
    """Energy sums into the device tensor out_dev (3 float64) without any
    allocation by the library; asynchronous on cuda_stream."""
    stream = ctypes.c_void_p(cuda_stream) if cuda_stream else None
    _check(_lib().stokes_energy_norm_noalloc(nx, ny, lx, ly, dtype, pitch, _ptr(eta_c), _ptr(eta_n), _ptr(fx),
                                             _ptr(fy), _ptr(p), _ptr(vx), _ptr(vy), _ptr(out_dev), stream),
           "stokes_energy_norm_noalloc")


def stokes_destroy(ctx):
    if ctx is not None:
        _check(_lib().stokes_destroy(ctx), "stokes_destroy")


def stokes_batch_create(nx, ny, lx, ly, dtype, cuda_stream=None):
    n = len(nx)
    out = ctypes.c_void_p()
    stream = ctypes.c_void_p(cuda_stream) if cuda_stream else None
    _check(_lib().stokes_batch_create(n, (_I * n)(*nx), (_I * n)(*ny), (_D * n)(*lx), (_D * n)(*ly), dtype, stream,
                                      ctypes.byref(out)), "stokes_batch_create")
    return out


def stokes_batch_get_layout(b, inst):
    """(pitch, offset, elements) of instance inst; inst = -1: (0, 0, slab size)."""
    pitch, off, n = _I(), ctypes.c_size_t(), ctypes.c_size_t()
    _check(_lib().stokes_batch_get_layout(b, inst, ctypes.byref(pitch), ctypes.byref(off), ctypes.byref(n)),
           "stokes_batch_get_layout")
    return pitch.value, off.value, n.value


def stokes_batch_set_viscosity(b, eta_c, eta_n):
    _check(_lib().stokes_batch_set_viscosity(b, _ptr(eta_c), _ptr(eta_n)), "stokes_batch_set_viscosity")


def stokes_batch_set_rhs(b, fx, fy):
    _check(_lib().stokes_batch_set_rhs(b, _ptr(fx), _ptr(fy)), "stokes_batch_set_rhs")


def stokes_batch_smooth(b, vx, vy, p, params):
    _check(_lib().stokes_batch_smooth(b, _ptr(vx), _ptr(vy), _ptr(p), ctypes.byref(params)), "stokes_batch_smooth")


def stokes_batch_residual_energy(b, count, vx, vy, p=None):
    out = (_D * (2 * count))()
    _check(_lib().stokes_batch_residual_energy(b, _ptr(vx), _ptr(vy), _ptr(p), out), "stokes_batch_residual_energy")
    return np.array(out[:], dtype=np.float64).reshape(count, 2)


def stokes_batch_solve(b, count, vx, vy, p, params):
    """Returns (status, E_v per instance, cycles per instance, status per
    instance); raises on errors other than STOKES_ERR_NOT_CONVERGED and
    STOKES_ERR_DIVERGED."""
    fe, cy, ss = (_D * count)(), (_I * count)(), (_I * count)()
    st = _lib().stokes_batch_solve(b, _ptr(vx), _ptr(vy), _ptr(p), ctypes.byref(params), fe, cy, ss)
    if st not in (STOKES_OK, STOKES_ERR_NOT_CONVERGED, STOKES_ERR_DIVERGED):
        raise StokesError(st, "stokes_batch_solve")
    return st, np.array(fe[:]), np.array(cy[:], dtype=np.int64), np.array(ss[:], dtype=np.int64)


def stokes_batch_set_option(b, option, value):
    _check(_lib().stokes_batch_set_option(b, option, int(value)), "stokes_batch_set_option")


def stokes_batch_kernels(b):
    k = ctypes.c_longlong()
    _check(_lib().stokes_batch_kernels(b, ctypes.byref(k)), "stokes_batch_kernels")
    return k.value


def stokes_batch_destroy(b):
    if b is not None:
        _check(_lib().stokes_batch_destroy(b), "stokes_batch_destroy")


def stokes_slab_plan(ny, nslabs, tile_j, overlap, slab):
    """(r0, r1, R0, R1): own and stored cell rows of one slab (host only)."""
    out = (_I * 4)()
    _check(_lib().stokes_slab_plan(ny, nslabs, tile_j, overlap, slab, out), "stokes_slab_plan")
    return tuple(out)


def stokes_slabs_create(nx, ny, lx, ly, dtype, nslabs, cuda_stream=None):
    out = ctypes.c_void_p()
    stream = ctypes.c_void_p(cuda_stream) if cuda_stream else None
    _check(_lib().stokes_slabs_create(nx, ny, lx, ly, dtype, nslabs, stream, ctypes.byref(out)),
           "stokes_slabs_create")
    return out


def stokes_slabs_set_viscosity(s, eta_c, eta_n):
    _check(_lib().stokes_slabs_set_viscosity(s, _ptr(eta_c), _ptr(eta_n)), "stokes_slabs_set_viscosity")


def stokes_slabs_set_rhs(s, fx, fy):
    _check(_lib().stokes_slabs_set_rhs(s, _ptr(fx), _ptr(fy)), "stokes_slabs_set_rhs")


def stokes_slabs_smooth(s, vx, vy, p, params):
    _check(_lib().stokes_slabs_smooth(s, _ptr(vx), _ptr(vy), _ptr(p), ctypes.byref(params)), "stokes_slabs_smooth")


def stokes_slabs_exchanges(s):
    c, b = ctypes.c_longlong(), ctypes.c_longlong()
    _check(_lib().stokes_slabs_exchanges(s, ctypes.byref(c), ctypes.byref(b)), "stokes_slabs_exchanges")
    return c.value, b.value


def stokes_slabs_destroy(s):
    if s is not None:
        _check(_lib().stokes_slabs_destroy(s), "stokes_slabs_destroy")


def stokes3d_create(nx, ny, nz, lx, ly, lz, dtype, cuda_stream=None):
    out = ctypes.c_void_p()
    stream = ctypes.c_void_p(cuda_stream) if cuda_stream else None
    _check(_lib().stokes3d_create(nx, ny, nz, lx, ly, lz, dtype, stream, ctypes.byref(out)), "stokes3d_create")
    return out


def stokes3d_get_layout(ctx):
    """(pitch, rows per plane, elements of one field buffer)."""
    p, r, n = _I(), _I(), ctypes.c_size_t()
    _check(_lib().stokes3d_get_layout(ctx, ctypes.byref(p), ctypes.byref(r), ctypes.byref(n)), "stokes3d_get_layout")
    return p.value, r.value, n.value


def stokes3d_set_viscosity(ctx, eta_c, eta_xy, eta_xz, eta_yz):
    _check(_lib().stokes3d_set_viscosity(ctx, _ptr(eta_c), _ptr(eta_xy), _ptr(eta_xz), _ptr(eta_yz)),
           "stokes3d_set_viscosity")


def stokes3d_set_rhs(ctx, fx, fy, fz):
    _check(_lib().stokes3d_set_rhs(ctx, _ptr(fx), _ptr(fy), _ptr(fz)), "stokes3d_set_rhs")


def stokes3d_apply_operator(ctx, vx, vy, vz, p, ox, oy, oz):
    _check(_lib().stokes3d_apply_operator(ctx, _ptr(vx), _ptr(vy), _ptr(vz), _ptr(p), _ptr(ox), _ptr(oy), _ptr(oz)),
           "stokes3d_apply_operator")


def smooth3d_params(variant="ras", sweeps=1, tile=(8, 8, 8), k=2, overlap=None, omega=0.3, seed=0, shift_mode=None,
                    shifts=None):
    """Build a stokes3d_smooth_params (overlap=None means k-1)."""
    v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    if overlap is None:
        overlap = max(k - 1, 0)
    if shift_mode is None:
        shift_mode = STOKES_SHIFT_LIST if shifts is not None else STOKES_SHIFT_SPLITMIX
    prm = stokes3d_smooth_params(v, sweeps, tile[0], tile[1], tile[2], k, overlap, omega, seed & (2**64 - 1),
                                 shift_mode, None)
    if shifts is not None:
        arr = np.ascontiguousarray(np.asarray(shifts, dtype=np.int32).reshape(-1))
        prm._shifts_keepalive = arr
        prm.shifts = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    return prm


def stokes3d_smooth(ctx, vx, vy, vz, p, params):
    _check(_lib().stokes3d_smooth(ctx, _ptr(vx), _ptr(vy), _ptr(vz), _ptr(p), ctypes.byref(params)),
           "stokes3d_smooth")


def stokes3d_residual_energy_norm(ctx, vx, vy, vz, p=None):
    out = (ctypes.c_double * 3)()
    _check(_lib().stokes3d_residual_energy_norm(ctx, _ptr(vx), _ptr(vy), _ptr(vz), _ptr(p), out),
           "stokes3d_residual_energy_norm")
    return float(out[0]), float(out[1]), float(out[2])


def stokes3d_kernels(ctx):
    k = ctypes.c_longlong()
    _check(_lib().stokes3d_kernels(ctx, ctypes.byref(k)), "stokes3d_kernels")
    return k.value


def stokes3d_destroy(ctx):
    if ctx is not None:
        _check(_lib().stokes3d_destroy(ctx), "stokes3d_destroy")


# --------------------------------------------------------------------------
# convenience wrapper with torch tensors
# --------------------------------------------------------------------------
_FIELD_OF = {"vx": STOKES_FIELD_VX, "fx": STOKES_FIELD_VX, "vy": STOKES_FIELD_VY, "fy": STOKES_FIELD_VY,
             "p": STOKES_FIELD_P, "eta_c": STOKES_FIELD_ETA_C, "eta_n": STOKES_FIELD_ETA_N}


class StokesContext:
    """Owns a stokes_ctx; allocates and converts field tensors."""

    def __init__(self, nx, ny, lx=1.0, ly=1.0, dtype="f64", device="cuda", stream=None):
        import torch
        self.torch = torch
        self.nx, self.ny, self.lx, self.ly = nx, ny, lx, ly
        self.dtype_code = STOKES_F64 if dtype in ("f64", "float64", torch.float64) else STOKES_F32
        self.tdtype = torch.float64 if self.dtype_code == STOKES_F64 else torch.float32
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.ctx = stokes_create(nx, ny, lx, ly, self.dtype_code, self.stream.cuda_stream)
        _, _, self.pitch, self.alloc = stokes_get_layout(self.ctx, STOKES_FIELD_VX)
        self.shape = {name: stokes_get_layout(self.ctx, f)[:2] for name, f in _FIELD_OF.items()}

    def close(self):
        if self.ctx is not None:
            stokes_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def field(self):
        return self.torch.zeros((self.ny + 1, self.pitch), dtype=self.tdtype, device=self.device)

    def pack(self, arr, name, out=None):
        """Natural-shape array -> library-layout device tensor (padding zero)."""
        r, c = self.shape[name]
        a = np.asarray(arr)
        assert a.shape == (r, c), "%s: expected %s, got %s" % (name, (r, c), a.shape)
        host = self.torch.zeros((self.ny + 1, self.pitch), dtype=self.tdtype)
        host[:r, :c] = self.torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(self.tdtype)
        if out is None:
            return host.to(self.device)
        out.copy_(host)
        return out

    def unpack(self, t, name):
        r, c = self.shape[name]
        return t[:r, :c].double().cpu().numpy()

    def set_problem(self, prob):
        """Viscosity and body force of an inputs.Problem."""
        ec, en = self.pack(prob.eta_c, "eta_c"), self.pack(prob.eta_n, "eta_n")
        fx, fy = self.pack(prob.fx, "fx"), self.pack(prob.fy, "fy")
        stokes_set_viscosity(self.ctx, ec, en)
        stokes_set_rhs(self.ctx, fx, fy)

    def set_viscosity_dev(self, eta_c, eta_n):
        """Viscosity from tensors already in the library layout."""
        stokes_set_viscosity(self.ctx, eta_c, eta_n)

    def set_rhs_dev(self, fx, fy):
        stokes_set_rhs(self.ctx, fx, fy)

    def set_viscosity(self, eta_c, eta_n):
        stokes_set_viscosity(self.ctx, self.pack(eta_c, "eta_c"), self.pack(eta_n, "eta_n"))

    def set_rhs(self, fx, fy):
        stokes_set_rhs(self.ctx, self.pack(fx, "fx"), self.pack(fy, "fy"))

    def smooth(self, vx, vy, p=None, **kw):
        stokes_smooth(self.ctx, vx, vy, p, smooth_params(**kw))

    def apply(self, vx, vy, p=None):
        ox, oy = self.field(), self.field()
        stokes_apply_operator(self.ctx, vx, vy, p, ox, oy)
        return ox, oy

    def energy(self, vx, vy, p=None):
        return stokes_residual_energy_norm(self.ctx, vx, vy, p)

    def set_option(self, option, value):
        stokes_set_option(self.ctx, option, value)

    def synchronize(self):
        stokes_synchronize(self.ctx)

    def vcycle(self, vx, vy, p=None, **kw):
        """Defect-correction multigrid solve; returns (status, E_v, cycles)."""
        return stokes_vcycle(self.ctx, vx, vy, p, mg_params(**kw))

    def uzawa(self, vx, vy, p, **kw):
        """Inexact Uzawa solve; returns (status, history, cycles, final E)."""
        return stokes_uzawa(self.ctx, vx, vy, p, uzawa_params(**kw))

    def profile_reset(self, timing=False):
        stokes_profile_reset(self.ctx, timing)

    def profile(self):
        """{class: (kernel launches, timed groups, total ms)}"""
        return {name: stokes_profile_read(self.ctx, i) for i, name in enumerate(KERNEL_CLASSES)}


class BatchContext:
    """Owns a stokes_batch: instance i is an nx[i] x ny[i] grid; every field is
    one slab tensor holding all instances (see stokes_batch_get_layout)."""

    def __init__(self, nx, ny, lx=None, ly=None, dtype="f64", device="cuda", stream=None):
        import torch
        self.torch = torch
        self.count = len(nx)
        self.nx, self.ny = list(nx), list(ny)
        self.lx = list(lx) if lx is not None else [1.0] * self.count
        self.ly = list(ly) if ly is not None else [1.0] * self.count
        self.dtype_code = STOKES_F64 if dtype in ("f64", "float64", torch.float64) else STOKES_F32
        self.tdtype = torch.float64 if self.dtype_code == STOKES_F64 else torch.float32
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.b = stokes_batch_create(self.nx, self.ny, self.lx, self.ly, self.dtype_code, self.stream.cuda_stream)
        self.total = stokes_batch_get_layout(self.b, -1)[2]
        self.layout = [stokes_batch_get_layout(self.b, i) for i in range(self.count)]

    def close(self):
        if self.b is not None:
            stokes_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def slab(self):
        return self.torch.zeros(self.total, dtype=self.tdtype, device=self.device)

    def view(self, slab, i):
        """Instance i of a slab as its (ny+1) x pitch array."""
        pitch, off, n = self.layout[i]
        return slab[off:off + n].view(self.ny[i] + 1, pitch)

    def _shape(self, name, i):
        nx, ny = self.nx[i], self.ny[i]
        return {"vx": (ny, nx + 1), "fx": (ny, nx + 1), "vy": (ny + 1, nx), "fy": (ny + 1, nx), "p": (ny, nx),
                "eta_c": (ny, nx), "eta_n": (ny + 1, nx + 1)}[name]

    def pack(self, arrs, name):
        """List of natural-shape arrays (one per instance) -> slab tensor."""
        host = self.torch.zeros(self.total, dtype=self.tdtype)
        for i, a in enumerate(arrs):
            r, c = self._shape(name, i)
            a = np.asarray(a)
            assert a.shape == (r, c), "%s[%d]: expected %s, got %s" % (name, i, (r, c), a.shape)
            pitch, off, n = self.layout[i]
            v = host[off:off + n].view(self.ny[i] + 1, pitch)
            v[:r, :c] = self.torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(self.tdtype)
        return host.to(self.device)

    def unpack(self, slab, name, i):
        r, c = self._shape(name, i)
        return self.view(slab, i)[:r, :c].double().cpu().numpy()

    def set_problems(self, probs):
        stokes_batch_set_viscosity(self.b, self.pack([q.eta_c for q in probs], "eta_c"),
                                   self.pack([q.eta_n for q in probs], "eta_n"))
        stokes_batch_set_rhs(self.b, self.pack([q.fx for q in probs], "fx"), self.pack([q.fy for q in probs], "fy"))

    def smooth(self, vx, vy, p=None, **kw):
        stokes_batch_smooth(self.b, vx, vy, p, smooth_params(**kw))

    def energy(self, vx, vy, p=None):
        """(count, 2): sum r^2/(-diag M), sum f^2/(-diag M) per instance."""
        return stokes_batch_residual_energy(self.b, self.count, vx, vy, p)

    def solve(self, vx, vy, p=None, **kw):
        """Returns (status, E_v[], cycles[], status[])."""
        return stokes_batch_solve(self.b, self.count, vx, vy, p, mg_params(**kw))

    def kernels(self):
        return stokes_batch_kernels(self.b)

    def set_option(self, option, value):
        stokes_batch_set_option(self.b, option, value)


class SlabContext:
    """Owns a stokes_slabs set; field tensors use the single-context layout
    (StokesContext.pack / unpack of the same grid)."""

    def __init__(self, nx, ny, lx=1.0, ly=1.0, dtype="f64", nslabs=2, device="cuda", stream=None):
        import torch
        self.torch = torch
        self.nx, self.ny, self.nslabs = nx, ny, nslabs
        self.dtype_code = STOKES_F64 if dtype in ("f64", "float64", torch.float64) else STOKES_F32
        self.stream = stream if stream is not None else torch.cuda.current_stream(torch.device(device))
        self.s = stokes_slabs_create(nx, ny, lx, ly, self.dtype_code, nslabs, self.stream.cuda_stream)

    def close(self):
        if self.s is not None:
            stokes_slabs_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_viscosity_dev(self, eta_c, eta_n):
        stokes_slabs_set_viscosity(self.s, eta_c, eta_n)

    def set_rhs_dev(self, fx, fy):
        stokes_slabs_set_rhs(self.s, fx, fy)

    def smooth(self, vx, vy, p=None, **kw):
        kw.setdefault("variant", "ras")
        stokes_slabs_smooth(self.s, vx, vy, p, smooth_params(**kw))

    def exchanges(self):
        return stokes_slabs_exchanges(self.s)


class Stokes3DContext:
    """Owns a stokes3d_ctx; allocates field tensors in the library layout
    ((nz+1) x (ny+1) x pitch) and converts from and to the natural [k][j][i]
    staggered shapes."""

    def __init__(self, nx, ny, nz, lx=1.0, ly=1.0, lz=1.0, dtype="f64", device="cuda", stream=None):
        import torch
        self.torch = torch
        self.nx, self.ny, self.nz = nx, ny, nz
        self.lx, self.ly, self.lz = lx, ly, lz
        self.dtype_code = STOKES_F64 if dtype in ("f64", "float64", torch.float64) else STOKES_F32
        self.tdtype = torch.float64 if self.dtype_code == STOKES_F64 else torch.float32
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.ctx = stokes3d_create(nx, ny, nz, lx, ly, lz, self.dtype_code, self.stream.cuda_stream)
        self.pitch, _, self.alloc = stokes3d_get_layout(self.ctx)
        self.shape = {"vx": (nz, ny, nx + 1), "vy": (nz, ny + 1, nx), "vz": (nz + 1, ny, nx), "p": (nz, ny, nx),
                      "eta_c": (nz, ny, nx), "eta_xy": (nz, ny + 1, nx + 1), "eta_xz": (nz + 1, ny, nx + 1),
                      "eta_yz": (nz + 1, ny + 1, nx)}
        for a, b in (("fx", "vx"), ("fy", "vy"), ("fz", "vz")):
            self.shape[a] = self.shape[b]

    def close(self):
        if self.ctx is not None:
            stokes3d_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def field(self):
        return self.torch.zeros((self.nz + 1, self.ny + 1, self.pitch), dtype=self.tdtype, device=self.device)

    def pack(self, arr, name):
        r = self.shape[name]
        a = np.asarray(arr)
        assert a.shape == r, "%s: expected %s, got %s" % (name, r, a.shape)
        host = self.torch.zeros((self.nz + 1, self.ny + 1, self.pitch), dtype=self.tdtype)
        host[:r[0], :r[1], :r[2]] = self.torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(self.tdtype)
        return host.to(self.device)

    def unpack(self, t, name):
        r = self.shape[name]
        return t[:r[0], :r[1], :r[2]].double().cpu().numpy()

    def set_problem(self, prob):
        stokes3d_set_viscosity(self.ctx, self.pack(prob.eta_c, "eta_c"), self.pack(prob.eta_xy, "eta_xy"),
                               self.pack(prob.eta_xz, "eta_xz"), self.pack(prob.eta_yz, "eta_yz"))
        stokes3d_set_rhs(self.ctx, self.pack(prob.fx, "fx"), self.pack(prob.fy, "fy"), self.pack(prob.fz, "fz"))

    def set_viscosity(self, eta_c, eta_xy, eta_xz, eta_yz):
        stokes3d_set_viscosity(self.ctx, self.pack(eta_c, "eta_c"), self.pack(eta_xy, "eta_xy"),
                               self.pack(eta_xz, "eta_xz"), self.pack(eta_yz, "eta_yz"))

    def apply(self, vx, vy, vz, p=None):
        out = (self.field(), self.field(), self.field())
        stokes3d_apply_operator(self.ctx, vx, vy, vz, p, *out)
        return out

    def smooth(self, vx, vy, vz, p=None, **kw):
        stokes3d_smooth(self.ctx, vx, vy, vz, p, smooth3d_params(**kw))

    def energy(self, vx, vy, vz, p=None):
        return stokes3d_residual_energy_norm(self.ctx, vx, vy, vz, p)

    def kernels(self):
        return stokes3d_kernels(self.ctx)
