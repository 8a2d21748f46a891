// mg.h -- geometric multigrid hierarchy of a context (internal).
#pragma once

#include <cuda_runtime.h>

#include "../../include/stokes.h"
#include "internal.h"

namespace stokes {

// One level of the hierarchy: every field is (ny+1) x pitch of the inner
// precision, including ivx/ivy = 1/diag(M) at the unknowns.
struct MgLevel {
    int nx, ny, pitch;
    size_t elems;
    double hx, hy;
    void *ec, *en, *ivx, *ivy, *bx, *by, *vx, *vy, *rx, *ry, *sx, *sy;
};

struct MgHierarchy;

// What the V-cycle needs from the context (outer precision `dtype`).
struct MgOuter {
    int nx, ny, pitch, dtype;
    double hx, hy;
    const void *eta_c, *eta_n; // context copies (boundary nodes of eta_n zeroed)
    const void *bx, *by;       // b = f - G p
};

// Mark the hierarchy stale (the viscosity changed); the next solve rebuilds it.
void mg_invalidate(MgHierarchy *h);
// Free every buffer of the hierarchy.  Accepts NULL.
void mg_destroy(MgHierarchy *h);

// Build (or rebuild, if stale or configured differently) the hierarchy for
// `params` (levels, coarsest, inner dtype).  Synchronises `s`.  Returns a
// stokes_status (STOKES_ERR_ARG if the coarsest level is too large for the
// dense solve, STOKES_ERR_DIVERGED if its matrix is not positive definite).
int mg_ensure(MgHierarchy **h, const MgOuter &o, const stokes_mg_params *params, cudaStream_t s);

// Number of levels of a built hierarchy, and level l of it.
int mg_levels(const MgHierarchy *h);
const MgLevel &mg_level(const MgHierarchy *h, int l);

// Enqueue one application of the preconditioner z = B r on `s`: r (outer
// precision `outer_dtype`, zero off the unknowns) is cast to the inner
// precision, one V-cycle runs from a zero initial guess, and its result is
// cast back into z.  Every buffer is (ny+1) x pitch of the finest level.
// rx = NULL: no input cast (the caller has written r, in the inner precision,
// to the finest level's right-hand side, mg_level(h, 0).bx / .by, beforehand);
// zx = NULL: no output cast (z stays in the inner precision, in the buffers
// mg_result reports after the enqueue).
int mg_enqueue_precond(MgHierarchy *h, int outer_dtype, const void *rx, const void *ry, void *zx, void *zy,
                       const stokes_mg_params *params, const RasRun &run, cudaStream_t s, LaunchHook &hook);
// The finest-level buffers that hold the V-cycle's result (inner precision)
// at the end of the last enqueued application.
void mg_result(const MgHierarchy *h, const void **zx, const void **zy);
// Inner precision of a built hierarchy (STOKES_F32 / STOKES_F64).
int mg_dtype(const MgHierarchy *h);

// ---- outer-solve vector kernels (krylov.cu) ---------------------------------
// Sums over the velocity unknowns, accumulated in FP64 in a fixed order; the
// two results land in out[0], out[1] (device).  `partials` holds
// krylov_partials() * 2 doubles.
struct KrylovView {
    int nx, ny, pitch;
    double *partials, *out;
};
int krylov_partials();
template <typename T> // (<a, b>, <a, c>); c may be NULL
cudaError_t kry_dot2(const KrylovView &k, const T *ax, const T *ay, const T *bx, const T *by, const T *cx,
                     const T *cy, cudaStream_t s);
template <typename T, typename Tz> // (<z, b>, 0) with z in its own precision
cudaError_t kry_dot_z(const KrylovView &k, const Tz *zx, const Tz *zy, const T *bx, const T *by, cudaStream_t s);
template <typename T, typename Tz> // p = (T) z + beta p (beta = 0: p = (T) z)
cudaError_t kry_direction_z(const KrylovView &k, double beta, const Tz *zx, const Tz *zy, T *px, T *py,
                            cudaStream_t s);
template <typename T, typename Ti> // kry_update, and bi = (Ti) r_new at the unknowns
cudaError_t kry_update_cast(const KrylovView &k, double a, const T *px, const T *py, const T *qx, const T *qy, T *vx,
                            T *vy, T *rx, T *ry, const T *ix, const T *iy, Ti *bix, Ti *biy, cudaStream_t s);
template <typename T> // q = M p (library eta_n: boundary nodes zero); out = (<p, q>, <p, r>);
                      // ax, ay: coefficients from kry_coef, or NULL to form them per flux
cudaError_t kry_apply_dot(const KrylovView &k, const GridDesc<T> &g, const T *ec, const T *en, const T *ax,
                          const T *ay, const T *px, const T *py, T *qx, T *qy, const T *rx, const T *ry,
                          cudaStream_t s);
template <typename T> // ax = 2 eta_c / hx^2, ay = 2 eta_c / hy^2 at every cell (coef_x / coef_y)
cudaError_t kry_coef(const KrylovView &k, const GridDesc<T> &g, const T *ec, T *ax, T *ay, cudaStream_t s);
template <typename T> // (sum r^2 w, sum f^2 w), w = -1/diag(M) from ix, iy
cudaError_t kry_energy(const KrylovView &k, const T *rx, const T *ry, const T *fx, const T *fy, const T *ix,
                       const T *iy, cudaStream_t s);
template <typename T> // v += a p, r -= a q; out[0] = sum r^2 w
cudaError_t kry_update(const KrylovView &k, double a, const T *px, const T *py, const T *qx, const T *qy, T *vx,
                       T *vy, T *rx, T *ry, const T *ix, const T *iy, cudaStream_t s);
template <typename T> // p = z + beta p
cudaError_t kry_direction(const KrylovView &k, double beta, const T *zx, const T *zy, T *px, T *py, cudaStream_t s);
template <typename T> // v += z
cudaError_t kry_add(const KrylovView &k, const T *zx, const T *zy, T *vx, T *vy, cudaStream_t s);
template <typename To, typename Ti> // v += (To) e at the unknowns
cudaError_t kry_add_cast(const KrylovView &k, const Ti *ex, const Ti *ey, To *vx, To *vy, cudaStream_t s);

// The smoother of level l (STOKES_MIXED: Jacobi on level 0, RAS below).
stokes_smooth_params level_smoother(const stokes_smooth_params &sm, int level);

// Sweeps of level l: ceil(nu0 growth^l), capped at nu_max when nu_max > 0.
int mg_sweeps(int nu0, double growth, int l, int nu_max);

// ---- kernels (mg_kernels.cu) ------------------------------------------------
template <typename T>
cudaError_t mg_coarsen_eta(const MgLevel &f, const MgLevel &c, cudaStream_t s);
template <typename Ts, typename Td>
cudaError_t mg_cast(size_t n, const void *src, void *dst, cudaStream_t s);
template <typename T>
cudaError_t mg_residual(const MgLevel &l, cudaStream_t s);
template <typename T>
cudaError_t mg_restrict(const MgLevel &f, const MgLevel &c, cudaStream_t s);
template <typename T>
cudaError_t mg_prolong_add(const MgLevel &f, const MgLevel &c, cudaStream_t s);
template <typename T>
cudaError_t mg_dense_setup(const MgLevel &l, int n, double *A, double *W, double *Ainv, int *status,
                           cudaStream_t s);
// One dense coarsest factorisation: the level's grid and viscosity (inner
// precision), its n unknowns, n x n FP64 work matrices A and W, the inverse
// Ainv and a status word (set to 1 if -M is not positive definite).
struct DenseJob {
    int nx, ny, pitch, n;
    double ihx, ihy;
    const void *ec, *en;
    double *A, *W, *Ainv;
    int *status;
};
// `count` factorisations at once (device table `jobs`, n <= nmax each).
template <typename T>
cudaError_t mg_dense_setup_many(const DenseJob *jobs, int count, int nmax, cudaStream_t s);
template <typename T>
cudaError_t mg_dense_solve(const MgLevel &l, int n, const double *Ainv, double *bvec, double *xvec, cudaStream_t s);

} // namespace stokes
