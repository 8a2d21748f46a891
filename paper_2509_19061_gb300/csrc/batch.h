// batch.h -- batched kernels over many independent instances (internal).
//
// An element-wise batched launch covers, for each participating instance, a
// rectangle of w x h points with 32 x 8 thread blocks; the blocks of all
// instances are numbered consecutively, and a segment map (one BSeg per
// instance, in block order) tells each block which instance it serves.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace stokes {

struct BSeg {
    int inst;        // instance index into the launch's tables
    int w, h;        // points covered
    int bxb;         // blocks per row: ceil(w / 32)
    int block_begin; // first block of this instance
};

// one instance at one multigrid level (inner precision T)
template <typename T>
struct BLevel {
    GridDesc<T> g;
    T *ec, *en, *ivx, *ivy, *bx, *by, *vx, *vy, *rx, *ry, *sx, *sy;
    // the next coarser level (restriction target, prolongation source)
    int cnx, cny, cp;
    T *cbx, *cby, *cvx, *cvy;
};

// coarsest dense solve of one instance
template <typename T>
struct BDense {
    int nx, ny, pitch, n;
    const double *Ainv;
    double *bvec, *xvec;
    const T *bx, *by;
    T *vx, *vy;
    int unk_begin; // first unknown of this instance in the concatenated numbering
};

// one instance's vectors of the outer solve (outer precision T)
template <typename T>
struct BOuter {
    GridDesc<T> g;
    const T *ec, *en, *ivx, *ivy, *fx, *fy, *bx, *by;
    const T *ax, *ay; // flux coefficients 2 eta_c / hx^2, 2 eta_c / hy^2
    T *vx, *vy, *rx, *ry, *zx, *zy, *px, *py, *qx, *qy;
};

// b = f - G p of one instance (p may be NULL)
template <typename T>
struct BRhs {
    GridDesc<T> g;
    const T *fx, *fy, *p;
    T *bx, *by;
};

constexpr int BATCH_BX = 32, BATCH_BY = 8;
// rows per thread of the tall element maps (blocks of 32 x BATCH_BY *
// BATCH_TALL cells): the setup-like copies take them, so that a block's
// segment lookup is shared by four times the cells and four rows' loads are
// in flight together
constexpr int BATCH_TALL = 4;

// The multigrid level kernels take `active` (device, one flag per instance,
// may be NULL): instances whose flag is 0 are skipped.

template <typename T> // over (nx+1) x (ny+1) per instance, a tall map
cudaError_t batch_rhs(const BRhs<T> *tab, const BSeg *map, int nseg, int nblocks, cudaStream_t s);

template <typename T>
cudaError_t batch_residual(const BLevel<T> *tab, const BSeg *map, int nseg, int nblocks, const int *active,
                           cudaStream_t s);
template <typename T>
cudaError_t batch_restrict(const BLevel<T> *tab, const BSeg *map, int nseg, int nblocks, const int *active,
                           cudaStream_t s);
template <typename T>
cudaError_t batch_prolong(const BLevel<T> *tab, const BSeg *map, int nseg, int nblocks, const int *active,
                          cudaStream_t s);
// zero v of every listed level (map over pitch x (ny+1))
template <typename T>
cudaError_t batch_zero_v(const BLevel<T> *tab, const BSeg *map, int nseg, int nblocks, const int *active,
                         cudaStream_t s);
// copy the in-extent entries of (vx, vy) into (sx, sy) when to_scratch, else
// the other way (a tall map)
template <typename T>
cudaError_t batch_copy(const BLevel<T> *tab, const BSeg *map, int nseg, int nblocks, bool to_scratch,
                       const int *active, cudaStream_t s);
// copy the wall entries of (vx, vy) into (sx, sy): one block per segment of
// the map (any block height)
template <typename T>
cudaError_t batch_copy_walls(const BLevel<T> *tab, const BSeg *map, int nseg, const int *active, cudaStream_t s);
// dense coarsest solves: `rows` unknowns in total over `count` instances
template <typename T>
cudaError_t batch_dense(const BDense<T> *tab, int count, int rows, const int *active, cudaStream_t s);
// level-0 inner b = (Ti) r and z = (To) level-0 inner v, over pitch x (ny+1)
template <typename To, typename Ti>
cudaError_t batch_cast_in(const BOuter<To> *out, const BLevel<Ti> *l0, const BSeg *map, int nseg, int nblocks,
                          const int *active, cudaStream_t s);
template <typename To, typename Ti>
cudaError_t batch_cast_out(const BOuter<To> *out, const BLevel<Ti> *l0, const BSeg *map, int nseg, int nblocks,
                           const int *active, cudaStream_t s);

// ---- outer solve (per-instance sums into out[2 * inst + {0, 1}]) -------------
// partials: 2 doubles per block of the launch
template <typename T> // r = b - M v; out = (sum r^2 w, sum f^2 w)
cudaError_t batch_residual_energy(const BOuter<T> *tab, const BSeg *map, int nseg, int nblocks, double *partials,
                                  double *out, cudaStream_t s);
template <typename T> // q = M p; out = (<p, q>, <p, r>)
cudaError_t batch_apply_dot(const BOuter<T> *tab, const BSeg *map, int nseg, int nblocks, double *partials,
                            double *out, cudaStream_t s);
template <typename T> // v += a p, r -= a q with a = alpha[inst]; out = (sum r^2 w, 0)
cudaError_t batch_update(const BOuter<T> *tab, const BSeg *map, int nseg, int nblocks, const double *alpha,
                         double *partials, double *out, cudaStream_t s);
template <typename T> // out = (<z, q>, 0)
cudaError_t batch_dot_zq(const BOuter<T> *tab, const BSeg *map, int nseg, int nblocks, double *partials,
                         double *out, cudaStream_t s);
template <typename T> // p = z + beta[inst] p  (beta NULL: p = z)
cudaError_t batch_direction(const BOuter<T> *tab, const BSeg *map, int nseg, int nblocks, const double *beta,
                            cudaStream_t s);
// Flexible CG with z and the V-cycle's right-hand side in the inner precision
// (no casts around the V-cycle): the update also writes (Ti) r_new into the
// finest level's b (table l0); <z, q> and p = z + beta p read z from the
// finest level's velocity buffers where the V-cycle leaves it (table fin).
template <typename To, typename Ti>
cudaError_t batch_update_cast(const BOuter<To> *tab, const BLevel<Ti> *l0, const BSeg *map, int nseg, int nblocks,
                              const double *alpha, double *partials, double *out, cudaStream_t s);
template <typename To, typename Ti>
cudaError_t batch_dot_zq_in(const BOuter<To> *tab, const BLevel<Ti> *fin, const BSeg *map, int nseg, int nblocks,
                            double *partials, double *out, cudaStream_t s);
template <typename To, typename Ti>
cudaError_t batch_direction_in(const BOuter<To> *tab, const BLevel<Ti> *fin, const BSeg *map, int nseg, int nblocks,
                               const double *beta, cudaStream_t s);
template <typename T> // v += z on instances whose active flag is set
cudaError_t batch_add(const BOuter<T> *tab, const BSeg *map, int nseg, int nblocks, const int *active, cudaStream_t s);
// alpha[i] = active[i] ? s[2i+1] / s[2i] : 0      (FCG step length)
// beta[i]  = active[i] ? -s2[2i] / s[2i] : 0      (FCG direction update)
cudaError_t batch_scalars(int count, const double *pq_pr, const double *zq, const int *active, double *alpha,
                          double *beta, cudaStream_t s);

} // namespace stokes
