// krylov.cu -- vector kernels of the outer solve around the multigrid cycle:
// fused updates and inner products over the velocity unknowns (FP64
// accumulation, fixed reduction order) for flexible CG and defect correction.
#include "../../include/stokes.h"
#include "internal.h"
#include "mg.h"
#include "gstencil.cuh"
#include "stencil.cuh"

namespace stokes {

namespace {

constexpr int RD_THREADS = 256;
static_assert(AT_X * AT_Y == RD_THREADS, "one thread per tile cell");
constexpr int RD_BLOCKS = 152 * 4;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block-reduce two sums and write them to partials[2 * blockIdx.x + {0, 1}].
__device__ __forceinline__ void block_store2(double s0, double s1, double *partials)
{
    __shared__ double sh[2][RD_THREADS / 32];
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][wid] = s0;
        sh[1][wid] = s1;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double s = 0.0;
        for (int q = 0; q < RD_THREADS / 32; ++q) s += sh[threadIdx.x][q];
        partials[2 * blockIdx.x + threadIdx.x] = s;
    }
}

// Visit every cell once: f(q, vx is an unknown, vy is an unknown) with q the
// element offset; for_unknowns visits every velocity unknown once: f(q, component).
template <class F>
__device__ __forceinline__ void for_cells(int nx, int ny, int pitch, F &&f)
{
    // rows round-robin over the blocks, columns over the threads
    for (int j = blockIdx.x; j <= ny; j += gridDim.x)
        for (int i = threadIdx.x; i <= nx; i += RD_THREADS)
            f((size_t)j * pitch + i, j < ny && i >= 1 && i <= nx - 1, i < nx && j >= 1 && j <= ny - 1);
}

template <class F>
__device__ __forceinline__ void for_unknowns(int nx, int ny, int pitch, F &&f)
{
    for_cells(nx, ny, pitch, [&](size_t q, bool ux, bool uy) {
        if (ux) f(q, 0);
        if (uy) f(q, 1);
    });
}

// (<a, b>, <a, c>)
template <typename T>
__global__ void __launch_bounds__(RD_THREADS) k_dot2(int nx, int ny, int pitch, const T *__restrict__ ax,
                                                     const T *__restrict__ ay, const T *__restrict__ bx,
                                                     const T *__restrict__ by, const T *__restrict__ cx,
                                                     const T *__restrict__ cy, double *__restrict__ partials)
{
    double s0 = 0.0, s1 = 0.0;
    for_unknowns(nx, ny, pitch, [&](size_t q, int comp) {
        const double a = (double)(comp ? ay[q] : ax[q]);
        s0 = fma(a, (double)(comp ? by[q] : bx[q]), s0);
        if (cx) s1 = fma(a, (double)(comp ? cy[q] : cx[q]), s1);
    });
    block_store2(s0, s1, partials);
}

// (sum r^2 w, sum f^2 w) with w = -1/diag(M)
template <typename T>
__global__ void __launch_bounds__(RD_THREADS) k_energy_r(int nx, int ny, int pitch, const T *__restrict__ rx,
                                                         const T *__restrict__ ry, const T *__restrict__ fx,
                                                         const T *__restrict__ fy, const T *__restrict__ ix,
                                                         const T *__restrict__ iy, double *__restrict__ partials)
{
    double s0 = 0.0, s1 = 0.0;
    for_cells(nx, ny, pitch, [&](size_t q, bool ux, bool uy) {
        CellSq<T> c0(s0), c1(s1); // the cell's vx and vy terms
        if (ux) {
            const T wgt = -ix[q];
            c0.add(rx[q], wgt);
            c1.add(fx[q], wgt);
        }
        if (uy) {
            const T wgt = -iy[q];
            c0.add(ry[q], wgt);
            c1.add(fy[q], wgt);
        }
        c0.done();
        c1.done();
    });
    block_store2(s0, s1, partials);
}

// v += a p, r -= a q; returns (sum r_new^2 w, 0)
template <typename T>
__global__ void __launch_bounds__(RD_THREADS) k_cg_update(int nx, int ny, int pitch, double a, const T *__restrict__ px,
                                                          const T *__restrict__ py, const T *__restrict__ qx,
                                                          const T *__restrict__ qy, T *__restrict__ vx,
                                                          T *__restrict__ vy, T *__restrict__ rx, T *__restrict__ ry,
                                                          const T *__restrict__ ix, const T *__restrict__ iy,
                                                          double *__restrict__ partials)
{
    const T at = (T)a;
    double s0 = 0.0;
    for_unknowns(nx, ny, pitch, [&](size_t q, int comp) {
        T *v = comp ? vy : vx;
        T *r = comp ? ry : rx;
        v[q] = r_fma(at, (comp ? py : px)[q], v[q]);
        const T rn = r_fma(-at, (comp ? qy : qx)[q], r[q]);
        r[q] = rn;
        s0 = acc_sq(s0, rn, -(comp ? iy[q] : ix[q]));
    });
    block_store2(s0, 0.0, partials);
}

// <z, b> with z in its own precision (the V-cycle's result): (double) z is exact
template <typename T, typename Tz>
__global__ void __launch_bounds__(RD_THREADS) k_dot_z(int nx, int ny, int pitch, const Tz *__restrict__ zx,
                                                      const Tz *__restrict__ zy, const T *__restrict__ bx,
                                                      const T *__restrict__ by, double *__restrict__ partials)
{
    double s0 = 0.0;
    for_unknowns(nx, ny, pitch, [&](size_t q, int comp) {
        s0 = fma((double)(comp ? zy[q] : zx[q]), (double)(comp ? by[q] : bx[q]), s0);
    });
    block_store2(s0, 0.0, partials);
}

// p = (T) z + beta p at the unknowns, z in its own precision; FIRST: p = (T) z
template <typename T, typename Tz, bool FIRST>
__global__ void __launch_bounds__(RD_THREADS) k_direction_z(int nx, int ny, int pitch, double beta,
                                                            const Tz *__restrict__ zx, const Tz *__restrict__ zy,
                                                            T *__restrict__ px, T *__restrict__ py)
{
    const T bt = (T)beta;
    for_unknowns(nx, ny, pitch, [&](size_t q, int comp) {
        T *p = comp ? py : px;
        const T z = (T)(comp ? zy : zx)[q];
        p[q] = FIRST ? z : r_fma(bt, p[q], z);
    });
}

// v += a p, r -= a q, bi = (Ti) r; returns (sum r_new^2 w, 0)
template <typename T, typename Ti>
__global__ void __launch_bounds__(RD_THREADS) k_cg_update_cast(int nx, int ny, int pitch, double a,
                                                               const T *__restrict__ px, const T *__restrict__ py,
                                                               const T *__restrict__ qx, const T *__restrict__ qy,
                                                               T *__restrict__ vx, T *__restrict__ vy,
                                                               T *__restrict__ rx, T *__restrict__ ry,
                                                               const T *__restrict__ ix, const T *__restrict__ iy,
                                                               Ti *__restrict__ bix, Ti *__restrict__ biy,
                                                               double *__restrict__ partials)
{
    const T at = (T)a;
    double s0 = 0.0;
    for_unknowns(nx, ny, pitch, [&](size_t q, int comp) {
        T *v = comp ? vy : vx;
        T *r = comp ? ry : rx;
        v[q] = r_fma(at, (comp ? py : px)[q], v[q]);
        const T rn = r_fma(-at, (comp ? qy : qx)[q], r[q]);
        r[q] = rn;
        (comp ? biy : bix)[q] = (Ti)rn;
        s0 = acc_sq(s0, rn, -(comp ? iy[q] : ix[q]));
    });
    block_store2(s0, 0.0, partials);
}

// p = z + beta p at the unknowns
template <typename T>
__global__ void __launch_bounds__(RD_THREADS) k_cg_direction(int nx, int ny, int pitch, double beta,
                                                             const T *__restrict__ zx, const T *__restrict__ zy,
                                                             T *__restrict__ px, T *__restrict__ py)
{
    const T bt = (T)beta;
    for_unknowns(nx, ny, pitch, [&](size_t q, int comp) {
        T *p = comp ? py : px;
        p[q] = r_fma(bt, p[q], (comp ? zy : zx)[q]);
    });
}

// v += z at the unknowns
template <typename T>
__global__ void __launch_bounds__(RD_THREADS) k_add(int nx, int ny, int pitch, const T *__restrict__ zx,
                                                    const T *__restrict__ zy, T *__restrict__ vx, T *__restrict__ vy)
{
    for_unknowns(nx, ny, pitch, [&](size_t q, int comp) {
        T *v = comp ? vy : vx;
        v[q] = r_add(v[q], (comp ? zy : zx)[q]);
    });
}

// q = M p and (<p, q>, <p, r>) over the unknowns, tile by tile (see
// apply_dot_tile); each block walks the 32 x 8 cell tiles t = blockIdx.x,
// blockIdx.x + gridDim.x, ...
template <typename T>
__global__ void __launch_bounds__(RD_THREADS) k_apply_dot(GridDesc<T> g, const T *__restrict__ ec,
                                                          const T *__restrict__ en, const T *__restrict__ ax,
                                                          const T *__restrict__ ay, const T *__restrict__ px,
                                                          const T *__restrict__ py, T *__restrict__ qx,
                                                          T *__restrict__ qy, const T *__restrict__ rx,
                                                          const T *__restrict__ ry, double *__restrict__ partials)
{
    __shared__ ApplyTile<T> sm;
    const int ntx = (g.nx + 1 + AT_X - 1) / AT_X, nty = (g.ny + 1 + AT_Y - 1) / AT_Y;
    double s0 = 0.0, s1 = 0.0;
    for (int t = blockIdx.x; t < ntx * nty; t += gridDim.x)
        apply_dot_tile<T>(g, ec, en, ax, ay, px, py, qx, qy, rx, ry, (t % ntx) * AT_X, (t / ntx) * AT_Y, (int)threadIdx.x,
                          sm, s0, s1);
    block_store2(s0, s1, partials);
}

// the flux coefficients of every cell: ax = coef_x(eta_c), ay = coef_y(eta_c)
template <typename T>
__global__ void __launch_bounds__(RD_THREADS) k_coef(GridDesc<T> g, int nx, int ny, int pitch,
                                                     const T *__restrict__ ec, T *__restrict__ ax,
                                                     T *__restrict__ ay)
{
    for (int j = blockIdx.x; j < ny; j += gridDim.x)
        for (int i = threadIdx.x; i < nx; i += RD_THREADS) {
            const size_t q = (size_t)j * pitch + i;
            const T e = ec[q];
            ax[q] = coef_x(g, e);
            ay[q] = coef_y(g, e);
        }
}

// v += (To) e at the unknowns
template <typename To, typename Ti>
__global__ void __launch_bounds__(RD_THREADS) k_add_cast(int nx, int ny, int pitch, const Ti *__restrict__ ex,
                                                         const Ti *__restrict__ ey, To *__restrict__ vx,
                                                         To *__restrict__ vy)
{
    for_unknowns(nx, ny, pitch, [&](size_t q, int comp) {
        To *v = comp ? vy : vx;
        v[q] = r_add(v[q], (To)(comp ? ey : ex)[q]);
    });
}

__global__ void k_final2(const double *__restrict__ partials, int nblocks, double *__restrict__ out)
{
    const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double s = 0.0;
    for (int b = lane; b < nblocks; b += 32) s += partials[2 * b + c];
    s = warp_sum(s);
    if (lane == 0) out[c] = s;
}

} // namespace

int krylov_partials() { return RD_BLOCKS; }

template <typename T>
cudaError_t kry_dot2(const KrylovView &k, const T *ax, const T *ay, const T *bx, const T *by, const T *cx,
                     const T *cy, cudaStream_t s)
{
    k_dot2<T><<<RD_BLOCKS, RD_THREADS, 0, s>>>(k.nx, k.ny, k.pitch, ax, ay, bx, by, cx, cy, k.partials);
    k_final2<<<1, 64, 0, s>>>(k.partials, RD_BLOCKS, k.out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t kry_apply_dot(const KrylovView &k, const GridDesc<T> &g, const T *ec, const T *en, const T *ax,
                          const T *ay, const T *px, const T *py, T *qx, T *qy, const T *rx, const T *ry,
                          cudaStream_t s)
{
    k_apply_dot<T><<<RD_BLOCKS, RD_THREADS, 0, s>>>(g, ec, en, ax, ay, px, py, qx, qy, rx, ry, k.partials);
    k_final2<<<1, 64, 0, s>>>(k.partials, RD_BLOCKS, k.out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t kry_coef(const KrylovView &k, const GridDesc<T> &g, const T *ec, T *ax, T *ay, cudaStream_t s)
{
    k_coef<T><<<RD_BLOCKS, RD_THREADS, 0, s>>>(g, k.nx, k.ny, k.pitch, ec, ax, ay);
    return cudaGetLastError();
}

template <typename T>
cudaError_t kry_energy(const KrylovView &k, const T *rx, const T *ry, const T *fx, const T *fy, const T *ix,
                       const T *iy, cudaStream_t s)
{
    k_energy_r<T><<<RD_BLOCKS, RD_THREADS, 0, s>>>(k.nx, k.ny, k.pitch, rx, ry, fx, fy, ix, iy, k.partials);
    k_final2<<<1, 64, 0, s>>>(k.partials, RD_BLOCKS, k.out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t kry_update(const KrylovView &k, double a, const T *px, const T *py, const T *qx, const T *qy, T *vx,
                       T *vy, T *rx, T *ry, const T *ix, const T *iy, cudaStream_t s)
{
    k_cg_update<T><<<RD_BLOCKS, RD_THREADS, 0, s>>>(k.nx, k.ny, k.pitch, a, px, py, qx, qy, vx, vy, rx, ry, ix, iy,
                                                    k.partials);
    k_final2<<<1, 64, 0, s>>>(k.partials, RD_BLOCKS, k.out);
    return cudaGetLastError();
}

template <typename T, typename Tz>
cudaError_t kry_dot_z(const KrylovView &k, const Tz *zx, const Tz *zy, const T *bx, const T *by, cudaStream_t s)
{
    k_dot_z<T, Tz><<<RD_BLOCKS, RD_THREADS, 0, s>>>(k.nx, k.ny, k.pitch, zx, zy, bx, by, k.partials);
    k_final2<<<1, 64, 0, s>>>(k.partials, RD_BLOCKS, k.out);
    return cudaGetLastError();
}

template <typename T, typename Tz>
cudaError_t kry_direction_z(const KrylovView &k, double beta, const Tz *zx, const Tz *zy, T *px, T *py,
                            cudaStream_t s)
{
    if (beta == 0.0)
        k_direction_z<T, Tz, true><<<RD_BLOCKS, RD_THREADS, 0, s>>>(k.nx, k.ny, k.pitch, beta, zx, zy, px, py);
    else
        k_direction_z<T, Tz, false><<<RD_BLOCKS, RD_THREADS, 0, s>>>(k.nx, k.ny, k.pitch, beta, zx, zy, px, py);
    return cudaGetLastError();
}

template <typename T, typename Ti>
cudaError_t kry_update_cast(const KrylovView &k, double a, const T *px, const T *py, const T *qx, const T *qy, T *vx,
                            T *vy, T *rx, T *ry, const T *ix, const T *iy, Ti *bix, Ti *biy, cudaStream_t s)
{
    k_cg_update_cast<T, Ti><<<RD_BLOCKS, RD_THREADS, 0, s>>>(k.nx, k.ny, k.pitch, a, px, py, qx, qy, vx, vy, rx, ry,
                                                             ix, iy, bix, biy, k.partials);
    k_final2<<<1, 64, 0, s>>>(k.partials, RD_BLOCKS, k.out);
    return cudaGetLastError();
}

#define INST_Z(T, Tz)                                                                                              \
    template cudaError_t kry_dot_z<T, Tz>(const KrylovView &, const Tz *, const Tz *, const T *, const T *,       \
                                          cudaStream_t);                                                           \
    template cudaError_t kry_direction_z<T, Tz>(const KrylovView &, double, const Tz *, const Tz *, T *, T *,     \
                                                cudaStream_t);                                                     \
    template cudaError_t kry_update_cast<T, Tz>(const KrylovView &, double, const T *, const T *, const T *,       \
                                                const T *, T *, T *, T *, T *, const T *, const T *, Tz *, Tz *,  \
                                                cudaStream_t);
INST_Z(double, float)
INST_Z(double, double)
INST_Z(float, float)
INST_Z(float, double)
#undef INST_Z

template <typename T>
cudaError_t kry_direction(const KrylovView &k, double beta, const T *zx, const T *zy, T *px, T *py, cudaStream_t s)
{
    k_cg_direction<T><<<RD_BLOCKS, RD_THREADS, 0, s>>>(k.nx, k.ny, k.pitch, beta, zx, zy, px, py);
    return cudaGetLastError();
}

template <typename T>
cudaError_t kry_add(const KrylovView &k, const T *zx, const T *zy, T *vx, T *vy, cudaStream_t s)
{
    k_add<T><<<RD_BLOCKS, RD_THREADS, 0, s>>>(k.nx, k.ny, k.pitch, zx, zy, vx, vy);
    return cudaGetLastError();
}

template <typename To, typename Ti>
cudaError_t kry_add_cast(const KrylovView &k, const Ti *ex, const Ti *ey, To *vx, To *vy, cudaStream_t s)
{
    k_add_cast<To, Ti><<<RD_BLOCKS, RD_THREADS, 0, s>>>(k.nx, k.ny, k.pitch, ex, ey, vx, vy);
    return cudaGetLastError();
}
template cudaError_t kry_add_cast<double, float>(const KrylovView &, const float *, const float *, double *, double *,
                                                 cudaStream_t);
template cudaError_t kry_add_cast<double, double>(const KrylovView &, const double *, const double *, double *,
                                                  double *, cudaStream_t);
template cudaError_t kry_add_cast<float, float>(const KrylovView &, const float *, const float *, float *, float *,
                                                cudaStream_t);
template cudaError_t kry_add_cast<float, double>(const KrylovView &, const double *, const double *, float *,
                                                 float *, cudaStream_t);

#define INST(T)                                                                                                    \
    template cudaError_t kry_dot2<T>(const KrylovView &, const T *, const T *, const T *, const T *, const T *,    \
                                     const T *, cudaStream_t);                                                     \
    template cudaError_t kry_energy<T>(const KrylovView &, const T *, const T *, const T *, const T *, const T *,  \
                                       const T *, cudaStream_t);                                                   \
    template cudaError_t kry_update<T>(const KrylovView &, double, const T *, const T *, const T *, const T *,     \
                                       T *, T *, T *, T *, const T *, const T *, cudaStream_t);                    \
    template cudaError_t kry_direction<T>(const KrylovView &, double, const T *, const T *, T *, T *,             \
                                          cudaStream_t);                                                           \
    template cudaError_t kry_add<T>(const KrylovView &, const T *, const T *, T *, T *, cudaStream_t);          \
    template cudaError_t kry_apply_dot<T>(const KrylovView &, const GridDesc<T> &, const T *, const T *,        \
                                          const T *, const T *, const T *, const T *, T *, T *, const T *,      \
                                          const T *, cudaStream_t);                                             \
    template cudaError_t kry_coef<T>(const KrylovView &, const GridDesc<T> &, const T *, T *, T *, cudaStream_t);
INST(float)
INST(double)
#undef INST

} // namespace stokes
