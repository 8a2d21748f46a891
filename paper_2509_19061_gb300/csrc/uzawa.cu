// uzawa.cu -- kernels of the inexact Uzawa iteration around the multigrid
// velocity solve (Sec. 3.1-3.2; solver configuration of Sec. 6.2): the
// lithostatic initial pressure, the pressure update with the viscosity as the
// approximate inverse Schur complement, the zero-mean shift, and the
// viscosity continuation.  Sums and the minimum are accumulated in FP64 in a
// fixed order.
#include <cfloat>

#include "../../include/stokes.h"
#include "internal.h"
#include "stencil.cuh"

namespace stokes {

namespace {

constexpr int UZ_THREADS = 256;
constexpr int UZ_BLOCKS = 152 * 4;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_min(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// block sum (or min) of v into partials[blockIdx.x]
template <bool MIN>
__device__ __forceinline__ void block_store(double v, double *partials)
{
    __shared__ double sh[UZ_THREADS / 32];
    v = MIN ? warp_min(v) : warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = sh[0];
        for (int q = 1; q < UZ_THREADS / 32; ++q) s = MIN ? fmin(s, sh[q]) : s + sh[q];
        partials[blockIdx.x] = s;
    }
}

// one warp: out[0] = sum (or min) of the partials, fixed order
template <bool MIN>
__global__ void k_final1(const double *__restrict__ partials, int n, double *__restrict__ out)
{
    double s = MIN ? DBL_MAX : 0.0;
    for (int b = threadIdx.x; b < n; b += 32) s = MIN ? fmin(s, partials[b]) : s + partials[b];
    s = MIN ? warp_min(s) : warp_sum(s);
    if (threadIdx.x == 0) out[0] = s;
}

// smallest viscosity over the cells and the interior nodes
template <typename T>
__global__ void __launch_bounds__(UZ_THREADS) k_eta_min(GridDesc<T> g, const T *__restrict__ ec,
                                                        const T *__restrict__ en, double *__restrict__ partials)
{
    double m = DBL_MAX;
    const long w = (long)g.nx + 1, total = w * (long)(g.ny + 1);
    for (long t = (long)blockIdx.x * UZ_THREADS + threadIdx.x; t < total; t += (long)gridDim.x * UZ_THREADS) {
        const int j = (int)(t / w), i = (int)(t - (long)j * w);
        const size_t q = (size_t)j * g.pitch + i;
        if (j < g.ny && i < g.nx) m = fmin(m, (double)ec[q]);
        if (j >= 1 && j <= g.ny - 1 && i >= 1 && i <= g.nx - 1) m = fmin(m, (double)en[q]);
    }
    block_store<true>(m, partials);
}

// eta = (1 - theta) eta_min + theta eta_base at the cells and interior nodes
// (boundary nodes stay zero: no shear stress there)
template <typename T>
__global__ void k_blend(GridDesc<T> g, T theta, const double *__restrict__ emin, const T *__restrict__ bc,
                        const T *__restrict__ bn, T *__restrict__ oc, T *__restrict__ on)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i > g.nx || j > g.ny) return;
    const size_t q = (size_t)j * g.pitch + i;
    const T base = r_mul(T(1) - theta, (T)emin[0]);
    if (j < g.ny && i < g.nx) oc[q] = r_add(base, r_mul(theta, bc[q]));
    const bool interior = j >= 1 && j <= g.ny - 1 && i >= 1 && i <= g.nx - 1;
    on[q] = interior ? r_add(base, r_mul(theta, bn[q])) : T(0);
}

// p <- p - omega_p eta_c D v at every cell; partial sums of the new p
template <typename T>
__global__ void __launch_bounds__(UZ_THREADS) k_p_update(GridDesc<T> g, T omega_p, const T *__restrict__ ec,
                                                         const T *__restrict__ vx, const T *__restrict__ vy,
                                                         T *__restrict__ p, double *__restrict__ partials)
{
    double s = 0.0;
    const long total = (long)g.nx * g.ny;
    for (long t = (long)blockIdx.x * UZ_THREADS + threadIdx.x; t < total; t += (long)gridDim.x * UZ_THREADS) {
        const int j = (int)(t / g.nx), i = (int)(t - (long)j * g.nx);
        const size_t q = (size_t)j * g.pitch + i;
        const T dv = r_fma(r_sub(vx[q + 1], vx[q]), g.ihx, r_mul(r_sub(vy[q + g.pitch], vy[q]), g.ihy));
        const T pn = r_sub(p[q], r_mul(r_mul(omega_p, ec[q]), dv));
        p[q] = pn;
        s += (double)pn;
    }
    block_store<false>(s, partials);
}

template <typename T>
__global__ void __launch_bounds__(UZ_THREADS) k_p_sum(GridDesc<T> g, const T *__restrict__ p,
                                                      double *__restrict__ partials)
{
    double s = 0.0;
    const long total = (long)g.nx * g.ny;
    for (long t = (long)blockIdx.x * UZ_THREADS + threadIdx.x; t < total; t += (long)gridDim.x * UZ_THREADS) {
        const int j = (int)(t / g.nx), i = (int)(t - (long)j * g.nx);
        s += (double)p[(size_t)j * g.pitch + i];
    }
    block_store<false>(s, partials);
}

// p <- p - sum / (nx ny)
template <typename T>
__global__ void k_p_shift(GridDesc<T> g, const double *__restrict__ sum, T *__restrict__ p)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const T mean = (T)(sum[0] / ((double)g.nx * (double)g.ny));
    const size_t q = (size_t)j * g.pitch + i;
    p[q] = r_sub(p[q], mean);
}

// lithostatic pressure: p[0][i] = 0, p[j][i] = p[j-1][i] - hy fy[j][i]
template <typename T>
__global__ void k_litho(GridDesc<T> g, T hy, const T *__restrict__ fy, T *__restrict__ p)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.nx) return;
    const size_t P = (size_t)g.pitch;
    T v = T(0);
    p[i] = v;
    for (int j = 1; j < g.ny; ++j) {
        v = r_sub(v, r_mul(hy, fy[(size_t)j * P + i]));
        p[(size_t)j * P + i] = v;
    }
}

// ---- Anderson acceleration (Algorithm 1) -----------------------------------
// r = F - x over whole arrays (walls and padding are zero in both)
template <typename T>
__global__ void k_diff(size_t n, const T *__restrict__ f, const T *__restrict__ x, T *__restrict__ r)
{
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        r[t] = r_sub(f[t], x[t]);
}

// <a, h_j> for j < hs.n, summed over the three fields; partials[blk * AA_MAX + j]
template <typename T>
__global__ void __launch_bounds__(UZ_THREADS) k_multidot(size_t n, AndersonSet<T> a, AndersonSet<T> hs,
                                                         double *__restrict__ partials)
{
    __shared__ double sh[UZ_THREADS / 32][AA_MAX];
    double s[AA_MAX];
#pragma unroll
    for (int j = 0; j < AA_MAX; ++j) s[j] = 0.0;
    for (size_t t = (size_t)blockIdx.x * UZ_THREADS + threadIdx.x; t < n; t += (size_t)gridDim.x * UZ_THREADS) {
        const double ax = (double)a.x[0][t], ay = (double)a.y[0][t], ap = (double)a.p[0][t];
#pragma unroll
        for (int j = 0; j < AA_MAX; ++j)
            if (j < hs.n) {
                s[j] = fma(ax, (double)hs.x[j][t], s[j]);
                s[j] = fma(ay, (double)hs.y[j][t], s[j]);
                s[j] = fma(ap, (double)hs.p[j][t], s[j]);
            }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < AA_MAX; ++j) {
        const double v = warp_sum(s[j]);
        if (lane == 0) sh[wid][j] = v;
    }
    __syncthreads();
    if (threadIdx.x < AA_MAX) {
        double v = 0.0;
        for (int q = 0; q < UZ_THREADS / 32; ++q) v += sh[q][threadIdx.x];
        partials[(size_t)blockIdx.x * AA_MAX + threadIdx.x] = v;
    }
}

// out[j] = sum over blocks of partials[b * AA_MAX + j], one warp per j
__global__ void k_final_multi(const double *__restrict__ partials, int nblocks, double *__restrict__ out)
{
    const int j = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double s = 0.0;
    for (int b = lane; b < nblocks; b += 32) s += partials[(size_t)b * AA_MAX + j];
    s = warp_sum(s);
    if (lane == 0) out[j] = s;
}

// x = sum_j alpha_j F_j, accumulated in the order j = 0, 1, ...
template <typename T>
__global__ void k_combine(size_t n, AndersonSet<T> F, AndersonAlpha al, T *__restrict__ x, T *__restrict__ y,
                          T *__restrict__ p)
{
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        T sx = r_mul((T)al.a[0], F.x[0][t]), sy = r_mul((T)al.a[0], F.y[0][t]), sp = r_mul((T)al.a[0], F.p[0][t]);
        for (int j = 1; j < F.n; ++j) {
            const T aj = (T)al.a[j];
            sx = r_add(sx, r_mul(aj, F.x[j][t]));
            sy = r_add(sy, r_mul(aj, F.y[j][t]));
            sp = r_add(sp, r_mul(aj, F.p[j][t]));
        }
        x[t] = sx;
        y[t] = sy;
        p[t] = sp;
    }
}

} // namespace

int uzawa_partials() { return UZ_BLOCKS; }

namespace {
inline dim3 grid2(int w, int h) { return dim3((unsigned)((w + 31) / 32), (unsigned)((h + 7) / 8)); }
} // namespace

template <typename T>
cudaError_t aa_diff(size_t n, const T *f, const T *x, T *r, cudaStream_t s)
{
    k_diff<T><<<UZ_BLOCKS, UZ_THREADS, 0, s>>>(n, f, x, r);
    return cudaGetLastError();
}

template <typename T>
cudaError_t aa_multidot(size_t n, const AndersonSet<T> &a, const AndersonSet<T> &hs, double *partials, double *out,
                        cudaStream_t s)
{
    k_multidot<T><<<UZ_BLOCKS, UZ_THREADS, 0, s>>>(n, a, hs, partials);
    k_final_multi<<<1, 32 * AA_MAX, 0, s>>>(partials, UZ_BLOCKS, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t aa_combine(size_t n, const AndersonSet<T> &F, const AndersonAlpha &al, T *x, T *y, T *p, cudaStream_t s)
{
    k_combine<T><<<UZ_BLOCKS, UZ_THREADS, 0, s>>>(n, F, al, x, y, p);
    return cudaGetLastError();
}

template <typename T>
cudaError_t uz_eta_min(const GridDesc<T> &g, const T *ec, const T *en, double *partials, double *out, cudaStream_t s)
{
    k_eta_min<T><<<UZ_BLOCKS, UZ_THREADS, 0, s>>>(g, ec, en, partials);
    k_final1<true><<<1, 32, 0, s>>>(partials, UZ_BLOCKS, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t uz_blend(const GridDesc<T> &g, double theta, const double *emin, const T *bc, const T *bn, T *oc, T *on,
                     cudaStream_t s)
{
    k_blend<T><<<grid2(g.nx + 1, g.ny + 1), dim3(32, 8), 0, s>>>(g, (T)theta, emin, bc, bn, oc, on);
    return cudaGetLastError();
}

template <typename T>
cudaError_t uz_pressure_update(const GridDesc<T> &g, double omega_p, const T *ec, const T *vx, const T *vy, T *p,
                               double *partials, double *sum, cudaStream_t s)
{
    k_p_update<T><<<UZ_BLOCKS, UZ_THREADS, 0, s>>>(g, (T)omega_p, ec, vx, vy, p, partials);
    k_final1<false><<<1, 32, 0, s>>>(partials, UZ_BLOCKS, sum);
    k_p_shift<T><<<grid2(g.nx, g.ny), dim3(32, 8), 0, s>>>(g, sum, p);
    return cudaGetLastError();
}

template <typename T>
cudaError_t uz_lithostatic(const GridDesc<T> &g, double hy, const T *fy, T *p, double *partials, double *sum,
                           cudaStream_t s)
{
    k_litho<T><<<(g.nx + 127) / 128, 128, 0, s>>>(g, (T)hy, fy, p);
    k_p_sum<T><<<UZ_BLOCKS, UZ_THREADS, 0, s>>>(g, p, partials);
    k_final1<false><<<1, 32, 0, s>>>(partials, UZ_BLOCKS, sum);
    k_p_shift<T><<<grid2(g.nx, g.ny), dim3(32, 8), 0, s>>>(g, sum, p);
    return cudaGetLastError();
}

#define INST(T)                                                                                                    \
    template cudaError_t aa_diff<T>(size_t, const T *, const T *, T *, cudaStream_t);                             \
    template cudaError_t aa_multidot<T>(size_t, const AndersonSet<T> &, const AndersonSet<T> &, double *,        \
                                        double *, cudaStream_t);                                                  \
    template cudaError_t aa_combine<T>(size_t, const AndersonSet<T> &, const AndersonAlpha &, T *, T *, T *,       \
                                       cudaStream_t);                                                              \
    template cudaError_t uz_eta_min<T>(const GridDesc<T> &, const T *, const T *, double *, double *,             \
                                       cudaStream_t);                                                              \
    template cudaError_t uz_blend<T>(const GridDesc<T> &, double, const double *, const T *, const T *, T *, T *,  \
                                     cudaStream_t);                                                                \
    template cudaError_t uz_pressure_update<T>(const GridDesc<T> &, double, const T *, const T *, const T *, T *,  \
                                               double *, double *, cudaStream_t);                                  \
    template cudaError_t uz_lithostatic<T>(const GridDesc<T> &, double, const T *, T *, double *, double *,        \
                                           cudaStream_t);
INST(float)
INST(double)
#undef INST

} // namespace stokes
