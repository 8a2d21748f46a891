// gstencil.cuh -- the velocity operator evaluated at one point from global
// memory (used by the global-memory smoothers, the residual, the energy norm
// and the multigrid kernels).  Same arithmetic as stencil.cuh.
#pragma once
#include "internal.h"
#include "stencil.cuh"

namespace stokes {

// (M v)_x and diag(M)_x at vx unknown (j, i), 1 <= i <= nx-1, 0 <= j < ny.
// Rows outside the vx extent (j = -1, j = ny) enter only through a zero
// eta_n and are read as zero.
// MASK: eta_n is the caller's raw array, so boundary nodes are zeroed here
// (the library's own copy already holds zeros there).
template <typename T, bool MASK = false>
__device__ __forceinline__ void op_x(const GridDesc<T> &g, const T *__restrict__ eta_c, const T *__restrict__ eta_n,
                                     const T *__restrict__ vx, const T *__restrict__ vy, int j, int i, T &m, T &d,
                                     T &vc)
{
    const size_t P = (size_t)g.pitch;
    const size_t q = (size_t)j * P + (size_t)i;
    vc = vx[q];
    const T vE = vx[q + 1], vW = vx[q - 1];
    const T vN = j + 1 < g.ny ? vx[q + P] : T(0);
    const T vS = j > 0 ? vx[q - P] : T(0);
    const T ecC = eta_c[q], ecW = eta_c[q - 1];
    const T enN = (MASK && j + 1 == g.ny) ? T(0) : eta_n[q + P];
    const T enS = (MASK && j == 0) ? T(0) : eta_n[q];
    const T txx_c = flux_n(coef_x(g, ecC), vE, vc);
    const T txx_w = flux_n(coef_x(g, ecW), vc, vW);
    const T sx_n = r_mul(shear(g, enN, vN, vc, vy[q + P], vy[q + P - 1]), g.ihy);
    const T sx_c = r_mul(shear(g, enS, vc, vS, vy[q], vy[q - 1]), g.ihy);
    m = m_x(txx_c, txx_w, sx_n, sx_c);
    d = diag_x(g, ecC, ecW, enN, enS);
}

// (M v)_y and diag(M)_y at vy unknown (j, i), 1 <= j <= ny-1, 0 <= i < nx.
template <typename T, bool MASK = false>
__device__ __forceinline__ void op_y(const GridDesc<T> &g, const T *__restrict__ eta_c, const T *__restrict__ eta_n,
                                     const T *__restrict__ vx, const T *__restrict__ vy, int j, int i, T &m, T &d,
                                     T &vc)
{
    const size_t P = (size_t)g.pitch;
    const size_t q = (size_t)j * P + (size_t)i;
    vc = vy[q];
    const T vN = vy[q + P], vS = vy[q - P];
    const T vE = i + 1 < g.nx ? vy[q + 1] : T(0);
    const T vW = i > 0 ? vy[q - 1] : T(0);
    const T ecC = eta_c[q], ecS = eta_c[q - P];
    const T enE = (MASK && i + 1 == g.nx) ? T(0) : eta_n[q + 1];
    const T enW = (MASK && i == 0) ? T(0) : eta_n[q];
    const T tyy_c = flux_n(coef_y(g, ecC), vN, vc);
    const T tyy_s = flux_n(coef_y(g, ecS), vc, vS);
    const T sy_e = r_mul(shear(g, enE, vx[q + 1], vx[q + 1 - P], vE, vc), g.ihx);
    const T sy_c = r_mul(shear(g, enW, vx[q], vx[q - P], vc, vW), g.ihx);
    m = m_y(sy_e, sy_c, tyy_c, tyy_s);
    d = diag_y(g, ecC, ecS, enE, enW);
}

template <typename T>
__device__ __forceinline__ bool vx_unknown(const GridDesc<T> &g, int j, int i)
{
    return j < g.ny && i >= 1 && i <= g.nx - 1;
}
template <typename T>
__device__ __forceinline__ bool vy_unknown(const GridDesc<T> &g, int j, int i)
{
    return i < g.nx && j >= 1 && j <= g.ny - 1;
}
template <typename T>
__device__ __forceinline__ bool vx_wall(const GridDesc<T> &g, int j, int i)
{
    return j < g.ny && (i == 0 || i == g.nx);
}
template <typename T>
__device__ __forceinline__ bool vy_wall(const GridDesc<T> &g, int j, int i)
{
    return i < g.nx && (j == 0 || j == g.ny);
}

} // namespace stokes
