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
template <typename T, bool MASK = false, int SQM = 2>
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
    const T sx_n = shear_x<SQM>(g, enN, vN, vc, vy[q + P], vy[q + P - 1]);
    const T sx_c = shear_x<SQM>(g, enS, vc, vS, vy[q], vy[q - 1]);
    m = m_x(txx_c, txx_w, sx_n, sx_c);
    d = diag_x(g, ecC, ecW, enN, enS);
}

// (M v)_y and diag(M)_y at vy unknown (j, i), 1 <= j <= ny-1, 0 <= i < nx.
template <typename T, bool MASK = false, int SQM = 2>
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
    const T sy_e = shear_y<SQM>(g, enE, vx[q + 1], vx[q + 1 - P], vE, vc);
    const T sy_c = shear_y<SQM>(g, enW, vx[q], vx[q - P], vc, vW);
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

// ---- tiled operator apply with shared fluxes --------------------------------
// q = M p on the 32 x 8 cell tile at (i0, j0), plus (<p, q>, <p, r>) over its
// unknowns added to (s0, s1).  Every flux of the tile and a one-cell halo
// (sigma'xx / hx at cells, sigma'yy / hy at cells, the shear at nodes scaled
// by 1/hy and by 1/hx) is computed once into shared memory and M p assembled
// from them: about half the arithmetic of evaluating the stencil per unknown,
// which computes each flux twice.  ax, ay (nullable): the cell coefficients
// 2 eta_c / hx^2 and 2 eta_c / hy^2 precomputed by coef_x / coef_y, which
// saves their evaluation per flux.  The operands and helpers are those of
// op_x / op_y (library eta_n with zero boundary nodes; rows and columns
// outside a field read as zero), so q is the same bit for bit.  Called by all
// 256 threads of the block; tid is the caller's linear thread index (0 .. 255).
constexpr int AT_X = 32, AT_Y = 8;

template <typename T>
struct ApplyTile {
    T txx[AT_Y][AT_X + 1];     // cells (j0 + a, i0 - 1 + b)
    T tyy[AT_Y + 1][AT_X];     // cells (j0 - 1 + a, i0 + b)
    T sx[AT_Y + 1][AT_X + 1];  // nodes (j0 + a, i0 + b): shear / hy
    T sy[AT_Y + 1][AT_X + 1];  // the same nodes: shear / hx
};

// The fluxes of the tile at (i0, j0) and its one-cell halo from the velocity
// (px, py) into shared memory, ending with a barrier.
template <typename T>
__device__ __forceinline__ void flux_tile_stage(const GridDesc<T> &g, const T *__restrict__ ec,
                                                const T *__restrict__ en, const T *__restrict__ ax,
                                                const T *__restrict__ ay, const T *__restrict__ px,
                                                const T *__restrict__ py, int i0, int j0, int tid, ApplyTile<T> &sm)
{
    const size_t P = (size_t)g.pitch;
    const int nt = AT_X * AT_Y;
    for (int e = tid; e < AT_Y * (AT_X + 1); e += nt) {
        const int a = e / (AT_X + 1), b = e % (AT_X + 1);
        const int J = j0 + a, I = i0 - 1 + b;
        T v = T(0);
        if (J < g.ny && I >= 0 && I < g.nx) {
            const size_t q = (size_t)J * P + I;
            v = flux_n(ax ? ax[q] : coef_x(g, ec[q]), px[q + 1], px[q]);
        }
        sm.txx[a][b] = v;
    }
    for (int e = tid; e < (AT_Y + 1) * AT_X; e += nt) {
        const int a = e / AT_X, b = e % AT_X;
        const int J = j0 - 1 + a, I = i0 + b;
        T v = T(0);
        if (J >= 0 && J < g.ny && I < g.nx) {
            const size_t q = (size_t)J * P + I;
            v = flux_n(ay ? ay[q] : coef_y(g, ec[q]), py[q + P], py[q]);
        }
        sm.tyy[a][b] = v;
    }
    for (int e = tid; e < (AT_Y + 1) * (AT_X + 1); e += nt) {
        const int a = e / (AT_X + 1), b = e % (AT_X + 1);
        const int J = j0 + a, I = i0 + b;
        T sx = T(0), sy = T(0);
        if (J <= g.ny && I <= g.nx) {
            const size_t q = (size_t)J * P + I;
            const T vxa = J < g.ny ? px[q] : T(0), vxb = J > 0 ? px[q - P] : T(0);
            const T vyr = I < g.nx ? py[q] : T(0), vyl = I > 0 ? py[q - 1] : T(0);
            shear_xy(g, en[q], vxa, vxb, vyr, vyl, sx, sy);
        }
        sm.sx[a][b] = sx;
        sm.sy[a][b] = sy;
    }
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ void apply_dot_tile(const GridDesc<T> &g, const T *__restrict__ ec,
                                               const T *__restrict__ en, const T *__restrict__ ax,
                                               const T *__restrict__ ay, const T *__restrict__ px,
                                               const T *__restrict__ py, T *__restrict__ qx, T *__restrict__ qy,
                                               const T *__restrict__ rx, const T *__restrict__ ry, int i0, int j0,
                                               int tid, ApplyTile<T> &sm, double &s0, double &s1)
{
    const size_t P = (size_t)g.pitch;
    const int tx = tid % AT_X, ty = tid / AT_X;
    flux_tile_stage<T>(g, ec, en, ax, ay, px, py, i0, j0, tid, sm);
    const int j = j0 + ty, i = i0 + tx;
    if (j <= g.ny && i <= g.nx) {
        const size_t q = (size_t)j * P + i;
        if (j < g.ny) {
            T m = T(0);
            if (vx_unknown(g, j, i)) {
                m = m_x(sm.txx[ty][tx + 1], sm.txx[ty][tx], sm.sx[ty + 1][tx], sm.sx[ty][tx]);
                s0 = fma((double)px[q], (double)m, s0);
                s1 = fma((double)px[q], (double)rx[q], s1);
            }
            qx[q] = m;
        }
        if (i < g.nx) {
            T m = T(0);
            if (vy_unknown(g, j, i)) {
                m = m_y(sm.sy[ty][tx + 1], sm.sy[ty][tx], sm.tyy[ty + 1][tx], sm.tyy[ty][tx]);
                s0 = fma((double)py[q], (double)m, s0);
                s1 = fma((double)py[q], (double)ry[q], s1);
            }
            qy[q] = m;
        }
    }
    __syncthreads();
}

} // namespace stokes
