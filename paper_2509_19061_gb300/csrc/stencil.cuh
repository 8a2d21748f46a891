// stencil.cuh -- the velocity-operator stencil of arXiv 2509.19061 as pure
// arithmetic on already-loaded values, shared by the global-memory and the
// shared-memory kernels so that both round identically.
//
// Eq. (3): sigma'_xx = 2 eta_c dvx/dx and sigma'_yy = 2 eta_c dvy/dy at cell
// centres, sigma'_xy = eta_n (dvx/dy + dvy/dx) at nodes (eta_n = 0 on
// boundary nodes); Eq. (1)-(2): (M v)_x = d sigma'_xx/dx + d sigma'_xy/dy,
// (M v)_y = d sigma'_xy/dx + d sigma'_yy/dy.  d is diag(M), the coefficient of
// the centre value.
#pragma once
#include "internal.h"

namespace stokes {

// vx unknown at (j, i).  vC/vE/vW/vN/vS: vx at (j,i), (j,i+1), (j,i-1),
// (j+1,i), (j-1,i); yNE/yNW/ySE/ySW: vy at (j+1,i), (j+1,i-1), (j,i), (j,i-1);
// ecE/ecW: eta_c at (j,i), (j,i-1); enN/enS: eta_n at (j+1,i), (j,i).
template <typename T>
__device__ __forceinline__ void stencil_x(const GridDesc<T> &g, T vC, T vE, T vW, T vN, T vS, T yNE, T yNW, T ySE,
                                          T ySW, T ecE, T ecW, T enN, T enS, T &m, T &d)
{
    const T txxE = T(2) * ecE * (vE - vC) * g.ihx;
    const T txxW = T(2) * ecW * (vC - vW) * g.ihx;
    const T sN = enN * ((vN - vC) * g.ihy + (yNE - yNW) * g.ihx);
    const T sS = enS * ((vC - vS) * g.ihy + (ySE - ySW) * g.ihx);
    m = (txxE - txxW) * g.ihx + (sN - sS) * g.ihy;
    d = -T(2) * (ecE + ecW) * g.ihx2 - (enN + enS) * g.ihy2;
}

// vy unknown at (j, i).  vC/vN/vS/vE/vW: vy at (j,i), (j+1,i), (j-1,i),
// (j,i+1), (j,i-1); xNE/xSE/xNW/xSW: vx at (j,i+1), (j-1,i+1), (j,i), (j-1,i);
// ecN/ecS: eta_c at (j,i), (j-1,i); enE/enW: eta_n at (j,i+1), (j,i).
template <typename T>
__device__ __forceinline__ void stencil_y(const GridDesc<T> &g, T vC, T vN, T vS, T vE, T vW, T xNE, T xSE, T xNW,
                                          T xSW, T ecN, T ecS, T enE, T enW, T &m, T &d)
{
    const T tyyN = T(2) * ecN * (vN - vC) * g.ihy;
    const T tyyS = T(2) * ecS * (vC - vS) * g.ihy;
    const T sE = enE * ((xNE - xSE) * g.ihy + (vE - vC) * g.ihx);
    const T sW = enW * ((xNW - xSW) * g.ihy + (vC - vW) * g.ihx);
    m = (sE - sW) * g.ihx + (tyyN - tyyS) * g.ihy;
    d = -T(2) * (ecN + ecS) * g.ihy2 - (enE + enW) * g.ihx2;
}

// damped Jacobi update v + omega (b - M v) / diag(M)
template <typename T>
__device__ __forceinline__ T jacobi_update(T vc, T b, T m, T d, T omega)
{
    return vc + omega * (b - m) / d;
}

} // namespace stokes
