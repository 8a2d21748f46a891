// stencil.cuh -- the velocity-operator stencil of arXiv 2509.19061 in flux
// form, as pure arithmetic shared by every kernel of the library.
//
// Eq. (3): sigma'_xx = 2 eta_c dvx/dx and sigma'_yy = 2 eta_c dvy/dy at cell
// centres, sigma'_xy = eta_n (dvx/dy + dvy/dx) at nodes (eta_n = 0 on
// boundary nodes); Eq. (1)-(2): (M v)_x = d sigma'_xx/dx + d sigma'_xy/dy and
// (M v)_y = d sigma'_xy/dx + d sigma'_yy/dy.  With the scaled fluxes
//   Txx(c) = sigma'_xx(c)/hx = ax(c) (vx(j,i+1) - vx(j,i)),  ax = 2 eta_c / hx^2
//   Tyy(c) = sigma'_yy(c)/hy = ay(c) (vy(j+1,i) - vy(j,i)),  ay = 2 eta_c / hy^2
//   Sx(n)  = sigma'_xy(n)/hy,  Sy(n) = sigma'_xy(n)/hx
// the operator is (M v)_x(j,i) = [Txx(j,i) - Txx(j,i-1)] + [Sx(j+1,i) - Sx(j,i)]
// and (M v)_y(j,i) = [Sy(j,i+1) - Sy(j,i)] + [Tyy(j,i) - Tyy(j-1,i)].
//
// Every operation below is an explicitly rounded intrinsic, so the compiler
// cannot contract or reorder it: a cell computed by the global-memory
// kernels and the same cell computed by the shared-memory tile kernel get
// identical bits.
#pragma once
#include "internal.h"

namespace stokes {

__device__ __forceinline__ float r_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double r_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float r_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double r_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float r_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double r_mul(double a, double b) { return __dmul_rn(a, b); }

// s + r^2 w, accumulated in FP64.  FP64 inputs: one FP64 fma.  FP32 inputs:
// the product in FP32 (its rounding, 2^-23 relative, is below that of the
// FP32 residual itself), then one FP64 add, a third of the FP64-pipe work
// (the FP64 pipe of this GPU runs at 1/64 of the FP32 rate).
__device__ __forceinline__ double acc_sq(double s, double r, double w) { return fma(r * r, w, s); }
__device__ __forceinline__ double acc_sq(double s, float r, float w) { return s + (double)r_mul(r_mul(r, r), w); }
__device__ __forceinline__ float r_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double r_fma(double a, double b, double c) { return __fma_rn(a, b, c); }
// The squared residual terms r^2 w of one cell (its vx and its vy unknown),
// added to an FP64 sum `s`.  FP64: each term with one FP64 fma, as acc_sq.
// FP32: the cell's two terms are added in FP32 (one more rounding, 2^-24
// relative, on a sum of two positive terms) and the cell enters the FP64 sum
// once, which halves the FP64-pipe operations of the energy reductions.
// Every energy kernel forms a cell's value this way, so the single-context
// and the batched reductions differ only in the order of their FP64 sums.
template <typename T>
struct CellSq;
template <>
struct CellSq<double> {
    double &s;
    __device__ __forceinline__ explicit CellSq(double &sum) : s(sum) {}
    __device__ __forceinline__ void add(double r, double w) { s = fma(r * r, w, s); }
    __device__ __forceinline__ void done() {}
};
template <>
struct CellSq<float> {
    double &s;
    float t = 0.f;
    bool any = false;
    __device__ __forceinline__ explicit CellSq(double &sum) : s(sum) {}
    __device__ __forceinline__ void add(float r, float w)
    {
        const float v = __fmul_rn(__fmul_rn(r, r), w);
        t = any ? __fadd_rn(t, v) : v;
        any = true;
    }
    __device__ __forceinline__ void done()
    {
        if (any) s += (double)t;
    }
};

// correctly rounded reciprocal (the same value as 1/x with IEEE division)
__device__ __forceinline__ float r_rcp(float a) { return __frcp_rn(a); }
__device__ __forceinline__ double r_rcp(double a) { return __drcp_rn(a); }

// ax = 2 eta_c / hx^2 and ay = 2 eta_c / hy^2
template <typename T>
__device__ __forceinline__ T coef_x(const GridDesc<T> &g, T ec)
{
    return r_mul(r_add(ec, ec), g.ihx2);
}
template <typename T>
__device__ __forceinline__ T coef_y(const GridDesc<T> &g, T ec)
{
    return r_mul(r_add(ec, ec), g.ihy2);
}

// Txx = ax (vx_E - vx_C), Tyy = ay (vy_N - vy_C)
template <typename T>
__device__ __forceinline__ T flux_n(T a, T v_next, T v_c)
{
    return r_mul(a, r_sub(v_next, v_c));
}

// sigma'_xy at node (i, j) from vx(j,i), vx(j-1,i), vy(j,i), vy(j,i-1)
template <typename T>
__device__ __forceinline__ T shear(const GridDesc<T> &g, T en, T vx_c, T vx_s, T vy_c, T vy_w)
{
    return r_mul(en, r_fma(r_sub(vx_c, vx_s), g.ihy, r_mul(r_sub(vy_c, vy_w), g.ihx)));
}

// Scaled shear fluxes Sx = sigma'_xy / hy and Sy = sigma'_xy / hx at node
// (i, j).  General cells: the shear above times 1/hy and 1/hx.  Square cells
// (g.square): Sx = Sy = (eta_n / h^2) ((vx_c - vx_s) + (vy_c - vy_w)), the
// same quantity in four operations instead of six.  Every kernel takes the
// form of its grid, so the schedules of one map still agree bit for bit.
template <typename T>
__device__ __forceinline__ T shear_sq(T en_h2, T vx_c, T vx_s, T vy_c, T vy_w)
{
    return r_mul(en_h2, r_add(r_sub(vx_c, vx_s), r_sub(vy_c, vy_w)));
}
// SQM: 0 the general form, 1 the square-cell form, 2 the form of the grid
// (g.square); kernels that know the form at launch take 0 or 1
template <int SQM = 2, typename T>
__device__ __forceinline__ bool square_form(const GridDesc<T> &g)
{
    return SQM == 2 ? g.square != 0 : SQM == 1;
}
template <int SQM = 2, typename T>
__device__ __forceinline__ T shear_x(const GridDesc<T> &g, T en, T vx_c, T vx_s, T vy_c, T vy_w)
{
    return square_form<SQM>(g) ? shear_sq(r_mul(en, g.ihx2), vx_c, vx_s, vy_c, vy_w)
                               : r_mul(shear(g, en, vx_c, vx_s, vy_c, vy_w), g.ihy);
}
template <int SQM = 2, typename T>
__device__ __forceinline__ T shear_y(const GridDesc<T> &g, T en, T vx_c, T vx_s, T vy_c, T vy_w)
{
    return square_form<SQM>(g) ? shear_sq(r_mul(en, g.ihx2), vx_c, vx_s, vy_c, vy_w)
                               : r_mul(shear(g, en, vx_c, vx_s, vy_c, vy_w), g.ihx);
}
// both at one node
template <int SQM = 2, typename T>
__device__ __forceinline__ void shear_xy(const GridDesc<T> &g, T en, T vx_c, T vx_s, T vy_c, T vy_w, T &sx, T &sy)
{
    if (square_form<SQM>(g)) {
        sx = sy = shear_sq(r_mul(en, g.ihx2), vx_c, vx_s, vy_c, vy_w);
    } else {
        const T sh = shear(g, en, vx_c, vx_s, vy_c, vy_w);
        sx = r_mul(sh, g.ihy);
        sy = r_mul(sh, g.ihx);
    }
}

// (M v)_x from Txx(j,i), Txx(j,i-1), Sx(j+1,i), Sx(j,i)
template <typename T>
__device__ __forceinline__ T m_x(T txx_c, T txx_w, T sx_n, T sx_c)
{
    return r_add(r_sub(txx_c, txx_w), r_sub(sx_n, sx_c));
}

// (M v)_y from Sy(j,i+1), Sy(j,i), Tyy(j,i), Tyy(j-1,i)
template <typename T>
__device__ __forceinline__ T m_y(T sy_e, T sy_c, T tyy_c, T tyy_s)
{
    return r_add(r_sub(sy_e, sy_c), r_sub(tyy_c, tyy_s));
}

// diag(M) at vx (j,i): -(2 (eta_c(j,i) + eta_c(j,i-1)) / hx^2 + (eta_n(j+1,i) + eta_n(j,i)) / hy^2)
template <typename T>
__device__ __forceinline__ T diag_x(const GridDesc<T> &g, T ec_c, T ec_w, T en_n, T en_s)
{
    return -r_fma(r_add(ec_c, ec_w), g.two_ihx2, r_mul(r_add(en_n, en_s), g.ihy2));
}

// diag(M) at vy (j,i): -(2 (eta_c(j,i) + eta_c(j-1,i)) / hy^2 + (eta_n(j,i+1) + eta_n(j,i)) / hx^2)
template <typename T>
__device__ __forceinline__ T diag_y(const GridDesc<T> &g, T ec_c, T ec_s, T en_e, T en_w)
{
    return -r_fma(r_add(ec_c, ec_s), g.two_ihy2, r_mul(r_add(en_e, en_w), g.ihx2));
}

// 1 / diag(M)
template <typename T>
__device__ __forceinline__ T inv_diag(T d)
{
    return r_rcp(d);
}

// damped-Jacobi weight omega / diag(M), from 1 / diag(M)
template <typename T>
__device__ __forceinline__ T jacobi_weight(T omega, T inv_d)
{
    return r_mul(omega, inv_d);
}

// v + (b - M v) omega / diag(M)
template <typename T>
__device__ __forceinline__ T jacobi_update(T v, T b, T m, T w)
{
    return r_fma(r_sub(b, m), w, v);
}

} // namespace stokes
