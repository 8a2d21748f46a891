// stokes3d.cu -- the 3D staggered-grid Stokes velocity operator and its
// smoothers: the 3D extension of the method that arXiv 2509.19061 names as
// future work (Sec. 9), with the flux form, readings and schedules of the 2D
// library carried over.
//
// Grid: nx x ny x nz cells; vx on x faces, vy on y faces, vz on z faces, p and
// eta_c at cell centres, the shear viscosities on the three edge sets
// (eta_xy for sigma'_xy, eta_xz for sigma'_xz, eta_yz for sigma'_yz).  Every
// field is one array of (nz+1) planes x (ny+1) rows x pitch elements; entry
// (k, j, i) is at (k (ny+1) + j) pitch + i.  The library's copies of the edge
// viscosities hold zero on the edges that lie in a wall they are tangential
// to (free slip), so the stencil needs no branch there.
//
// Kernels (every update goes through the per-point arithmetic of op3_*, so
// schedules of the same map agree bit for bit):
//   k3_jacobi  fused damped Jacobi, one thread per cell (its vx, vy and vz
//              faces), neighbours through L1/L2;
//   k3_ras     RAS-Jacobi on 3D tiles (Algorithm 2 in 3D): one CTA per tile,
//              the window (tile grown by overlap + 1) of the velocity (twice,
//              for the ping-pong of the local sweeps) and the viscosities
//              staged in shared memory, the k local sweeps on chip (each sweep
//              updates only the cells within min(overlap, k - s) of the tile),
//              the tile's own unknowns written back.  Space and time are
//              blocked together: the "4D blocking" of Sec. 9;
//   k3_ras_col the same map for windows 16 to 32 cells wide: a warp per
//              window row, each thread's z column in registers, each flux
//              formed once, y neighbours through shared memory.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "../../include/stokes.h"
#include "internal.h"
#include "stencil.cuh"

using namespace stokes;

namespace {

#define CK(call)                                                                                                   \
    do {                                                                                                           \
        cudaError_t e_ = (call);                                                                                   \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);                                                        \
    } while (0)

template <typename T>
struct G3 {
    int nx, ny, nz, pitch;
    size_t plane; // (ny + 1) * pitch
    T ihx, ihy, ihz, ihx2, ihy2, ihz2, two_ihx2, two_ihy2, two_ihz2;
    double lap; // 2/hx^2 + 2/hy^2 + 2/hz^2 (pressure weight of the energy norm)
    __host__ __device__ size_t at(int k, int j, int i) const { return (size_t)k * plane + (size_t)j * pitch + i; }
};

template <typename T>
G3<T> make_g3(int nx, int ny, int nz, int pitch, double hx, double hy, double hz)
{
    G3<T> g;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.pitch = pitch;
    g.plane = (size_t)(ny + 1) * pitch;
    g.ihx = (T)(1.0 / hx);
    g.ihy = (T)(1.0 / hy);
    g.ihz = (T)(1.0 / hz);
    g.ihx2 = (T)(1.0 / (hx * hx));
    g.ihy2 = (T)(1.0 / (hy * hy));
    g.ihz2 = (T)(1.0 / (hz * hz));
    g.two_ihx2 = g.ihx2 + g.ihx2;
    g.two_ihy2 = g.ihy2 + g.ihy2;
    g.two_ihz2 = g.ihz2 + g.ihz2;
    g.lap = 2.0 / (hx * hx) + 2.0 / (hy * hy) + 2.0 / (hz * hz);
    return g;
}

template <typename T>
struct C3 {
    const T *ec, *exy, *exz, *eyz; // library copies (wall edges zero)
    const T *bx, *by, *bz;
    const T *ix, *iy, *iz; // 1 / diag(M) at the unknowns (zero elsewhere)
};

// field extents: x-like rows < ny, cols <= nx, planes < nz; and so on
template <typename T>
__device__ __forceinline__ bool in_vx(const G3<T> &g, int k, int j, int i)
{
    return k >= 0 && k < g.nz && j >= 0 && j < g.ny && i >= 0 && i <= g.nx;
}
template <typename T>
__device__ __forceinline__ bool in_vy(const G3<T> &g, int k, int j, int i)
{
    return k >= 0 && k < g.nz && j >= 0 && j <= g.ny && i >= 0 && i < g.nx;
}
template <typename T>
__device__ __forceinline__ bool in_vz(const G3<T> &g, int k, int j, int i)
{
    return k >= 0 && k <= g.nz && j >= 0 && j < g.ny && i >= 0 && i < g.nx;
}
template <typename T>
__device__ __forceinline__ bool in_c(const G3<T> &g, int k, int j, int i)
{
    return k >= 0 && k < g.nz && j >= 0 && j < g.ny && i >= 0 && i < g.nx;
}
template <typename T>
__device__ __forceinline__ bool in_xy(const G3<T> &g, int k, int j, int i)
{
    return k >= 0 && k < g.nz && j >= 0 && j <= g.ny && i >= 0 && i <= g.nx;
}
template <typename T>
__device__ __forceinline__ bool in_xz(const G3<T> &g, int k, int j, int i)
{
    return k >= 0 && k <= g.nz && j >= 0 && j < g.ny && i >= 0 && i <= g.nx;
}
template <typename T>
__device__ __forceinline__ bool in_yz(const G3<T> &g, int k, int j, int i)
{
    return k >= 0 && k <= g.nz && j >= 0 && j <= g.ny && i >= 0 && i < g.nx;
}
template <typename T>
__device__ __forceinline__ bool unk_x(const G3<T> &g, int k, int j, int i)
{
    return k >= 0 && k < g.nz && j >= 0 && j < g.ny && i >= 1 && i <= g.nx - 1;
}
template <typename T>
__device__ __forceinline__ bool unk_y(const G3<T> &g, int k, int j, int i)
{
    return k >= 0 && k < g.nz && i >= 0 && i < g.nx && j >= 1 && j <= g.ny - 1;
}
template <typename T>
__device__ __forceinline__ bool unk_z(const G3<T> &g, int k, int j, int i)
{
    return j >= 0 && j < g.ny && i >= 0 && i < g.nx && k >= 1 && k <= g.nz - 1;
}

// ---- per-point arithmetic --------------------------------------------------
// A is an accessor: vx(k, j, i), vy, vz, ec, exy, exz, eyz return the value of
// that field, zero outside its extent.  Scaled fluxes:
//   Txx = 2 eta_c (vx(i+1) - vx(i)) / hx^2 (and Tyy, Tzz),
//   sigma'_xy = eta_xy ((vx(j) - vx(j-1)) / hy + (vy(i) - vy(i-1)) / hx), then / hy
//   for the x row and / hx for the y row; sigma'_xz, sigma'_yz likewise.
template <typename T, class A>
__device__ __forceinline__ T sig_xy(const G3<T> &g, const A &a, int k, int j, int i)
{
    return r_mul(a.exy(k, j, i),
                 r_fma(r_sub(a.vx(k, j, i), a.vx(k, j - 1, i)), g.ihy, r_mul(r_sub(a.vy(k, j, i), a.vy(k, j, i - 1)), g.ihx)));
}
template <typename T, class A>
__device__ __forceinline__ T sig_xz(const G3<T> &g, const A &a, int k, int j, int i)
{
    return r_mul(a.exz(k, j, i),
                 r_fma(r_sub(a.vx(k, j, i), a.vx(k - 1, j, i)), g.ihz, r_mul(r_sub(a.vz(k, j, i), a.vz(k, j, i - 1)), g.ihx)));
}
template <typename T, class A>
__device__ __forceinline__ T sig_yz(const G3<T> &g, const A &a, int k, int j, int i)
{
    return r_mul(a.eyz(k, j, i),
                 r_fma(r_sub(a.vy(k, j, i), a.vy(k - 1, j, i)), g.ihz, r_mul(r_sub(a.vz(k, j, i), a.vz(k, j - 1, i)), g.ihy)));
}

// diag(M) at vx, vy, vz (k, j, i): the viscosities only
template <typename T, class A>
__device__ __forceinline__ T diag3_x(const G3<T> &g, const A &a, int k, int j, int i)
{
    return -r_fma(r_add(a.ec(k, j, i), a.ec(k, j, i - 1)), g.two_ihx2,
                  r_fma(r_add(a.exy(k, j + 1, i), a.exy(k, j, i)), g.ihy2,
                        r_mul(r_add(a.exz(k + 1, j, i), a.exz(k, j, i)), g.ihz2)));
}
template <typename T, class A>
__device__ __forceinline__ T diag3_y(const G3<T> &g, const A &a, int k, int j, int i)
{
    return -r_fma(r_add(a.ec(k, j, i), a.ec(k, j - 1, i)), g.two_ihy2,
                  r_fma(r_add(a.exy(k, j, i + 1), a.exy(k, j, i)), g.ihx2,
                        r_mul(r_add(a.eyz(k + 1, j, i), a.eyz(k, j, i)), g.ihz2)));
}
template <typename T, class A>
__device__ __forceinline__ T diag3_z(const G3<T> &g, const A &a, int k, int j, int i)
{
    return -r_fma(r_add(a.ec(k, j, i), a.ec(k - 1, j, i)), g.two_ihz2,
                  r_fma(r_add(a.exz(k, j, i + 1), a.exz(k, j, i)), g.ihx2,
                        r_mul(r_add(a.eyz(k, j + 1, i), a.eyz(k, j, i)), g.ihy2)));
}

// (M v)_x at vx (k, j, i)
template <typename T, class A>
__device__ __forceinline__ T op3_x(const G3<T> &g, const A &a, int k, int j, int i)
{
    const T ecC = a.ec(k, j, i), ecW = a.ec(k, j, i - 1);
    const T vc = a.vx(k, j, i);
    const T txx_c = r_mul(r_mul(r_add(ecC, ecC), g.ihx2), r_sub(a.vx(k, j, i + 1), vc));
    const T txx_w = r_mul(r_mul(r_add(ecW, ecW), g.ihx2), r_sub(vc, a.vx(k, j, i - 1)));
    const T sn = r_mul(sig_xy(g, a, k, j + 1, i), g.ihy), ss = r_mul(sig_xy(g, a, k, j, i), g.ihy);
    const T su = r_mul(sig_xz(g, a, k + 1, j, i), g.ihz), sd = r_mul(sig_xz(g, a, k, j, i), g.ihz);
    return r_add(r_add(r_sub(txx_c, txx_w), r_sub(sn, ss)), r_sub(su, sd));
}
// (M v)_y at vy (k, j, i)
template <typename T, class A>
__device__ __forceinline__ T op3_y(const G3<T> &g, const A &a, int k, int j, int i)
{
    const T ecC = a.ec(k, j, i), ecS = a.ec(k, j - 1, i);
    const T vc = a.vy(k, j, i);
    const T tyy_c = r_mul(r_mul(r_add(ecC, ecC), g.ihy2), r_sub(a.vy(k, j + 1, i), vc));
    const T tyy_s = r_mul(r_mul(r_add(ecS, ecS), g.ihy2), r_sub(vc, a.vy(k, j - 1, i)));
    const T se = r_mul(sig_xy(g, a, k, j, i + 1), g.ihx), sw = r_mul(sig_xy(g, a, k, j, i), g.ihx);
    const T su = r_mul(sig_yz(g, a, k + 1, j, i), g.ihz), sd = r_mul(sig_yz(g, a, k, j, i), g.ihz);
    return r_add(r_add(r_sub(se, sw), r_sub(tyy_c, tyy_s)), r_sub(su, sd));
}
// (M v)_z at vz (k, j, i)
template <typename T, class A>
__device__ __forceinline__ T op3_z(const G3<T> &g, const A &a, int k, int j, int i)
{
    const T ecC = a.ec(k, j, i), ecD = a.ec(k - 1, j, i);
    const T vc = a.vz(k, j, i);
    const T tzz_c = r_mul(r_mul(r_add(ecC, ecC), g.ihz2), r_sub(a.vz(k + 1, j, i), vc));
    const T tzz_d = r_mul(r_mul(r_add(ecD, ecD), g.ihz2), r_sub(vc, a.vz(k - 1, j, i)));
    const T se = r_mul(sig_xz(g, a, k, j, i + 1), g.ihx), sw = r_mul(sig_xz(g, a, k, j, i), g.ihx);
    const T sn = r_mul(sig_yz(g, a, k, j + 1, i), g.ihy), ss = r_mul(sig_yz(g, a, k, j, i), g.ihy);
    return r_add(r_add(r_sub(se, sw), r_sub(sn, ss)), r_sub(tzz_c, tzz_d));
}

// accessor of the pitched global arrays (zero outside a field's extent)
template <typename T>
struct GAcc {
    G3<T> g;
    const T *__restrict__ x, *__restrict__ y, *__restrict__ z;
    const T *__restrict__ c, *__restrict__ xy, *__restrict__ xz, *__restrict__ yz;
    __device__ T vx(int k, int j, int i) const { return in_vx(g, k, j, i) ? x[g.at(k, j, i)] : T(0); }
    __device__ T vy(int k, int j, int i) const { return in_vy(g, k, j, i) ? y[g.at(k, j, i)] : T(0); }
    __device__ T vz(int k, int j, int i) const { return in_vz(g, k, j, i) ? z[g.at(k, j, i)] : T(0); }
    __device__ T ec(int k, int j, int i) const { return in_c(g, k, j, i) ? c[g.at(k, j, i)] : T(0); }
    __device__ T exy(int k, int j, int i) const { return in_xy(g, k, j, i) ? xy[g.at(k, j, i)] : T(0); }
    __device__ T exz(int k, int j, int i) const { return in_xz(g, k, j, i) ? xz[g.at(k, j, i)] : T(0); }
    __device__ T eyz(int k, int j, int i) const { return in_yz(g, k, j, i) ? yz[g.at(k, j, i)] : T(0); }
};

constexpr int B3X = 32, B3Y = 4, B3Z = 2;

inline dim3 grid3(int w, int h, int d)
{
    return dim3((unsigned)((w + B3X - 1) / B3X), (unsigned)((h + B3Y - 1) / B3Y), (unsigned)((d + B3Z - 1) / B3Z));
}

// ---- coefficient preparation, right-hand side, operator ----------------------
template <typename T>
__global__ void k3_coeffs(G3<T> g, const T *__restrict__ ec_in, const T *__restrict__ xy_in, const T *__restrict__ xz_in,
                          const T *__restrict__ yz_in, T *__restrict__ ec, T *__restrict__ xy, T *__restrict__ xz,
                          T *__restrict__ yz)
{
    const int i = blockIdx.x * B3X + threadIdx.x, j = blockIdx.y * B3Y + threadIdx.y, k = blockIdx.z * B3Z + threadIdx.z;
    if (i > g.nx || j > g.ny || k > g.nz) return;
    const size_t q = g.at(k, j, i);
    if (in_c(g, k, j, i)) ec[q] = ec_in[q];
    const bool ix = i >= 1 && i <= g.nx - 1, jy = j >= 1 && j <= g.ny - 1, kz = k >= 1 && k <= g.nz - 1;
    if (in_xy(g, k, j, i)) xy[q] = (ix && jy) ? xy_in[q] : T(0);
    if (in_xz(g, k, j, i)) xz[q] = (ix && kz) ? xz_in[q] : T(0);
    if (in_yz(g, k, j, i)) yz[q] = (jy && kz) ? yz_in[q] : T(0);
}

template <typename T>
GAcc<T> gacc(const G3<T> &g, const T *vx, const T *vy, const T *vz, const T *ec, const T *xy, const T *xz, const T *yz)
{
    GAcc<T> a;
    a.g = g;
    a.x = vx;
    a.y = vy;
    a.z = vz;
    a.c = ec;
    a.xy = xy;
    a.xz = xz;
    a.yz = yz;
    return a;
}

// 1 / diag(M) at the unknowns, zero elsewhere
template <typename T>
__global__ void k3_inv_diag(G3<T> g, GAcc<T> a, T *__restrict__ ix, T *__restrict__ iy, T *__restrict__ iz)
{
    const int i = blockIdx.x * B3X + threadIdx.x, j = blockIdx.y * B3Y + threadIdx.y, k = blockIdx.z * B3Z + threadIdx.z;
    if (i > g.nx || j > g.ny || k > g.nz) return;
    const size_t q = g.at(k, j, i);
    if (in_vx(g, k, j, i)) ix[q] = unk_x(g, k, j, i) ? inv_diag(diag3_x(g, a, k, j, i)) : T(0);
    if (in_vy(g, k, j, i)) iy[q] = unk_y(g, k, j, i) ? inv_diag(diag3_y(g, a, k, j, i)) : T(0);
    if (in_vz(g, k, j, i)) iz[q] = unk_z(g, k, j, i) ? inv_diag(diag3_z(g, a, k, j, i)) : T(0);
}

// b = f - G p with (G p) = -grad p at the unknowns (p may be NULL), zero elsewhere in the extents
template <typename T>
__global__ void k3_rhs(G3<T> g, const T *__restrict__ fx, const T *__restrict__ fy, const T *__restrict__ fz,
                       const T *__restrict__ p, T *__restrict__ bx, T *__restrict__ by, T *__restrict__ bz)
{
    const int i = blockIdx.x * B3X + threadIdx.x, j = blockIdx.y * B3Y + threadIdx.y, k = blockIdx.z * B3Z + threadIdx.z;
    if (i > g.nx || j > g.ny || k > g.nz) return;
    const size_t q = g.at(k, j, i);
    if (in_vx(g, k, j, i))
        bx[q] = unk_x(g, k, j, i) ? (p ? r_fma(r_sub(p[q], p[q - 1]), g.ihx, fx[q]) : fx[q]) : T(0);
    if (in_vy(g, k, j, i))
        by[q] = unk_y(g, k, j, i) ? (p ? r_fma(r_sub(p[q], p[q - g.pitch]), g.ihy, fy[q]) : fy[q]) : T(0);
    if (in_vz(g, k, j, i))
        bz[q] = unk_z(g, k, j, i) ? (p ? r_fma(r_sub(p[q], p[q - g.plane]), g.ihz, fz[q]) : fz[q]) : T(0);
}

// out = M v + G p at the unknowns, zero elsewhere in the extents
template <typename T>
__global__ void k3_apply(G3<T> g, GAcc<T> a, const T *__restrict__ p, T *__restrict__ ox, T *__restrict__ oy,
                         T *__restrict__ oz)
{
    const int i = blockIdx.x * B3X + threadIdx.x, j = blockIdx.y * B3Y + threadIdx.y, k = blockIdx.z * B3Z + threadIdx.z;
    if (i > g.nx || j > g.ny || k > g.nz) return;
    const size_t q = g.at(k, j, i);
    if (in_vx(g, k, j, i))
        ox[q] = unk_x(g, k, j, i) ? r_sub(op3_x(g, a, k, j, i), p ? r_mul(r_sub(p[q], p[q - 1]), g.ihx) : T(0)) : T(0);
    if (in_vy(g, k, j, i))
        oy[q] = unk_y(g, k, j, i) ? r_sub(op3_y(g, a, k, j, i), p ? r_mul(r_sub(p[q], p[q - g.pitch]), g.ihy) : T(0))
                                  : T(0);
    if (in_vz(g, k, j, i))
        oz[q] = unk_z(g, k, j, i) ? r_sub(op3_z(g, a, k, j, i), p ? r_mul(r_sub(p[q], p[q - g.plane]), g.ihz) : T(0))
                                  : T(0);
}

// accessor without extent tests, for points whose neighbours all lie inside
// every field's extent (the same values as GAcc there)
template <typename T>
struct UAcc {
    G3<T> g;
    const T *__restrict__ x, *__restrict__ y, *__restrict__ z;
    const T *__restrict__ c, *__restrict__ xy, *__restrict__ xz, *__restrict__ yz;
    __device__ __forceinline__ T vx(int k, int j, int i) const { return x[g.at(k, j, i)]; }
    __device__ __forceinline__ T vy(int k, int j, int i) const { return y[g.at(k, j, i)]; }
    __device__ __forceinline__ T vz(int k, int j, int i) const { return z[g.at(k, j, i)]; }
    __device__ __forceinline__ T ec(int k, int j, int i) const { return c[g.at(k, j, i)]; }
    __device__ __forceinline__ T exy(int k, int j, int i) const { return xy[g.at(k, j, i)]; }
    __device__ __forceinline__ T exz(int k, int j, int i) const { return xz[g.at(k, j, i)]; }
    __device__ __forceinline__ T eyz(int k, int j, int i) const { return yz[g.at(k, j, i)]; }
};

// ---- fused damped Jacobi -------------------------------------------------------
// Every unknown from the old (vx, vy, vz); walls copied, padding untouched.
// A point in the cells 1 .. n - 2 of every axis has three unknowns, and it
// and its neighbours (one cell each way) lie inside every extent: it takes
// the same arithmetic without extent or unknown tests.  FP32 decides per
// point (only warps at the domain's faces take both paths); FP64, bound by
// its FP64 pipe, per block (measured: 4.8 against 3.9 Gcell-updates/s per
// point at 192^3).  FP32 runs five blocks per SM (48 registers, no spills).
template <typename T>
__global__ void __launch_bounds__(B3X * B3Y * B3Z, sizeof(T) == 4 ? 5 : 4) k3_jacobi(G3<T> g, GAcc<T> a, C3<T> c, T omega, T *__restrict__ ox, T *__restrict__ oy,
                          T *__restrict__ oz)
{
    const int i0 = blockIdx.x * B3X, j0 = blockIdx.y * B3Y, k0 = blockIdx.z * B3Z;
    const int i = i0 + threadIdx.x, j = j0 + threadIdx.y, k = k0 + threadIdx.z;
    const bool fast = sizeof(T) == 4
                          ? (i >= 1 && i <= g.nx - 2 && j >= 1 && j <= g.ny - 2 && k >= 1 && k <= g.nz - 2)
                          : (i0 >= 1 && i0 + B3X <= g.nx - 1 && j0 >= 1 && j0 + B3Y <= g.ny - 1 && k0 >= 1 &&
                             k0 + B3Z <= g.nz - 1);
    if (fast) {
        UAcc<T> u;
        u.g = g;
        u.x = a.x; u.y = a.y; u.z = a.z;
        u.c = a.c; u.xy = a.xy; u.xz = a.xz; u.yz = a.yz;
        const size_t q = g.at(k, j, i);
        ox[q] = jacobi_update(a.x[q], c.bx[q], op3_x(g, u, k, j, i), jacobi_weight(omega, c.ix[q]));
        oy[q] = jacobi_update(a.y[q], c.by[q], op3_y(g, u, k, j, i), jacobi_weight(omega, c.iy[q]));
        oz[q] = jacobi_update(a.z[q], c.bz[q], op3_z(g, u, k, j, i), jacobi_weight(omega, c.iz[q]));
        return;
    }
    if (i > g.nx || j > g.ny || k > g.nz) return;
    const size_t q = g.at(k, j, i);
    if (in_vx(g, k, j, i)) {
        const T v = a.x[q];
        ox[q] = unk_x(g, k, j, i) ? jacobi_update(v, c.bx[q], op3_x(g, a, k, j, i), jacobi_weight(omega, c.ix[q])) : v;
    }
    if (in_vy(g, k, j, i)) {
        const T v = a.y[q];
        oy[q] = unk_y(g, k, j, i) ? jacobi_update(v, c.by[q], op3_y(g, a, k, j, i), jacobi_weight(omega, c.iy[q])) : v;
    }
    if (in_vz(g, k, j, i)) {
        const T v = a.z[q];
        oz[q] = unk_z(g, k, j, i) ? jacobi_update(v, c.bz[q], op3_z(g, a, k, j, i), jacobi_weight(omega, c.iz[q])) : v;
    }
}

// copy the wall entries (in extent, not unknowns) of (vx, vy, vz)
template <typename T>
__global__ void k3_copy_walls(G3<T> g, const T *__restrict__ ax, const T *__restrict__ ay, const T *__restrict__ az,
                              T *__restrict__ bx, T *__restrict__ by, T *__restrict__ bz)
{
    const int i = blockIdx.x * B3X + threadIdx.x, j = blockIdx.y * B3Y + threadIdx.y, k = blockIdx.z * B3Z + threadIdx.z;
    if (i > g.nx || j > g.ny || k > g.nz) return;
    const size_t q = g.at(k, j, i);
    if (in_vx(g, k, j, i) && !unk_x(g, k, j, i)) bx[q] = ax[q];
    if (in_vy(g, k, j, i) && !unk_y(g, k, j, i)) by[q] = ay[q];
    if (in_vz(g, k, j, i) && !unk_z(g, k, j, i)) bz[q] = az[q];
}

// ---- RAS-Jacobi on 3D tiles ------------------------------------------------------
constexpr int R3_THREADS = 256;
constexpr int R3_FIELDS = 10; // vx, vy, vz (twice: ping-pong), eta_c and the three edge viscosities

struct Tiles3 {
    int ti, tj, tk, si, sj, sk, ntx, nty, ntz;
};

// tile b of [0, n) cut at s + m T
__host__ __device__ inline void tile_iv(int n, int T, int s, int b, int &lo, int &hi)
{
    const int first = s > 0 ? s : T;
    lo = b == 0 ? 0 : first + (b - 1) * T;
    hi = first + b * T;
    if (hi > n) hi = n;
}

inline int tiles_of(int n, int T, int s)
{
    const int first = s > 0 ? s : T;
    return first >= n ? 1 : 1 + (n - first + T - 1) / T;
}

// accessor of the staged window: explicit plane pointers (the current
// velocity copy and the viscosities) and the window geometry
template <typename T>
struct WAcc {
    const T *px, *py, *pz, *pc, *pxy, *pxz, *pyz;
    int ox0, oy0, oz0, wx, wy;
    __device__ __forceinline__ int idx(int k, int j, int i) const { return ((k - oz0) * wy + (j - oy0)) * wx + (i - ox0); }
    __device__ __forceinline__ T vx(int k, int j, int i) const { return px[idx(k, j, i)]; }
    __device__ __forceinline__ T vy(int k, int j, int i) const { return py[idx(k, j, i)]; }
    __device__ __forceinline__ T vz(int k, int j, int i) const { return pz[idx(k, j, i)]; }
    __device__ __forceinline__ T ec(int k, int j, int i) const { return pc[idx(k, j, i)]; }
    __device__ __forceinline__ T exy(int k, int j, int i) const { return pxy[idx(k, j, i)]; }
    __device__ __forceinline__ T exz(int k, int j, int i) const { return pxz[idx(k, j, i)]; }
    __device__ __forceinline__ T eyz(int k, int j, int i) const { return pyz[idx(k, j, i)]; }
};

// shared-memory planes of a window of S cells: velocity copy 0 (vx, vy, vz),
// copy 1, then eta_c, eta_xy, eta_xz, eta_yz
template <typename T>
__global__ void __launch_bounds__(R3_THREADS) k3_ras(G3<T> g, GAcc<T> a, C3<T> c, T omega, Tiles3 tg, int ks,
                                                    int overlap, T *__restrict__ ox, T *__restrict__ oy,
                                                    T *__restrict__ oz)
{
    extern __shared__ __align__(16) unsigned char r3_raw[];
    T *const sm = reinterpret_cast<T *>(r3_raw);
    const int tile = (int)blockIdx.x;
    const int tbx = tile % tg.ntx, tby = (tile / tg.ntx) % tg.nty, tbz = tile / (tg.ntx * tg.nty);
    int x0, x1, y0, y1, z0, z1;
    tile_iv(g.nx, tg.ti, tg.si, tbx, x0, x1);
    tile_iv(g.ny, tg.tj, tg.sj, tby, y0, y1);
    tile_iv(g.nz, tg.tk, tg.sk, tbz, z0, z1);
    const int h = overlap + 1;
    const int ox0 = x0 - h, oy0 = y0 - h, oz0 = z0 - h;
    const int wx = x1 - x0 + 2 * h, wy = y1 - y0 + 2 * h, wz = z1 - z0 + 2 * h;
    const int S = wx * wy * wz;
    T *const V0 = sm, *const V1 = sm + 3 * S; // the two velocity copies (vx, vy, vz planes)
    T *const EC = sm + 6 * S, *const EXY = sm + 7 * S, *const EXZ = sm + 8 * S, *const EYZ = sm + 9 * S;
    const int tid = (int)threadIdx.x;
    // stage the window (zero outside each field's extent); both velocity
    // copies start from the snapshot, so cells a sweep does not update keep it.
    // A window inside the cells of the grid lies inside every extent and is
    // read without extent tests.  Window cells are visited with incremental
    // indices (one division per thread instead of two per cell).
    const bool inside = ox0 >= 0 && oy0 >= 0 && oz0 >= 0 && ox0 + wx <= g.nx && oy0 + wy <= g.ny && oz0 + wz <= g.nz;
    {
        const int st = R3_THREADS, di = st % wx, dj = (st / wx) % wy, dk = st / (wx * wy);
        int i = tid % wx, j = (tid / wx) % wy, k = tid / (wx * wy);
        for (int e = tid; e < S; e += st) {
            const int gi = ox0 + i, gj = oy0 + j, gk = oz0 + k;
            T u, v, w, ec, exy, exz, eyz;
            if (inside) {
                const size_t q = g.at(gk, gj, gi);
                u = a.x[q]; v = a.y[q]; w = a.z[q];
                ec = a.c[q]; exy = a.xy[q]; exz = a.xz[q]; eyz = a.yz[q];
            } else {
                u = a.vx(gk, gj, gi); v = a.vy(gk, gj, gi); w = a.vz(gk, gj, gi);
                ec = a.ec(gk, gj, gi); exy = a.exy(gk, gj, gi); exz = a.exz(gk, gj, gi); eyz = a.eyz(gk, gj, gi);
            }
            V0[e] = u;
            V0[S + e] = v;
            V0[2 * S + e] = w;
            V1[e] = u;
            V1[S + e] = v;
            V1[2 * S + e] = w;
            EC[e] = ec;
            EXY[e] = exy;
            EXZ[e] = exz;
            EYZ[e] = eyz;
            i += di;
            j += dj;
            k += dk;
            if (i >= wx) {
                i -= wx;
                ++j;
            }
            if (j >= wy) {
                j -= wy;
                ++k;
            }
        }
    }
    __syncthreads();
    WAcc<T> wa;
    wa.pc = EC;
    wa.pxy = EXY;
    wa.pxz = EXZ;
    wa.pyz = EYZ;
    wa.ox0 = ox0;
    wa.oy0 = oy0;
    wa.oz0 = oz0;
    wa.wx = wx;
    wa.wy = wy;
    // local problem: the tile grown by `overlap`, clipped to the grid
    const int lx0 = max(x0 - overlap, 0), lx1 = min(x1 + overlap, g.nx);
    const int ly0 = max(y0 - overlap, 0), ly1 = min(y1 + overlap, g.ny);
    const int lz0 = max(z0 - overlap, 0), lz1 = min(z1 + overlap, g.nz);
    T *cur = V0, *nxt = V1;
    for (int s = 1; s <= ks; ++s) {
        // cells within min(overlap, ks - s) of the tile matter after this sweep
        const int r = min(overlap, ks - s);
        const int cx0 = max(x0 - r, lx0), cx1 = min(x1 + r, lx1);
        const int cy0 = max(y0 - r, ly0), cy1 = min(y1 + r, ly1);
        const int cz0 = max(z0 - r, lz0), cz1 = min(z1 + r, lz1);
        const int nxr = cx1 - cx0, nyr = cy1 - cy0;
        const int npts = nxr * nyr * (cz1 - cz0);
        wa.px = cur;
        wa.py = cur + S;
        wa.pz = cur + 2 * S;
        // the right-hand side and 1/diag are read from global memory (L1/L2 after
        // the first sweep): shared memory holds only the velocity and viscosity
        const int di = R3_THREADS % nxr, dj = (R3_THREADS / nxr) % nyr, dk = R3_THREADS / (nxr * nyr);
        int i = cx0 + tid % nxr, j = cy0 + (tid / nxr) % nyr, k = cz0 + tid / (nxr * nyr);
        for (int e = tid; e < npts; e += R3_THREADS) {
            const int q = wa.idx(k, j, i);
            const size_t gq = g.at(k, j, i);
            T u = cur[q], v = cur[S + q], w = cur[2 * S + q];
            if (unk_x(g, k, j, i)) u = jacobi_update(u, c.bx[gq], op3_x(g, wa, k, j, i), jacobi_weight(omega, c.ix[gq]));
            if (unk_y(g, k, j, i)) v = jacobi_update(v, c.by[gq], op3_y(g, wa, k, j, i), jacobi_weight(omega, c.iy[gq]));
            if (unk_z(g, k, j, i)) w = jacobi_update(w, c.bz[gq], op3_z(g, wa, k, j, i), jacobi_weight(omega, c.iz[gq]));
            nxt[q] = u;
            nxt[S + q] = v;
            nxt[2 * S + q] = w;
            i += di;
            j += dj;
            k += dk;
            if (i >= cx1) {
                i -= nxr;
                ++j;
            }
            if (j >= cy1) {
                j -= nyr;
                ++k;
            }
        }
        __syncthreads();
        // A cell outside this sweep's region keeps a stale value in the copy
        // just written.  No later sweep reads it: the regions shrink by at most
        // one cell per sweep and an update reads one cell beyond its own
        // region, which lies inside this sweep's region or in the Dirichlet
        // ring, whose two copies both hold the snapshot.
        T *const t = cur;
        cur = nxt;
        nxt = t;
    }
    // write back the unknowns of the tile's own cells
    const int tw = x1 - x0, th = y1 - y0, tn = tw * th * (z1 - z0);
    for (int e = tid; e < tn; e += R3_THREADS) {
        const int i = x0 + e % tw, j = y0 + (e / tw) % th, k = z0 + e / (tw * th);
        const int q = wa.idx(k, j, i);
        const size_t gq = g.at(k, j, i);
        if (unk_x(g, k, j, i)) ox[gq] = cur[q];
        if (unk_y(g, k, j, i)) oy[gq] = cur[S + q];
        if (unk_z(g, k, j, i)) oz[gq] = cur[2 * S + q];
    }
}

// ---- RAS-Jacobi on 3D tiles, column form ------------------------------------------
// The same map as k3_ras (and, for overlap >= k - 1, as k3_jacobi), for windows
// of 16 to 32 x at most WY x at most WZ cells: one warp per window row (lane =
// x, warp = y), each thread holding its window column of WZ cells (z) of the
// velocity and the four viscosities in registers.  Every flux is formed once
// per sweep by the cell that owns it; x neighbours (velocity and flux) move by
// shuffles, z neighbours are in the thread's own registers, and only the y
// neighbours go through shared memory: the velocity (vx, vy, vz) and the
// three fluxes read across rows (sigma'_xy, Tyy, sigma'_yz), one plane per
// window level and field, rows padded by one on each side; values read
// together sit side by side ({vx, vz}, {sigma'_xy, sigma'_yz}, {b, 1/diag})
// and move as one 8- or 16-byte access.  The right-hand side and 1/diag of
// the levels 1 .. WZ - 2 are copied to shared memory once per tile
// (cp.async, no registers), so the updates read no global memory (from
// global memory they waited on L2 once per level).  (Prefetching the
// windows of the next wave of tiles into L2 with bulk prefetches, at the start
// of a CTA or after its staging, made the kernel slower: 88 against 114
// Gcell-updates/s on 30 x 6 x 6 tiles.)  A sweep is two
// phases, a barrier after each: (A) the row-crossing fluxes from the staged
// velocity, (B) the updates, the remaining fluxes carried along z in
// registers, and the new velocity.  Both phases run over every level as
// straight-line code (the sweep's region selects which results are kept), so
// the compiler interleaves the levels' dependency chains; the window strides
// are compile-time constants.  Every value is the rounded arithmetic of op3_*,
// in its order, so the results equal those of the other kernels bit for bit.
// Window cells outside the tile's window (lanes beyond 2 h + tile width, rows
// and levels beyond 2 h + tile extent) are staged but never updated, and no
// updated cell reads them.
constexpr int RC_FIELDS = 6;
constexpr size_t RC_SMEM_MAX = 227 * 1024;

template <typename T>
struct V2;
template <>
struct V2<float> {
    using type = float2;
    static __device__ __forceinline__ float2 make(float a, float b) { return make_float2(a, b); }
};
template <>
struct V2<double> {
    using type = double2;
    static __device__ __forceinline__ double2 make(double a, double b) { return make_double2(a, b); }
};

// one element global -> shared, asynchronously; zero-filled when !valid
// (src must still be a valid address)
template <typename T>
__device__ __forceinline__ void cp_async_elem(T *smem, const T *src, bool valid)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    if (sizeof(T) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(s), "l"(src), "r"(valid ? 8 : 0) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(s), "l"(src), "r"(valid ? 4 : 0) : "memory");
}

template <typename T, int WZ, int WY, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k3_ras_col(G3<T> g, GAcc<T> a, C3<T> c, T omega, Tiles3 tg, int ks,
                                                      int overlap, T *__restrict__ ox, T *__restrict__ oy,
                                                      T *__restrict__ oz)
{
    static_assert(32 * WY <= MAXT, "one warp per window row");
    constexpr int PS = (WY + 2) * 32;      // one level of an exchange field
    constexpr int FS = WZ * PS;            // one exchange field
    constexpr int BS = (WZ - 2) * WY * 32; // one field of b / (1/diag)
    extern __shared__ __align__(16) unsigned char rc_raw[];
    T *const sm = reinterpret_cast<T *>(rc_raw);
    const int lane = (int)threadIdx.x, w = (int)threadIdx.y;
    const int tile = (int)blockIdx.x;
    const int tbx = tile % tg.ntx, tby = (tile / tg.ntx) % tg.nty, tbz = tile / (tg.ntx * tg.nty);
    int x0, x1, y0, y1, z0, z1;
    tile_iv(g.nx, tg.ti, tg.si, tbx, x0, x1);
    tile_iv(g.ny, tg.tj, tg.sj, tby, y0, y1);
    tile_iv(g.nz, tg.tk, tg.sk, tbz, z0, z1);
    const int h = overlap + 1;
    const int ox0 = x0 - h, oy0 = y0 - h, oz0 = z0 - h;
    const int gi = ox0 + lane, gj = oy0 + w;
    // this thread's entries (level stride PS): the exchange planes {vx, vz},
    // vy, {sigma'_xy, sigma'_yz} and Tyy at row w + 1 of each level, and the
    // pairs {b, 1/diag} of x, y, z (component stride BS) at row w of each
    // level 1 .. WZ - 2
    using T2 = typename V2<T>::type;
    T2 *const pxz = reinterpret_cast<T2 *>(sm) + (w + 1) * 32 + lane;
    T *const pvy = sm + 2 * FS + (w + 1) * 32 + lane;
    T2 *const pf = reinterpret_cast<T2 *>(sm + 3 * FS) + (w + 1) * 32 + lane;
    T *const pyy = sm + 5 * FS + (w + 1) * 32 + lane;
    T2 *const pbw = reinterpret_cast<T2 *>(sm + RC_FIELDS * FS) + w * 32 + lane;
    if (w >= 1 && w < WY - 1) { // the rows a sweep can update
        const bool xv_ = gi >= 0 && gi <= g.nx, xc = gi >= 0 && gi < g.nx;
        const bool yc = gj >= 0 && gj < g.ny, yv = gj >= 0 && gj <= g.ny;
#pragma unroll
        for (int kk = 1; kk < WZ - 1; ++kk) {
            const int gk = oz0 + kk;
            const bool zc = gk >= 0 && gk < g.nz, zv = gk >= 0 && gk <= g.nz;
            const bool okx = xv_ && yc && zc, oky = xc && yv && zc, okz = xc && yc && zv;
            const size_t q = (okx || oky || okz) ? g.at(gk, gj, gi) : 0;
            T *const d = reinterpret_cast<T *>(pbw + (kk - 1) * WY * 32);
            cp_async_elem(d, c.bx + (okx ? q : 0), okx);
            cp_async_elem(d + 1, c.ix + (okx ? q : 0), okx);
            cp_async_elem(d + 2 * BS, c.by + (oky ? q : 0), oky);
            cp_async_elem(d + 2 * BS + 1, c.iy + (oky ? q : 0), oky);
            cp_async_elem(d + 4 * BS, c.bz + (okz ? q : 0), okz);
            cp_async_elem(d + 4 * BS + 1, c.iz + (okz ? q : 0), okz);
        }
    }
    T vx[WZ], vy[WZ], vz[WZ], ec[WZ], exy[WZ], exz[WZ], eyz[WZ];
    // stage the column (zero outside each field's extent); a window inside
    // the cells of the grid lies inside every extent and is read without tests
    const bool inside = ox0 >= 0 && oy0 >= 0 && oz0 >= 0 && ox0 + 32 <= g.nx && oy0 + WY <= g.ny && oz0 + WZ <= g.nz;
    if (inside) {
        const size_t q0 = g.at(oz0, gj, gi);
#pragma unroll
        for (int kk = 0; kk < WZ; ++kk) {
            const size_t q = q0 + (size_t)kk * g.plane;
            vx[kk] = a.x[q];
            vy[kk] = a.y[q];
            vz[kk] = a.z[q];
            ec[kk] = a.c[q];
            exy[kk] = a.xy[q];
            exz[kk] = a.xz[q];
            eyz[kk] = a.yz[q];
        }
    } else {
#pragma unroll
        for (int kk = 0; kk < WZ; ++kk) {
            const int gk = oz0 + kk;
            vx[kk] = a.vx(gk, gj, gi);
            vy[kk] = a.vy(gk, gj, gi);
            vz[kk] = a.vz(gk, gj, gi);
            ec[kk] = a.ec(gk, gj, gi);
            exy[kk] = a.exy(gk, gj, gi);
            exz[kk] = a.exz(gk, gj, gi);
            eyz[kk] = a.eyz(gk, gj, gi);
        }
    }
#pragma unroll
    for (int kk = 0; kk < WZ; ++kk) {
        pxz[kk * PS] = V2<T>::make(vx[kk], vz[kk]);
        pvy[kk * PS] = vy[kk];
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    const int lx0 = max(x0 - overlap, 0), lx1 = min(x1 + overlap, g.nx);
    const int ly0 = max(y0 - overlap, 0), ly1 = min(y1 + overlap, g.ny);
    const int lz0 = max(z0 - overlap, 0), lz1 = min(z1 + overlap, g.nz);
    const unsigned full = 0xffffffffu;
    for (int s = 1; s <= ks; ++s) {
        // cells within min(overlap, ks - s) of the tile are updated; in window
        // coordinates the lanes [ax0, ax1), rows [ay0, ay1) and levels
        // [az0, az1), all inside [1, extent - 1)
        const int r = min(overlap, ks - s);
        const int ax0 = max(x0 - r, lx0) - ox0, ax1 = min(x1 + r, lx1) - ox0;
        const int ay0 = max(y0 - r, ly0) - oy0, ay1 = min(y1 + r, ly1) - oy0;
        const int az0 = max(z0 - r, lz0) - oz0, az1 = min(z1 + r, lz1) - oz0;
        // (A) sigma'_xy, Tyy and sigma'_yz of rows ay0 - 1 .. ay1, levels 1 .. WZ - 1
        if (w >= ay0 - 1 && w <= ay1) {
#pragma unroll
            for (int kk = 1; kk < WZ; ++kk) {
                const T vys = __shfl_up_sync(full, vy[kk], 1);
                const T2 xzs = pxz[kk * PS - 32]; // {vx, vz} of row w - 1
                const T vyn = pvy[kk * PS + 32];
                const T sxy = r_mul(exy[kk], r_fma(r_sub(vx[kk], xzs.x), g.ihy, r_mul(r_sub(vy[kk], vys), g.ihx)));
                const T syz = r_mul(eyz[kk], r_fma(r_sub(vy[kk], vy[kk - 1]), g.ihz, r_mul(r_sub(vz[kk], xzs.y), g.ihy)));
                pf[kk * PS] = V2<T>::make(sxy, syz);
                pyy[kk * PS] = r_mul(r_mul(r_add(ec[kk], ec[kk]), g.ihy2), r_sub(vyn, vy[kk]));
            }
        }
        __syncthreads();
        // (B) the updates of rows ay0 .. ay1 - 1; sigma'_xz(kk) and Tzz(kk - 1)
        // are carried from the level below, all formed from the velocity
        // before this sweep (level kk's update reads no level below kk)
        if (w >= ay0 && w < ay1) {
            const bool xin = lane >= ax0 && lane < ax1;
            const bool ux = xin && gi >= 1, uy = xin && gj >= 1;
            T sxz = r_mul(exz[1], r_fma(r_sub(vx[1], vx[0]), g.ihz, r_mul(r_sub(vz[1], __shfl_up_sync(full, vz[1], 1)), g.ihx)));
            T tzz_d = r_mul(r_mul(r_add(ec[0], ec[0]), g.ihz2), r_sub(vz[1], vz[0]));
            T2 fc = pf[PS]; // {sigma'_xy, sigma'_yz} of this row, carried up the levels
#pragma unroll
            for (int kk = 1; kk < WZ - 1; ++kk) {
                const T vxe = __shfl_down_sync(full, vx[kk], 1);
                const T txx_c = r_mul(r_mul(r_add(ec[kk], ec[kk]), g.ihx2), r_sub(vxe, vx[kk]));
                const T txx_w = __shfl_up_sync(full, txx_c, 1);
                const T vzw_u = __shfl_up_sync(full, vz[kk + 1], 1);
                const T sxz_u =
                    r_mul(exz[kk + 1], r_fma(r_sub(vx[kk + 1], vx[kk]), g.ihz, r_mul(r_sub(vz[kk + 1], vzw_u), g.ihx)));
                const T tzz_c = r_mul(r_mul(r_add(ec[kk], ec[kk]), g.ihz2), r_sub(vz[kk + 1], vz[kk]));
                const T2 fn = pf[kk * PS + 32], fu = pf[(kk + 1) * PS];
                const T tyy_c = pyy[kk * PS], tyy_s = pyy[kk * PS - 32];
                const T sxy_c = fc.x, sxy_n = fn.x, syz_c = fc.y, syz_n = fn.y, syz_u = fu.y;
                fc = fu;
                const T sxy_e = __shfl_down_sync(full, sxy_c, 1);
                const T sxz_e = __shfl_down_sync(full, sxz, 1);
                const T mx = r_add(r_add(r_sub(txx_c, txx_w), r_sub(r_mul(sxy_n, g.ihy), r_mul(sxy_c, g.ihy))),
                                   r_sub(r_mul(sxz_u, g.ihz), r_mul(sxz, g.ihz)));
                const T my = r_add(r_add(r_sub(r_mul(sxy_e, g.ihx), r_mul(sxy_c, g.ihx)), r_sub(tyy_c, tyy_s)),
                                   r_sub(r_mul(syz_u, g.ihz), r_mul(syz_c, g.ihz)));
                const T mz = r_add(r_add(r_sub(r_mul(sxz_e, g.ihx), r_mul(sxz, g.ihx)),
                                         r_sub(r_mul(syz_n, g.ihy), r_mul(syz_c, g.ihy))),
                                   r_sub(tzz_c, tzz_d));
                sxz = sxz_u;
                tzz_d = tzz_c;
                const T2 *const e = pbw + (kk - 1) * WY * 32;
                const T2 ex = e[0], ey = e[BS], ez = e[2 * BS];
                const bool lev = kk >= az0 && kk < az1;
                if (lev && ux) vx[kk] = jacobi_update(vx[kk], ex.x, mx, jacobi_weight(omega, ex.y));
                if (lev && uy) vy[kk] = jacobi_update(vy[kk], ey.x, my, jacobi_weight(omega, ey.y));
                if (lev && xin && oz0 + kk >= 1) vz[kk] = jacobi_update(vz[kk], ez.x, mz, jacobi_weight(omega, ez.y));
                pxz[kk * PS] = V2<T>::make(vx[kk], vz[kk]);
                pvy[kk * PS] = vy[kk];
            }
        }
        __syncthreads();
    }
    // write back the unknowns of the tile's own cells
    if (w >= h && w < h + (y1 - y0) && lane >= h && lane < h + (x1 - x0)) {
        const size_t q0 = g.at(oz0, gj, gi);
#pragma unroll
        for (int kk = 1; kk < WZ - 1; ++kk) {
            if (kk >= h && kk < h + (z1 - z0)) {
                const size_t q = q0 + (size_t)kk * g.plane;
                if (gi >= 1) ox[q] = vx[kk];
                if (gj >= 1) oy[q] = vy[kk];
                if (oz0 + kk >= 1) oz[q] = vz[kk];
            }
        }
    }
}

// the column kernels: FP32 up to 16 rows (8 levels) or 12 rows (12 levels), FP64 8 x 8
template <typename T>
struct RasCol {
    static constexpr int MAXT = sizeof(T) == 4 ? 512 : 256;
};

size_t rc_smem(int wz, int wy, size_t es)
{
    return ((size_t)RC_FIELDS * wz * (wy + 2) + (size_t)6 * (wz - 2) * wy) * 32 * es;
}

// the column kernel's window (levels wz, rows wy) for a tile; wz = 0 when it
// does not apply (the window must span 16 to 32 lanes and fit one of the
// instantiated shapes and the shared memory)
template <typename T>
void ras_col_shape(int ti, int tj, int tk, int overlap, int nx, int ny, int nz, int &wz, int &wy)
{
    const int h = overlap + 1;
    const int wx = std::min(ti, nx) + 2 * h, ny_ = std::min(tj, ny) + 2 * h, nz_ = std::min(tk, nz) + 2 * h;
    wz = 0;
    wy = 0;
    if (wx < 16 || wx > 32) return;
    if (sizeof(T) == 8) {
        if (nz_ <= 8 && ny_ <= 8) wz = 8, wy = 8;
    } else if (nz_ <= 8) {
        wz = 8;
        wy = ny_ <= 8 ? 8 : ny_ <= 12 ? 12 : ny_ <= 16 ? 16 : 0;
    } else if (nz_ <= 12) {
        wz = 12;
        wy = ny_ <= 8 ? 8 : ny_ <= 12 ? 12 : 0;
    }
    if (!wy || rc_smem(wz, wy, sizeof(T)) > RC_SMEM_MAX) wz = wy = 0;
}

template <typename T>
using ras_col_fn = void (*)(G3<T>, GAcc<T>, C3<T>, T, Tiles3, int, int, T *, T *, T *);

template <typename T>
ras_col_fn<T> ras_col_kernel(int wz, int wy);
template <>
ras_col_fn<float> ras_col_kernel<float>(int wz, int wy)
{
    if (wz == 8 && wy == 8) return k3_ras_col<float, 8, 8, 512>;
    if (wz == 8 && wy == 12) return k3_ras_col<float, 8, 12, 512>;
    if (wz == 8 && wy == 16) return k3_ras_col<float, 8, 16, 512>;
    if (wz == 12 && wy == 8) return k3_ras_col<float, 12, 8, 512>;
    if (wz == 12 && wy == 12) return k3_ras_col<float, 12, 12, 512>;
    return nullptr;
}
template <>
ras_col_fn<double> ras_col_kernel<double>(int wz, int wy)
{
    if (wz == 8 && wy == 8) return k3_ras_col<double, 8, 8, 256>;
    return nullptr;
}

size_t r3_smem(int ti, int tj, int tk, int overlap, size_t es, int nx, int ny, int nz)
{
    const int h = overlap + 1;
    const size_t wx = (size_t)std::min(ti, nx) + 2 * h, wy = (size_t)std::min(tj, ny) + 2 * h;
    const size_t wz = (size_t)std::min(tk, nz) + 2 * h;
    return (size_t)R3_FIELDS * wx * wy * wz * es;
}

// ---- energy norm ---------------------------------------------------------------------
constexpr int E3_THREADS = 256;
constexpr int E3_BLOCKS = 152 * 4;

__device__ __forceinline__ double warp_sum3(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// partial sums per block (fixed order): r_v^2 / (-diag), (D v)^2 eta_c / lap, f^2 / (-diag)
template <typename T>
__global__ void __launch_bounds__(E3_THREADS) k3_energy(G3<T> g, GAcc<T> a, C3<T> c, const T *__restrict__ fx,
                                                        const T *__restrict__ fy, const T *__restrict__ fz,
                                                        const T *__restrict__ p, double *__restrict__ partials)
{
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    const long long n = (long long)(g.nx + 1) * (g.ny + 1) * (g.nz + 1);
    for (long long e = (long long)blockIdx.x * E3_THREADS + threadIdx.x; e < n; e += (long long)gridDim.x * E3_THREADS) {
        const int i = (int)(e % (g.nx + 1)), j = (int)((e / (g.nx + 1)) % (g.ny + 1)), k = (int)(e / ((long long)(g.nx + 1) * (g.ny + 1)));
        const size_t q = g.at(k, j, i);
        if (unk_x(g, k, j, i)) {
            const T m = op3_x(g, a, k, j, i), d = diag3_x(g, a, k, j, i);
            const T b = p ? r_fma(r_sub(p[q], p[q - 1]), g.ihx, fx[q]) : fx[q];
            const double r = (double)r_sub(b, m), w = -1.0 / (double)d, f = (double)fx[q];
            s0 = fma(r * r, w, s0);
            s2 = fma(f * f, w, s2);
        }
        if (unk_y(g, k, j, i)) {
            const T m = op3_y(g, a, k, j, i), d = diag3_y(g, a, k, j, i);
            const T b = p ? r_fma(r_sub(p[q], p[q - g.pitch]), g.ihy, fy[q]) : fy[q];
            const double r = (double)r_sub(b, m), w = -1.0 / (double)d, f = (double)fy[q];
            s0 = fma(r * r, w, s0);
            s2 = fma(f * f, w, s2);
        }
        if (unk_z(g, k, j, i)) {
            const T m = op3_z(g, a, k, j, i), d = diag3_z(g, a, k, j, i);
            const T b = p ? r_fma(r_sub(p[q], p[q - g.plane]), g.ihz, fz[q]) : fz[q];
            const double r = (double)r_sub(b, m), w = -1.0 / (double)d, f = (double)fz[q];
            s0 = fma(r * r, w, s0);
            s2 = fma(f * f, w, s2);
        }
        if (in_c(g, k, j, i)) {
            const double dv = (double)r_add(r_add(r_mul(r_sub(a.x[q + 1], a.x[q]), g.ihx),
                                                  r_mul(r_sub(a.y[q + g.pitch], a.y[q]), g.ihy)),
                                            r_mul(r_sub(a.z[q + g.plane], a.z[q]), g.ihz));
            s1 = fma(dv * dv, (double)c.ec[q] / g.lap, s1);
        }
    }
    __shared__ double sh[3][E3_THREADS / 32];
    s0 = warp_sum3(s0);
    s1 = warp_sum3(s1);
    s2 = warp_sum3(s2);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][wid] = s0;
        sh[1][wid] = s1;
        sh[2][wid] = s2;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int q = 0; q < E3_THREADS / 32; ++q) t += sh[threadIdx.x][q];
        partials[blockIdx.x * 3 + threadIdx.x] = t;
    }
}

__global__ void k3_energy_final(const double *__restrict__ partials, int nb, double *__restrict__ out)
{
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int b = 0; b < nb; ++b) t += partials[b * 3 + threadIdx.x];
        out[threadIdx.x] = t;
    }
}

} // namespace

struct stokes3d_ctx {
    int nx, ny, nz, dtype, pitch;
    double hx, hy, hz;
    size_t elems, esize;
    cudaStream_t stream;
    void *ec = nullptr, *exy = nullptr, *exz = nullptr, *eyz = nullptr;
    void *fx = nullptr, *fy = nullptr, *fz = nullptr, *bx = nullptr, *by = nullptr, *bz = nullptr;
    void *ix = nullptr, *iy = nullptr, *iz = nullptr, *sx = nullptr, *sy = nullptr, *sz = nullptr;
    double *partials = nullptr, *dsum = nullptr, *hsum = nullptr;
    bool have_eta = false, have_f = false;
    long long kernels = 0;
};

namespace {

template <typename T>
G3<T> g3_of(const stokes3d_ctx *c)
{
    return make_g3<T>(c->nx, c->ny, c->nz, c->pitch, c->hx, c->hy, c->hz);
}

template <typename T>
C3<T> c3_of(const stokes3d_ctx *c, bool b_is_f)
{
    C3<T> k;
    k.ec = (const T *)c->ec;
    k.exy = (const T *)c->exy;
    k.exz = (const T *)c->exz;
    k.eyz = (const T *)c->eyz;
    k.bx = (const T *)(b_is_f ? c->fx : c->bx);
    k.by = (const T *)(b_is_f ? c->fy : c->by);
    k.bz = (const T *)(b_is_f ? c->fz : c->bz);
    k.ix = (const T *)c->ix;
    k.iy = (const T *)c->iy;
    k.iz = (const T *)c->iz;
    return k;
}

template <typename T>
int set_viscosity_impl(stokes3d_ctx *c, const void *ec, const void *xy, const void *xz, const void *yz)
{
    const G3<T> g = g3_of<T>(c);
    const dim3 gr = grid3(c->nx + 1, c->ny + 1, c->nz + 1), bl(B3X, B3Y, B3Z);
    k3_coeffs<T><<<gr, bl, 0, c->stream>>>(g, (const T *)ec, (const T *)xy, (const T *)xz, (const T *)yz, (T *)c->ec,
                                          (T *)c->exy, (T *)c->exz, (T *)c->eyz);
    const GAcc<T> a = gacc<T>(g, nullptr, nullptr, nullptr, (const T *)c->ec, (const T *)c->exy, (const T *)c->exz,
                              (const T *)c->eyz);
    // the diagonal reads only the viscosities (the accessor's velocity is unused)
    k3_inv_diag<T><<<gr, bl, 0, c->stream>>>(g, a, (T *)c->ix, (T *)c->iy, (T *)c->iz);
    c->kernels += 2;
    CK(cudaGetLastError());
    return STOKES_OK;
}

template <typename T>
int smooth_impl(stokes3d_ctx *c, T *vx, T *vy, T *vz, const T *p, const stokes3d_smooth_params *prm)
{
    const G3<T> g = g3_of<T>(c);
    const dim3 gr = grid3(c->nx + 1, c->ny + 1, c->nz + 1), bl(B3X, B3Y, B3Z);
    const bool b_is_f = p == nullptr;
    if (!b_is_f) {
        k3_rhs<T><<<gr, bl, 0, c->stream>>>(g, (const T *)c->fx, (const T *)c->fy, (const T *)c->fz, p, (T *)c->bx,
                                           (T *)c->by, (T *)c->bz);
        ++c->kernels;
    }
    const C3<T> k = c3_of<T>(c, b_is_f);
    const T omega = (T)prm->omega;
    // ping-pong between the caller's velocity and the scratch triple; the
    // scratch walls take the caller's Dirichlet values from the first pass
    T *A[3] = {vx, vy, vz}, *B[3] = {(T *)c->sx, (T *)c->sy, (T *)c->sz};
    int passes = 0;
    auto pass_jacobi = [&]() {
        const GAcc<T> a = gacc<T>(g, A[0], A[1], A[2], k.ec, k.exy, k.exz, k.eyz);
        k3_jacobi<T><<<gr, bl, 0, c->stream>>>(g, a, k, omega, B[0], B[1], B[2]);
        ++c->kernels;
    };
    if (prm->variant == STOKES_JACOBI_FUSED) {
        for (int s = 0; s < prm->sweeps; ++s) {
            pass_jacobi();
            std::swap(A[0], B[0]);
            std::swap(A[1], B[1]);
            std::swap(A[2], B[2]);
            ++passes;
        }
    } else {
        const int ti = prm->tile_i, tj = prm->tile_j, tk = prm->tile_k;
        // windows of 16 to 32 lanes take the column kernel, others the general one
        int wz = 0, wyk = 0;
        ras_col_shape<T>(ti, tj, tk, prm->overlap, c->nx, c->ny, c->nz, wz, wyk);
        const ras_col_fn<T> col = ras_col_kernel<T>(wz, wyk);
        const size_t smem = col ? rc_smem(wz, wyk, sizeof(T))
                                : r3_smem(ti, tj, tk, prm->overlap, sizeof(T), c->nx, c->ny, c->nz);
        if (col)
            CK(cudaFuncSetAttribute(col, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        else
            CK(cudaFuncSetAttribute(k3_ras<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        // every unknown of the output is written by its tile; the scratch takes
        // the caller's wall values once
        const int n_outer = (prm->sweeps + prm->k - 1) / prm->k;
        if (n_outer > 0) {
            k3_copy_walls<T><<<gr, bl, 0, c->stream>>>(g, A[0], A[1], A[2], B[0], B[1], B[2]);
            ++c->kernels;
        }
        for (int t = 0; t < n_outer; ++t) {
            const int ks = (t == n_outer - 1) ? prm->sweeps - (n_outer - 1) * prm->k : prm->k;
            int sh[3] = {0, 0, 0};
            if (prm->shift_mode == STOKES_SHIFT_SPLITMIX) {
                sh[0] = (int)(splitmix64(prm->seed, 3u * (uint64_t)t) % (uint64_t)ti);
                sh[1] = (int)(splitmix64(prm->seed, 3u * (uint64_t)t + 1u) % (uint64_t)tj);
                sh[2] = (int)(splitmix64(prm->seed, 3u * (uint64_t)t + 2u) % (uint64_t)tk);
            } else if (prm->shift_mode == STOKES_SHIFT_LIST) {
                for (int d = 0; d < 3; ++d) sh[d] = prm->shifts[3 * t + d];
                if (sh[0] < 0 || sh[0] >= ti || sh[1] < 0 || sh[1] >= tj || sh[2] < 0 || sh[2] >= tk)
                    return STOKES_ERR_ARG;
            }
            Tiles3 tg;
            tg.ti = ti;
            tg.tj = tj;
            tg.tk = tk;
            tg.si = sh[0];
            tg.sj = sh[1];
            tg.sk = sh[2];
            tg.ntx = tiles_of(c->nx, ti, sh[0]);
            tg.nty = tiles_of(c->ny, tj, sh[1]);
            tg.ntz = tiles_of(c->nz, tk, sh[2]);
            const GAcc<T> a = gacc<T>(g, A[0], A[1], A[2], k.ec, k.exy, k.exz, k.eyz);
            if (col)
                col<<<tg.ntx * tg.nty * tg.ntz, dim3(32, (unsigned)wyk), smem, c->stream>>>(
                    g, a, k, omega, tg, ks, prm->overlap, B[0], B[1], B[2]);
            else
                k3_ras<T><<<tg.ntx * tg.nty * tg.ntz, R3_THREADS, smem, c->stream>>>(g, a, k, omega, tg, ks,
                                                                                    prm->overlap, B[0], B[1], B[2]);
            ++c->kernels;
            std::swap(A[0], B[0]);
            std::swap(A[1], B[1]);
            std::swap(A[2], B[2]);
            ++passes;
        }
    }
    CK(cudaGetLastError());
    if (passes & 1) { // the result is in the scratch triple: copy it back
        const size_t nb = c->elems * c->esize;
        CK(cudaMemcpyAsync(vx, A[0], nb, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(vy, A[1], nb, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(vz, A[2], nb, cudaMemcpyDeviceToDevice, c->stream));
    }
    return STOKES_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

int alloc3(stokes3d_ctx *c, void **p)
{
    CK(cudaMalloc(p, c->elems * c->esize));
    CK(cudaMemsetAsync(*p, 0, c->elems * c->esize, c->stream));
    return STOKES_OK;
}

} // namespace

extern "C" {

int stokes3d_create(int nx, int ny, int nz, double lx, double ly, double lz, int dtype, void *cuda_stream,
                    stokes3d_ctx **out)
{
    if (!out) return STOKES_ERR_ARG;
    *out = nullptr;
    if (nx < 2 || ny < 2 || nz < 2 || nx > 4096 || ny > 4096 || nz > 4096 || !(lx > 0.0) || !(ly > 0.0) || !(lz > 0.0))
        return STOKES_ERR_ARG;
    if (dtype != STOKES_F32 && dtype != STOKES_F64) return STOKES_ERR_ARG;
    const size_t pitch = ((size_t)(nx + 1) + 31) / 32 * 32;
    const size_t elems = (size_t)(nz + 1) * (size_t)(ny + 1) * pitch;
    if (elems >= (size_t)1 << 40) return STOKES_ERR_ARG;
    stokes3d_ctx *c = new (std::nothrow) stokes3d_ctx();
    if (!c) return STOKES_ERR_OOM;
    c->nx = nx;
    c->ny = ny;
    c->nz = nz;
    c->hx = lx / nx;
    c->hy = ly / ny;
    c->hz = lz / nz;
    c->dtype = dtype;
    c->esize = dtype == STOKES_F64 ? 8 : 4;
    c->pitch = (int)pitch;
    c->elems = elems;
    c->stream = (cudaStream_t)cuda_stream;
    int st = STOKES_OK;
    void **f[] = {&c->ec, &c->exy, &c->exz, &c->eyz, &c->fx, &c->fy, &c->fz, &c->bx, &c->by, &c->bz,
                  &c->ix, &c->iy, &c->iz, &c->sx, &c->sy, &c->sz};
    for (void **p : f)
        if ((st = alloc3(c, p)) != STOKES_OK) break;
    if (st == STOKES_OK) {
        cudaError_t e = cudaMalloc(&c->partials, (size_t)E3_BLOCKS * 3 * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&c->dsum, 3 * sizeof(double));
        if (e == cudaSuccess) e = cudaMallocHost(&c->hsum, 3 * sizeof(double));
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "stokes3d_create");
    }
    if (st != STOKES_OK) {
        stokes3d_destroy(c);
        return st;
    }
    *out = c;
    return STOKES_OK;
}

int stokes3d_get_layout(const stokes3d_ctx *c, int *pitch_elems, int *plane_rows, size_t *alloc_elems)
{
    if (!c) return STOKES_ERR_ARG;
    if (pitch_elems) *pitch_elems = c->pitch;
    if (plane_rows) *plane_rows = c->ny + 1;
    if (alloc_elems) *alloc_elems = c->elems;
    return STOKES_OK;
}

int stokes3d_set_viscosity(stokes3d_ctx *c, const void *eta_c, const void *eta_xy, const void *eta_xz,
                           const void *eta_yz)
{
    if (!c || !eta_c || !eta_xy || !eta_xz || !eta_yz) return STOKES_ERR_ARG;
    const int st = c->dtype == STOKES_F64 ? set_viscosity_impl<double>(c, eta_c, eta_xy, eta_xz, eta_yz)
                                          : set_viscosity_impl<float>(c, eta_c, eta_xy, eta_xz, eta_yz);
    if (st == STOKES_OK) c->have_eta = true;
    return st;
}

int stokes3d_set_rhs(stokes3d_ctx *c, const void *fx, const void *fy, const void *fz)
{
    if (!c || !fx || !fy || !fz) return STOKES_ERR_ARG;
    // f at the unknowns, zero elsewhere: f is then b = f - G p for p = 0
    const dim3 gr = grid3(c->nx + 1, c->ny + 1, c->nz + 1), bl(B3X, B3Y, B3Z);
    if (c->dtype == STOKES_F64)
        k3_rhs<double><<<gr, bl, 0, c->stream>>>(g3_of<double>(c), (const double *)fx, (const double *)fy,
                                                 (const double *)fz, nullptr, (double *)c->fx, (double *)c->fy,
                                                 (double *)c->fz);
    else
        k3_rhs<float><<<gr, bl, 0, c->stream>>>(g3_of<float>(c), (const float *)fx, (const float *)fy,
                                                (const float *)fz, nullptr, (float *)c->fx, (float *)c->fy,
                                                (float *)c->fz);
    ++c->kernels;
    CK(cudaGetLastError());
    c->have_f = true;
    return STOKES_OK;
}

int stokes3d_apply_operator(stokes3d_ctx *c, const void *vx, const void *vy, const void *vz, const void *p, void *ox,
                            void *oy, void *oz)
{
    if (!c || !vx || !vy || !vz || !ox || !oy || !oz) return STOKES_ERR_ARG;
    if (!c->have_eta) return STOKES_ERR_STATE;
    const dim3 gr = grid3(c->nx + 1, c->ny + 1, c->nz + 1), bl(B3X, B3Y, B3Z);
    if (c->dtype == STOKES_F64) {
        const G3<double> g = g3_of<double>(c);
        const GAcc<double> a = gacc<double>(g, (const double *)vx, (const double *)vy, (const double *)vz,
                                            (const double *)c->ec, (const double *)c->exy, (const double *)c->exz,
                                            (const double *)c->eyz);
        k3_apply<double><<<gr, bl, 0, c->stream>>>(g, a, (const double *)p, (double *)ox, (double *)oy, (double *)oz);
    } else {
        const G3<float> g = g3_of<float>(c);
        const GAcc<float> a = gacc<float>(g, (const float *)vx, (const float *)vy, (const float *)vz,
                                          (const float *)c->ec, (const float *)c->exy, (const float *)c->exz,
                                          (const float *)c->eyz);
        k3_apply<float><<<gr, bl, 0, c->stream>>>(g, a, (const float *)p, (float *)ox, (float *)oy, (float *)oz);
    }
    ++c->kernels;
    CK(cudaGetLastError());
    return STOKES_OK;
}

int stokes3d_smooth(stokes3d_ctx *c, void *vx, void *vy, void *vz, const void *p, const stokes3d_smooth_params *prm)
{
    if (!c || !vx || !vy || !vz || !prm) return STOKES_ERR_ARG;
    if (!aligned16(vx) || !aligned16(vy) || !aligned16(vz) || !aligned16(p)) return STOKES_ERR_ARG;
    if (prm->sweeps < 0 || !(prm->omega > 0.0) || !std::isfinite(prm->omega)) return STOKES_ERR_ARG;
    if (prm->variant != STOKES_JACOBI_FUSED && prm->variant != STOKES_RAS) return STOKES_ERR_ARG;
    if (prm->variant == STOKES_RAS) {
        if (prm->k < 1 || prm->overlap < 0 || prm->tile_i < 1 || prm->tile_j < 1 || prm->tile_k < 1) return STOKES_ERR_ARG;
        if (prm->shift_mode < STOKES_SHIFT_NONE || prm->shift_mode > STOKES_SHIFT_LIST) return STOKES_ERR_ARG;
        if (prm->shift_mode == STOKES_SHIFT_LIST && prm->sweeps > 0 && !prm->shifts) return STOKES_ERR_ARG;
        int maxs = 0, dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&maxs, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
            cudaGetLastError();
            return STOKES_ERR_CUDA;
        }
        int wz = 0, wy = 0;
        if (c->dtype == STOKES_F64)
            ras_col_shape<double>(prm->tile_i, prm->tile_j, prm->tile_k, prm->overlap, c->nx, c->ny, c->nz, wz, wy);
        else
            ras_col_shape<float>(prm->tile_i, prm->tile_j, prm->tile_k, prm->overlap, c->nx, c->ny, c->nz, wz, wy);
        const bool col = wz > 0;
        if (!col &&
            r3_smem(prm->tile_i, prm->tile_j, prm->tile_k, prm->overlap, c->esize, c->nx, c->ny, c->nz) > (size_t)maxs)
            return STOKES_ERR_ARG;
    }
    if (!c->have_eta || !c->have_f) return STOKES_ERR_STATE;
    if (c->dtype == STOKES_F64)
        return smooth_impl<double>(c, (double *)vx, (double *)vy, (double *)vz, (const double *)p, prm);
    return smooth_impl<float>(c, (float *)vx, (float *)vy, (float *)vz, (const float *)p, prm);
}

int stokes3d_residual_energy_norm(stokes3d_ctx *c, const void *vx, const void *vy, const void *vz, const void *p,
                                  double out[3])
{
    if (!c || !vx || !vy || !vz || !out) return STOKES_ERR_ARG;
    if (!c->have_eta || !c->have_f) return STOKES_ERR_STATE;
    if (c->dtype == STOKES_F64) {
        const G3<double> g = g3_of<double>(c);
        const GAcc<double> a = gacc<double>(g, (const double *)vx, (const double *)vy, (const double *)vz,
                                            (const double *)c->ec, (const double *)c->exy, (const double *)c->exz,
                                            (const double *)c->eyz);
        k3_energy<double><<<E3_BLOCKS, E3_THREADS, 0, c->stream>>>(g, a, c3_of<double>(c, true), (const double *)c->fx,
                                                                   (const double *)c->fy, (const double *)c->fz,
                                                                   (const double *)p, c->partials);
    } else {
        const G3<float> g = g3_of<float>(c);
        const GAcc<float> a = gacc<float>(g, (const float *)vx, (const float *)vy, (const float *)vz,
                                          (const float *)c->ec, (const float *)c->exy, (const float *)c->exz,
                                          (const float *)c->eyz);
        k3_energy<float><<<E3_BLOCKS, E3_THREADS, 0, c->stream>>>(g, a, c3_of<float>(c, true), (const float *)c->fx,
                                                                  (const float *)c->fy, (const float *)c->fz,
                                                                  (const float *)p, c->partials);
    }
    k3_energy_final<<<1, 32, 0, c->stream>>>(c->partials, E3_BLOCKS, c->dsum);
    c->kernels += 2;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(c->hsum, c->dsum, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    std::memcpy(out, c->hsum, 3 * sizeof(double));
    return STOKES_OK;
}

int stokes3d_kernels(const stokes3d_ctx *c, long long *kernels)
{
    if (!c || !kernels) return STOKES_ERR_ARG;
    *kernels = c->kernels;
    return STOKES_OK;
}

int stokes3d_destroy(stokes3d_ctx *c)
{
    if (!c) return STOKES_OK;
    if (c->stream) cudaStreamSynchronize(c->stream);
    void *f[] = {c->ec, c->exy, c->exz, c->eyz, c->fx, c->fy, c->fz, c->bx, c->by, c->bz,
                 c->ix, c->iy, c->iz, c->sx, c->sy, c->sz, c->partials, c->dsum};
    for (void *p : f)
        if (p) cudaFree(p);
    if (c->hsum) cudaFreeHost(c->hsum);
    delete c;
    return STOKES_OK;
}

} // extern "C"
