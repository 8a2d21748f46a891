// sweep_kernels.cu -- the global-memory smoothers of Sec. 5 of arXiv
// 2509.19061: damped Jacobi as separate vx / vy passes (Sec. 5 (ii)), fused
// Jacobi (Sec. 4.1, Sec. 5 (iii)) and red-black Gauss-Seidel (Sec. 5 (i)).
//
// Jacobi (k_jacobi_rows).  A warp owns a strip of 30 x VW columns (VW = 16 B
// / element: 4 FP32, 2 FP64 values per lane) and marches up a band of rows.
// Each lane loads one 16-byte vector per field and row, so every load is one
// coalesced 512-byte line per warp; lanes 0 and 31 load the strip's left and
// right neighbour columns and are not stored.  Per row the warp forms each
// flux once (Txx and Tyy at the cells, the shear at the nodes of the row
// above) and keeps the fluxes and velocities of the row below in registers,
// so every field is read from memory once per sweep; horizontal neighbours
// come from the next lane by shuffles.  The arithmetic is that of
// stencil.cuh operation for operation, so the results equal those of the
// tile kernels bit for bit.  FP32 forms 1/diag(M) from the viscosity on the
// fly (two fewer fields to read; the kernel is memory-bound); FP64 reads the
// precomputed 1/diag arrays (an FP64 reciprocal costs more than the bytes).
//
// Red-black Gauss-Seidel (k_rbgs_tile).  One launch runs a whole sweep, the
// four half-sweeps vx-red, vx-black, vy-red, vy-black, on a tile grown by a
// halo: a half-sweep's points depend on the previous half-sweeps only
// within one cell, so vx-red runs on the tile grown by 3 cells, vx-black by
// 2, vy-red by 1 and vy-black on the tile itself, from a window grown by 4
// cells staged in shared memory.  The tile writes its own unknowns to a
// second buffer (every tile reads the same input), so the result is the
// in-place sweep's, bit for bit: within one half-sweep no point of a colour
// reads another point of that colour.  Every field is read from DRAM about
// once per sweep instead of once per half-sweep.
#include <algorithm>

#include "internal.h"
#include "stencil.cuh"

namespace stokes {

namespace {

// N values of T as one vector load or store (8 or 16 bytes)
template <typename T, int N>
struct VecT;
template <>
struct VecT<float, 4> {
    using V = float4;
};
template <>
struct VecT<float, 2> {
    using V = float2;
};
template <>
struct VecT<double, 2> {
    using V = double2;
};

// one vector of VW values of field `f` at (row j, column c) into a[], zero
// where the row is outside [0, rows) or the column is at or beyond `cols`;
// the vector itself is read only if it lies inside the array (row <= ny,
// column inside the pitch, which is a multiple of 32 elements)
template <int VW, typename T>
__device__ __forceinline__ void ld_row(const T *__restrict__ f, const GridDesc<T> &g, int j, int c, int rows, int cols,
                                       T (&a)[VW])
{
    using V = typename VecT<T, VW>::V;
    if (j >= 0 && j < rows && c >= 0 && c < g.pitch) {
        const V v = *reinterpret_cast<const V *>(f + (size_t)j * g.pitch + c);
        const T *e = reinterpret_cast<const T *>(&v);
#pragma unroll
        for (int k = 0; k < VW; ++k) a[k] = (c + k < cols) ? e[k] : T(0);
    } else {
#pragma unroll
        for (int k = 0; k < VW; ++k) a[k] = T(0);
    }
}

// store the elements of a[] whose column is below `cols` (one vector store
// when all are)
template <int VW, typename T>
__device__ __forceinline__ void st_row(T *__restrict__ f, const GridDesc<T> &g, int j, int c, int cols,
                                       const T (&a)[VW])
{
    using V = typename VecT<T, VW>::V;
    T *p = f + (size_t)j * g.pitch + c;
    if (c + VW <= cols) {
        V v;
        T *e = reinterpret_cast<T *>(&v);
#pragma unroll
        for (int k = 0; k < VW; ++k) e[k] = a[k];
        *reinterpret_cast<V *>(p) = v;
    } else {
#pragma unroll
        for (int k = 0; k < VW; ++k)
            if (c + k < cols) p[k] = a[k];
    }
}

__device__ __forceinline__ float shfl_up1(float v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ float shfl_dn1(float v) { return __shfl_down_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_up1(double v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_dn1(double v) { return __shfl_down_sync(0xffffffffu, v, 1); }

// 16-byte asynchronous global-to-shared copies (cp.async, no register
// staging): the row loads of the next iterations stay in flight while a
// warp computes, without holding registers
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

constexpr int JR_WARPS = 4; // warps per block, neighbouring column strips

// Row fields one iteration j of jacobi_rows reads: vx, vy and eta_n of row
// j + 1, eta_c of row j, then bx, by (for the components updated) and, with
// INV, 1/diag of row j.
template <bool DX, bool DY, bool INV>
struct JrFields {
    static constexpr int BX = 4, BY = 4 + (DX ? 1 : 0);
    static constexpr int IX = BY + (DY ? 1 : 0), IY = IX + ((INV && DX) ? 1 : 0);
    static constexpr int N = IY + ((INV && DY) ? 1 : 0);
};

// Staged row buffer of one warp: JR_PD iterations x N fields x 32 lanes x 16 B.
constexpr int JR_PD = 3;

// One damped Jacobi pass over rows [j0, j0 + rows) of cells (row ny holds
// only vy walls).  DX / DY: update vx / vy (both read the old velocity);
// INV: read 1/diag(M) from c.inv_dx / c.inv_dy, else form it.  Writes the
// unknowns and walls of (ox, oy), nothing else.  The row loads of iterations
// j + 1 .. j + JR_PD - 1 are in flight (cp.async into the warp's `stage`)
// while iteration j computes.
template <typename T, int VW, bool DX, bool DY, bool INV, int SQM>
__device__ __forceinline__ void jacobi_rows(const GridDesc<T> &g, const Coeffs<T> &c, T omega,
                                            const T *__restrict__ vx, const T *__restrict__ vy, T *__restrict__ ox,
                                            T *__restrict__ oy, int rows, int strip, T *stage)
{
    using F = JrFields<DX, DY, INV>;
    using V = typename VecT<T, VW>::V;
    constexpr int OWN = 30 * VW;
    const int lane = (int)threadIdx.x & 31;
    const int w0 = strip * OWN;
    if (w0 > g.nx) return; // whole warp: no owned column in range
    const int c0 = w0 - VW + lane * VW;
    const bool own = lane >= 1 && lane <= 30;
    const int j0 = (int)blockIdx.y * rows;
    const int j1 = min(j0 + rows, g.ny + 1);
    const int nx = g.nx, ny = g.ny;
    const int cx = nx + 1, cy = nx; // columns of vx / eta_n and of vy / eta_c
    const bool col_ok = c0 >= 0 && c0 < g.pitch;
    V *const st = reinterpret_cast<V *>(stage);

    // the row (and its row count) field f of iteration j reads
    auto src = [&](int f, int j, int &row, int &nrows) -> const T * {
        switch (f) {
        case 0: row = j + 1; nrows = ny; return vx;
        case 1: row = j + 1; nrows = ny + 1; return vy;
        case 2: row = j + 1; nrows = ny + 1; return c.eta_n;
        case 3: row = j; nrows = ny; return c.eta_c;
        default: break;
        }
        row = j;
        if (DX && f == F::BX) { nrows = ny; return c.bx; }
        if (DY && f == F::BY) { nrows = ny + 1; return c.by; }
        if (INV && DX && f == F::IX) { nrows = ny; return c.inv_dx; }
        nrows = ny + 1;
        return c.inv_dy;
    };
    // enqueue the row loads of iteration j into stage slot j % JR_PD (one
    // commit group per iteration, empty past the band)
    auto issue = [&](int j) {
        if (j < j1 && col_ok) {
            V *const slot = st + (j % JR_PD) * F::N * 32 + lane;
#pragma unroll
            for (int f = 0; f < F::N; ++f) {
                int row, nrows;
                const T *p = src(f, j, row, nrows);
                if (row >= 0 && row < nrows) cp_async16(slot + f * 32, p + (size_t)row * g.pitch + c0);
            }
        }
        cp_async_commit();
    };
    // field f of iteration j from the stage, zero outside its extent
    auto take = [&](int f, int j, int cols, T(&a)[VW]) {
        int row, nrows;
        (void)src(f, j, row, nrows);
        if (col_ok && row >= 0 && row < nrows) {
            const V v = st[(j % JR_PD) * F::N * 32 + f * 32 + lane];
            const T *e = reinterpret_cast<const T *>(&v);
#pragma unroll
            for (int k = 0; k < VW; ++k) a[k] = (c0 + k < cols) ? e[k] : T(0);
        } else {
#pragma unroll
            for (int k = 0; k < VW; ++k) a[k] = T(0);
        }
    };
#pragma unroll
    for (int d = 0; d < JR_PD - 1; ++d) issue(j0 + d);

    // state at row j: vx(j), vy(j), eta_n(j), eta_c(j-1), Tyy(j-1) and the
    // scaled shear Sx, Sy at the nodes of row j
    T vxC[VW], vyC[VW], enC[VW], ecS[VW], tyyS[VW], sxC[VW], syC[VW];
    {
        T vxS[VW], vyS[VW];
        ld_row(vx, g, j0, c0, ny, cx, vxC);
        ld_row(vy, g, j0, c0, ny + 1, cy, vyC);
        ld_row(c.eta_n, g, j0, c0, ny + 1, cx, enC);
        ld_row(c.eta_c, g, j0 - 1, c0, ny, cy, ecS);
        ld_row(vx, g, j0 - 1, c0, ny, cx, vxS);
        ld_row(vy, g, j0 - 1, c0, ny + 1, cy, vyS);
        const T vyw = shfl_up1(vyC[VW - 1]);
#pragma unroll
        for (int k = 0; k < VW; ++k) {
            tyyS[k] = flux_n(coef_y(g, ecS[k]), vyC[k], vyS[k]);
            shear_xy<SQM>(g, enC[k], vxC[k], vxS[k], vyC[k], k ? vyC[k - 1] : vyw, sxC[k], syC[k]);
        }
    }
    for (int j = j0; j < j1; ++j) {
        // slot (j - 1) % JR_PD was read in iteration j - 1: refill it
        issue(j + JR_PD - 1);
        cp_async_wait<JR_PD - 1>(); // iteration j's group has landed
        T vxN[VW], vyN[VW], enN[VW], ecC[VW], b[2][VW], iv[2][VW];
        take(0, j, cx, vxN);
        take(1, j, cy, vyN);
        take(2, j, cx, enN);
        take(3, j, cy, ecC);
        if (DX) take(F::BX, j, cx, b[0]);
        if (DY) take(F::BY, j, cy, b[1]);
        if (INV && DX) take(F::IX, j, cx, iv[0]);
        if (INV && DY) take(F::IY, j, cy, iv[1]);
        // the shear at the nodes of row j + 1 (the row above)
        T sxN[VW], syN[VW];
        {
            const T vyw = shfl_up1(vyN[VW - 1]);
#pragma unroll
            for (int k = 0; k < VW; ++k) {
                shear_xy<SQM>(g, enN[k], vxN[k], vxC[k], vyN[k], k ? vyN[k - 1] : vyw, sxN[k], syN[k]);
            }
        }
        T tyy[VW];
#pragma unroll
        for (int k = 0; k < VW; ++k) tyy[k] = flux_n(coef_y(g, ecC[k]), vyN[k], vyC[k]);
        if (DX && j < ny) {
            T txx[VW];
            const T vxe = shfl_dn1(vxC[0]);
#pragma unroll
            for (int k = 0; k < VW; ++k) txx[k] = flux_n(coef_x(g, ecC[k]), k + 1 < VW ? vxC[k + 1] : vxe, vxC[k]);
            const T txw = shfl_up1(txx[VW - 1]);
            const T ecw = shfl_up1(ecC[VW - 1]);
            T out[VW];
#pragma unroll
            for (int k = 0; k < VW; ++k) {
                const int col = c0 + k;
                const T m = m_x(txx[k], k ? txx[k - 1] : txw, sxN[k], sxC[k]);
                const T inv = INV ? iv[0][k] : inv_diag(diag_x(g, ecC[k], k ? ecC[k - 1] : ecw, enN[k], enC[k]));
                const T nv = jacobi_update(vxC[k], b[0][k], m, jacobi_weight(omega, inv));
                out[k] = (col >= 1 && col <= nx - 1) ? nv : vxC[k];
            }
            if (own) st_row(ox, g, j, c0, cx, out);
        }
        if (DY) {
            const T sye = shfl_dn1(syC[0]);
            const T ene = shfl_dn1(enC[0]);
            T out[VW];
#pragma unroll
            for (int k = 0; k < VW; ++k) {
                const T m = m_y(k + 1 < VW ? syC[k + 1] : sye, syC[k], tyy[k], tyyS[k]);
                const T inv =
                    INV ? iv[1][k] : inv_diag(diag_y(g, ecC[k], ecS[k], k + 1 < VW ? enC[k + 1] : ene, enC[k]));
                const T nv = jacobi_update(vyC[k], b[1][k], m, jacobi_weight(omega, inv));
                out[k] = (j >= 1 && j <= ny - 1) ? nv : vyC[k];
            }
            if (own) st_row(oy, g, j, c0, cy, out);
        }
#pragma unroll
        for (int k = 0; k < VW; ++k) {
            vxC[k] = vxN[k];
            vyC[k] = vyN[k];
            enC[k] = enN[k];
            ecS[k] = ecC[k];
            tyyS[k] = tyy[k];
            sxC[k] = sxN[k];
            syC[k] = syN[k];
        }
    }
    cp_async_wait<0>(); // no copy outlives the warp
}

// shared bytes of one warp's stage
template <typename T, bool DX, bool DY, bool INV>
constexpr size_t jr_stage_bytes() { return (size_t)JR_PD * JrFields<DX, DY, INV>::N * 32 * 16; }

template <typename T, int VW, bool DX, bool DY, bool INV, int SQM>
__global__ void __launch_bounds__(JR_WARPS * 32) k_jacobi_rows(GridDesc<T> g, Coeffs<T> c, T omega,
                                                               const T *__restrict__ vx, const T *__restrict__ vy,
                                                               T *__restrict__ ox, T *__restrict__ oy, int rows)
{
    extern __shared__ __align__(16) unsigned char jr_smem[];
    const int w = (int)threadIdx.x >> 5;
    const int strip = (int)blockIdx.x * JR_WARPS + w;
    T *stage = reinterpret_cast<T *>(jr_smem + (size_t)w * jr_stage_bytes<T, DX, DY, INV>());
    jacobi_rows<T, VW, DX, DY, INV, SQM>(g, c, omega, vx, vy, ox, oy, rows, strip, stage);
}

// values per lane: one 16-byte vector
template <typename T>
constexpr int jr_vw() { return 16 / (int)sizeof(T); }

// rows per warp: enough warps to fill the GPU a few times over, at most 16
// (the band's first row is read twice)
inline int jacobi_rows_per_warp(int nx, int ny, int vw)
{
    const long long strips = (nx + 30 * vw) / (30 * vw);
    const long long want = 152LL * 48; // warps
    const long long r = (long long)(ny + 1) * strips / want;
    return (int)std::max(4LL, std::min(16LL, r));
}

template <typename T, bool DX, bool DY>
cudaError_t jacobi_pass(const GridDesc<T> &g, const Coeffs<T> &c, T omega, const T *vx, const T *vy, T *ox, T *oy,
                        cudaStream_t s)
{
    constexpr int VW = jr_vw<T>();
    constexpr int OWN = 30 * VW;
    const int strips = (g.nx + OWN) / OWN; // columns 0 .. nx
    const int rows = jacobi_rows_per_warp(g.nx, g.ny, VW);
    const dim3 grid((unsigned)((strips + JR_WARPS - 1) / JR_WARPS), (unsigned)((g.ny + rows) / rows));
    // FP32 forms 1/diag on the fly; FP64 reads it when the arrays exist
    const bool inv = sizeof(T) == 8 && c.inv_dx && c.inv_dy;
    // the shear form is fixed per launch (square cells or not)
    const size_t smem_t = JR_WARPS * jr_stage_bytes<T, DX, DY, true>();
    const size_t smem_f = JR_WARPS * jr_stage_bytes<T, DX, DY, false>();
    if (inv && g.square)
        k_jacobi_rows<T, VW, DX, DY, true, 1><<<grid, JR_WARPS * 32, smem_t, s>>>(g, c, omega, vx, vy, ox, oy, rows);
    else if (inv)
        k_jacobi_rows<T, VW, DX, DY, true, 0><<<grid, JR_WARPS * 32, smem_t, s>>>(g, c, omega, vx, vy, ox, oy, rows);
    else if (g.square)
        k_jacobi_rows<T, VW, DX, DY, false, 1><<<grid, JR_WARPS * 32, smem_f, s>>>(g, c, omega, vx, vy, ox, oy, rows);
    else
        k_jacobi_rows<T, VW, DX, DY, false, 0><<<grid, JR_WARPS * 32, smem_f, s>>>(g, c, omega, vx, vy, ox, oy, rows);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// red-black Gauss-Seidel, one sweep per launch
// ---------------------------------------------------------------------------
constexpr int GS_TX = 32, GS_TY = 32, GS_H = 4; // tile and window halo
constexpr int GS_WX = GS_TX + 2 * GS_H, GS_WY = GS_TY + 2 * GS_H;
constexpr int GS_THREADS = 256;

template <typename T>
struct GsWin {
    T vx[GS_WY][GS_WX], vy[GS_WY][GS_WX], ec[GS_WY][GS_WX], en[GS_WY][GS_WX], bx[GS_WY][GS_WX], by[GS_WY][GS_WX];
};
template <typename T, bool INV>
struct GsInv {
    T ix[GS_WY][GS_WX], iy[GS_WY][GS_WX];
};
template <typename T>
struct GsInv<T, false> {};

template <typename T, bool INV>
struct GsSmem : GsWin<T>, GsInv<T, INV> {};
static_assert(GS_TX % 32 == 0 && GS_H == 4 && (GS_WX * 4) % 16 == 0, "RBGS window rows must start 16-byte aligned");

// One colour of one component on the window cells at least `ring` cells
// inside the window's edge.  X: vx, else vy.  Updates in place in shared
// memory: a point of one colour reads only points of the other colour of its
// own component (and the other component, which this half-sweep does not
// change).
template <typename T, bool INV, bool X, int SQM>
__device__ __forceinline__ void gs_half(const GridDesc<T> &g, GsSmem<T, INV> &w, T omega, int ox0, int oy0, int colour,
                                        int ring, int tid)
{
    const int h = GS_WY - 2 * ring, wdt = GS_WX - 2 * ring;
    const int per_row = (wdt + 1) / 2;
    for (int e = tid; e < h * per_row; e += GS_THREADS) {
        const int a = ring + e / per_row;
        const int J = oy0 + a;
        // first window column of this colour in row a: global (I + J) even = red
        const int b0 = ring + (((ox0 + ring + J + colour) & 1) ? 1 : 0);
        const int b = b0 + 2 * (e % per_row);
        if (b >= GS_WX - ring) continue;
        const int I = ox0 + b;
        if (X) {
            if (J < 0 || J >= g.ny || I < 1 || I > g.nx - 1) continue;
            const T vc = w.vx[a][b];
            const T ecC = w.ec[a][b], ecW = w.ec[a][b - 1], enN = w.en[a + 1][b], enS = w.en[a][b];
            const T txx_c = flux_n(coef_x(g, ecC), w.vx[a][b + 1], vc);
            const T txx_w = flux_n(coef_x(g, ecW), vc, w.vx[a][b - 1]);
            const T sx_n = shear_x<SQM>(g, enN, w.vx[a + 1][b], vc, w.vy[a + 1][b], w.vy[a + 1][b - 1]);
            const T sx_c = shear_x<SQM>(g, enS, vc, w.vx[a - 1][b], w.vy[a][b], w.vy[a][b - 1]);
            const T m = m_x(txx_c, txx_w, sx_n, sx_c);
            T inv;
            if constexpr (INV) inv = w.ix[a][b];
            else inv = inv_diag(diag_x(g, ecC, ecW, enN, enS));
            w.vx[a][b] = jacobi_update(vc, w.bx[a][b], m, jacobi_weight(omega, inv));
        } else {
            if (I < 0 || I >= g.nx || J < 1 || J > g.ny - 1) continue;
            const T vc = w.vy[a][b];
            const T ecC = w.ec[a][b], ecS = w.ec[a - 1][b], enE = w.en[a][b + 1], enW = w.en[a][b];
            const T tyy_c = flux_n(coef_y(g, ecC), w.vy[a + 1][b], vc);
            const T tyy_s = flux_n(coef_y(g, ecS), vc, w.vy[a - 1][b]);
            const T sy_e = shear_y<SQM>(g, enE, w.vx[a][b + 1], w.vx[a - 1][b + 1], w.vy[a][b + 1], vc);
            const T sy_c = shear_y<SQM>(g, enW, w.vx[a][b], w.vx[a - 1][b], vc, w.vy[a][b - 1]);
            const T m = m_y(sy_e, sy_c, tyy_c, tyy_s);
            T inv;
            if constexpr (INV) inv = w.iy[a][b];
            else inv = inv_diag(diag_y(g, ecC, ecS, enE, enW));
            w.vy[a][b] = jacobi_update(vc, w.by[a][b], m, jacobi_weight(omega, inv));
        }
    }
    __syncthreads();
}

// One RBGS sweep of tile (blockIdx.x, blockIdx.y) from (vx, vy) into (ox, oy).
template <typename T, bool INV, int SQM>
__global__ void __launch_bounds__(GS_THREADS) k_rbgs_tile(GridDesc<T> g, Coeffs<T> c, T omega,
                                                          const T *__restrict__ vx, const T *__restrict__ vy,
                                                          T *__restrict__ ox, T *__restrict__ oy)
{
    extern __shared__ __align__(16) unsigned char gs_raw[];
    GsSmem<T, INV> &w = *reinterpret_cast<GsSmem<T, INV> *>(gs_raw);
    const int tid = (int)threadIdx.x;
    const int x0 = (int)blockIdx.x * GS_TX, y0 = (int)blockIdx.y * GS_TY;
    const int ox0 = x0 - GS_H, oy0 = y0 - GS_H;
    const size_t P = (size_t)g.pitch;
    // stage the window by 16-byte asynchronous copies (the window's first
    // column is 4 cells left of a multiple of 32, so every vector is aligned);
    // vectors that cross a field's extent are filled value by value, with zero
    // outside it
    constexpr int VW = 16 / (int)sizeof(T);
    constexpr int NV = GS_WX / VW;
    auto stage = [&](T(*dst)[GS_WX], const T *__restrict__ src, int a, int v, int nrows, int ncols) {
        const int J = oy0 + a, I0 = ox0 + v * VW;
        if (J >= 0 && J < nrows && I0 >= 0 && I0 + VW <= ncols) {
            cp_async16(&dst[a][v * VW], src + (size_t)J * P + (size_t)I0);
        } else {
#pragma unroll
            for (int k = 0; k < VW; ++k) {
                const int I = I0 + k;
                dst[a][v * VW + k] = (J >= 0 && J < nrows && I >= 0 && I < ncols) ? src[(size_t)J * P + I] : T(0);
            }
        }
    };
    for (int e = tid; e < GS_WY * NV; e += GS_THREADS) {
        const int a = e / NV, v = e % NV;
        stage(w.vx, vx, a, v, g.ny, g.nx + 1);
        stage(w.vy, vy, a, v, g.ny + 1, g.nx);
        stage(w.ec, c.eta_c, a, v, g.ny, g.nx);
        stage(w.en, c.eta_n, a, v, g.ny + 1, g.nx + 1);
        stage(w.bx, c.bx, a, v, g.ny, g.nx + 1);
        stage(w.by, c.by, a, v, g.ny + 1, g.nx);
        if constexpr (INV) {
            stage(w.ix, c.inv_dx, a, v, g.ny, g.nx + 1);
            stage(w.iy, c.inv_dy, a, v, g.ny + 1, g.nx);
        }
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    gs_half<T, INV, true, SQM>(g, w, omega, ox0, oy0, 0, 1, tid);  // vx red on the tile + 3
    gs_half<T, INV, true, SQM>(g, w, omega, ox0, oy0, 1, 2, tid);  // vx black on the tile + 2
    gs_half<T, INV, false, SQM>(g, w, omega, ox0, oy0, 0, 3, tid); // vy red on the tile + 1
    gs_half<T, INV, false, SQM>(g, w, omega, ox0, oy0, 1, 4, tid); // vy black on the tile
    // the unknowns of the tile's own cells
    for (int e = tid; e < GS_TY * GS_TX; e += GS_THREADS) {
        const int a = GS_H + e / GS_TX, b = GS_H + e % GS_TX;
        const int J = oy0 + a, I = ox0 + b;
        const size_t q = (size_t)J * P + (size_t)I;
        if (J < g.ny && I >= 1 && I <= g.nx - 1) ox[q] = w.vx[a][b];
        if (I < g.nx && J >= 1 && J <= g.ny - 1) oy[q] = w.vy[a][b];
    }
}

// ---------------------------------------------------------------------------
// FP32 energy sums (Sec. 6.4) by row-marching warps
// ---------------------------------------------------------------------------
// The warp layout and row staging of jacobi_rows; per position the terms of
// the other FP32 energy kernels: r = b - M v (b = f - G p formed on the fly),
// r^2 / (-diag M) and f^2 / (-diag M) of the vx and the vy unknown (a cell's
// two terms added in FP32), (D v)^2 eta_c / (2/hx^2 + 2/hy^2) of the cell;
// 1/diag from the viscosity, as k_inv_diag forms it.  Per lane the terms go
// into compensated FP32 sums over a band of rows, flushed into FP64 sums.
struct CompSum {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float t)
    {
        const float s = __fadd_rn(hi, t);
        const float bb = __fsub_rn(s, hi);
        const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(t, bb));
        hi = s;
        lo = __fadd_rn(lo, e);
    }
    __device__ __forceinline__ void flush(double &S)
    {
        S += (double)hi + (double)lo;
        hi = lo = 0.f;
    }
};

// row fields of iteration j: vx, vy, eta_n of row j + 1; eta_c, fx, fy, (with
// INV) 1/diag at vx and vy, (with HASP) p of row j
template <bool INV, bool HASP>
struct ErFields {
    static constexpr int IX = 6, IY = 7, P = INV ? 8 : 6;
    static constexpr int N = P + (HASP ? 1 : 0);
};

template <int SQM, bool INV, bool HASP>
__device__ __forceinline__ void energy_band(const GridDesc<float> &g, const float *__restrict__ ec,
                                            const float *__restrict__ en, const float *__restrict__ fx,
                                            const float *__restrict__ fy, const float *__restrict__ ix,
                                            const float *__restrict__ iy, const float *__restrict__ p,
                                            const float *__restrict__ vx, const float *__restrict__ vy, int j0,
                                            int j1, int strip, float *stage, double &s_rv, double &s_rp,
                                            double &s_ff)
{
    using EF = ErFields<INV, HASP>;
    constexpr int VW = 4, OWN = 30 * VW, N = EF::N;
    using V = float4;
    const int lane = (int)threadIdx.x & 31;
    const int w0 = strip * OWN;
    if (w0 > g.nx) return;
    const int c0 = w0 - VW + lane * VW;
    const bool own = lane >= 1 && lane <= 30;
    const int nx = g.nx, ny = g.ny;
    const int cx = nx + 1, cy = nx;
    const bool col_ok = c0 >= 0 && c0 < g.pitch;
    const float ilap = (float)(1.0 / g.lap);
    V *const st = reinterpret_cast<V *>(stage);
    auto src = [&](int f, int j, int &row, int &nrows) -> const float * {
        switch (f) {
        case 0: row = j + 1; nrows = ny; return vx;
        case 1: row = j + 1; nrows = ny + 1; return vy;
        case 2: row = j + 1; nrows = ny + 1; return en;
        case 3: row = j; nrows = ny; return ec;
        case 4: row = j; nrows = ny; return fx;
        case 5: row = j; nrows = ny + 1; return fy;
        default: break;
        }
        row = j;
        if (INV && f == EF::IX) { nrows = ny; return ix; }
        if (INV && f == EF::IY) { nrows = ny + 1; return iy; }
        nrows = ny;
        return p;
    };
    auto issue = [&](int j) {
        if (j < j1 && col_ok) {
            V *const slot = st + (j % JR_PD) * N * 32 + lane;
#pragma unroll
            for (int f = 0; f < N; ++f) {
                int row, nrows;
                const float *q = src(f, j, row, nrows);
                if (row >= 0 && row < nrows) cp_async16(slot + f * 32, q + (size_t)row * g.pitch + c0);
            }
        }
        cp_async_commit();
    };
    auto take = [&](int f, int j, int cols, float(&a)[VW]) {
        int row, nrows;
        (void)src(f, j, row, nrows);
        if (col_ok && row >= 0 && row < nrows) {
            const V v = st[(j % JR_PD) * N * 32 + f * 32 + lane];
            const float *e = reinterpret_cast<const float *>(&v);
#pragma unroll
            for (int k = 0; k < VW; ++k) a[k] = (c0 + k < cols) ? e[k] : 0.f;
        } else {
#pragma unroll
            for (int k = 0; k < VW; ++k) a[k] = 0.f;
        }
    };
#pragma unroll
    for (int d = 0; d < JR_PD - 1; ++d) issue(j0 + d);

    float vxC[VW], vyC[VW], enC[VW], ecS[VW], tyyS[VW], sxC[VW], syC[VW], pS[VW];
    {
        float vxS[VW], vyS[VW];
        ld_row(vx, g, j0, c0, ny, cx, vxC);
        ld_row(vy, g, j0, c0, ny + 1, cy, vyC);
        ld_row(en, g, j0, c0, ny + 1, cx, enC);
        ld_row(ec, g, j0 - 1, c0, ny, cy, ecS);
        ld_row(vx, g, j0 - 1, c0, ny, cx, vxS);
        ld_row(vy, g, j0 - 1, c0, ny + 1, cy, vyS);
        if (HASP) ld_row(p, g, j0 - 1, c0, ny, cy, pS);
        const float vyw = shfl_up1(vyC[VW - 1]);
#pragma unroll
        for (int k = 0; k < VW; ++k) {
            tyyS[k] = flux_n(coef_y(g, ecS[k]), vyC[k], vyS[k]);
            shear_xy<SQM>(g, enC[k], vxC[k], vxS[k], vyC[k], k ? vyC[k - 1] : vyw, sxC[k], syC[k]);
        }
    }
    CompSum rv, rp, ff;
    for (int j = j0; j < j1; ++j) {
        issue(j + JR_PD - 1);
        cp_async_wait<JR_PD - 1>();
        float vxN[VW], vyN[VW], enN[VW], ecC[VW], fxC[VW], fyC[VW], pC[VW], ivx[VW], ivy[VW];
        take(0, j, cx, vxN);
        take(1, j, cy, vyN);
        take(2, j, cx, enN);
        take(3, j, cy, ecC);
        take(4, j, cx, fxC);
        take(5, j, cy, fyC);
        if (INV) {
            take(EF::IX, j, cx, ivx);
            take(EF::IY, j, cy, ivy);
        }
        if (HASP) take(EF::P, j, cy, pC);
        float sxN[VW], syN[VW];
        {
            const float vyw = shfl_up1(vyN[VW - 1]);
#pragma unroll
            for (int k = 0; k < VW; ++k)
                shear_xy<SQM>(g, enN[k], vxN[k], vxC[k], vyN[k], k ? vyN[k - 1] : vyw, sxN[k], syN[k]);
        }
        float tyy[VW], txx[VW];
        const float vxe = shfl_dn1(vxC[0]);
#pragma unroll
        for (int k = 0; k < VW; ++k) {
            tyy[k] = flux_n(coef_y(g, ecC[k]), vyN[k], vyC[k]);
            txx[k] = flux_n(coef_x(g, ecC[k]), k + 1 < VW ? vxC[k + 1] : vxe, vxC[k]);
        }
        const float txw = shfl_up1(txx[VW - 1]), ecw = shfl_up1(ecC[VW - 1]);
        const float sye = shfl_dn1(syC[0]), ene = shfl_dn1(enC[0]);
        const float pw = HASP ? shfl_up1(pC[VW - 1]) : 0.f;
#pragma unroll
        for (int k = 0; k < VW; ++k) {
            const int col = c0 + k;
            float tv = 0.f, tf = 0.f;
            bool any = false;
            if (j < ny && col >= 1 && col <= nx - 1) { // vx unknown
                const float m = m_x(txx[k], k ? txx[k - 1] : txw, sxN[k], sxC[k]);
                const float wi = -(INV ? ivx[k] : inv_diag(diag_x(g, ecC[k], k ? ecC[k - 1] : ecw, enN[k], enC[k])));
                const float b = HASP ? r_fma(r_sub(pC[k], k ? pC[k - 1] : pw), g.ihx, fxC[k]) : fxC[k];
                const float r = r_sub(b, m);
                tv = r_mul(r_mul(r, r), wi);
                tf = r_mul(r_mul(fxC[k], fxC[k]), wi);
                any = true;
            }
            if (col < nx && j >= 1 && j <= ny - 1) { // vy unknown
                const float m = m_y(k + 1 < VW ? syC[k + 1] : sye, syC[k], tyy[k], tyyS[k]);
                const float wi =
                    -(INV ? ivy[k] : inv_diag(diag_y(g, ecC[k], ecS[k], k + 1 < VW ? enC[k + 1] : ene, enC[k])));
                const float b = HASP ? r_fma(r_sub(pC[k], pS[k]), g.ihy, fyC[k]) : fyC[k];
                const float r = r_sub(b, m);
                const float a = r_mul(r_mul(r, r), wi), cf = r_mul(r_mul(fyC[k], fyC[k]), wi);
                tv = any ? r_add(tv, a) : a;
                tf = any ? r_add(tf, cf) : cf;
                any = true;
            }
            if (own && any) {
                rv.add(tv);
                ff.add(tf);
            }
            if (own && j < ny && col < nx) { // the cell's divergence
                const float dv = r_fma(r_sub(k + 1 < VW ? vxC[k + 1] : vxe, vxC[k]), g.ihx,
                                       r_mul(r_sub(vyN[k], vyC[k]), g.ihy));
                rp.add(r_mul(r_mul(dv, dv), r_mul(ecC[k], ilap)));
            }
        }
#pragma unroll
        for (int k = 0; k < VW; ++k) {
            vxC[k] = vxN[k];
            vyC[k] = vyN[k];
            enC[k] = enN[k];
            ecS[k] = ecC[k];
            tyyS[k] = tyy[k];
            sxC[k] = sxN[k];
            syC[k] = syN[k];
            if (HASP) pS[k] = pC[k];
        }
    }
    cp_async_wait<0>(); // no copy outlives the band
    rv.flush(s_rv);
    rp.flush(s_rp);
    ff.flush(s_ff);
}

// Work items (a group of JR_WARPS column strips, a band of rows) in a fixed
// order per block (at most energy_partials() blocks, one partial triple
// each), so the sums are repeatable bit for bit.
template <int SQM, bool INV, bool HASP>
__global__ void __launch_bounds__(JR_WARPS * 32) k_energy_rows(GridDesc<float> g, const float *__restrict__ ec,
                                                               const float *__restrict__ en,
                                                               const float *__restrict__ fx,
                                                               const float *__restrict__ fy,
                                                               const float *__restrict__ ix,
                                                               const float *__restrict__ iy,
                                                               const float *__restrict__ p,
                                                               const float *__restrict__ vx,
                                                               const float *__restrict__ vy, int rows, int ngx,
                                                               int nitems, double *__restrict__ partials)
{
    extern __shared__ __align__(16) unsigned char er_smem[];
    const int w = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
    float *stage = reinterpret_cast<float *>(er_smem + (size_t)w * JR_PD * ErFields<INV, HASP>::N * 32 * 16);
    double s_rv = 0.0, s_rp = 0.0, s_ff = 0.0;
    for (int it = (int)blockIdx.x; it < nitems; it += (int)gridDim.x) {
        const int gx = it % ngx, band = it / ngx;
        const int j0 = band * rows, j1 = min(j0 + rows, g.ny + 1);
        energy_band<SQM, INV, HASP>(g, ec, en, fx, fy, ix, iy, p, vx, vy, j0, j1, gx * JR_WARPS + w, stage, s_rv, s_rp,
                                    s_ff);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s_rv += __shfl_down_sync(0xffffffffu, s_rv, o);
        s_rp += __shfl_down_sync(0xffffffffu, s_rp, o);
        s_ff += __shfl_down_sync(0xffffffffu, s_ff, o);
    }
    __shared__ double sh[3][JR_WARPS];
    if (lane == 0) {
        sh[0][w] = s_rv;
        sh[1][w] = s_rp;
        sh[2][w] = s_ff;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int q = 0; q < JR_WARPS; ++q) t += sh[threadIdx.x][q];
        partials[(size_t)blockIdx.x * 3 + threadIdx.x] = t;
    }
}

} // namespace

cudaError_t launch_energy_rows(const GridDesc<float> &g, const float *eta_c, const float *eta_n, const float *fx,
                               const float *fy, const float *inv_dx, const float *inv_dy, const float *p,
                               const float *vx, const float *vy, double *partials, int *nblocks, cudaStream_t s)
{
    constexpr int OWN = 30 * 4;
    const int strips = (g.nx + OWN) / OWN;
    const int ngx = (strips + JR_WARPS - 1) / JR_WARPS;
    const int rows = jacobi_rows_per_warp(g.nx, g.ny, 4);
    const int nband = (g.ny + rows) / rows;
    const int nitems = ngx * nband;
    const int grid = std::min(nitems, energy_partials()); // the partial triples the caller holds
    const size_t smem = (size_t)JR_WARPS * JR_PD * ErFields<true, true>::N * 32 * 16;
    const int sel = (g.square ? 4 : 0) | (inv_dx && inv_dy ? 2 : 0) | (p ? 1 : 0);
    cudaError_t e = cudaSuccess;
    auto go = [&](auto kern) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            kern<<<grid, JR_WARPS * 32, smem, s>>>(g, eta_c, eta_n, fx, fy, inv_dx, inv_dy, p, vx, vy, rows, ngx,
                                                   nitems, partials);
    };
    switch (sel) {
    case 0: go(k_energy_rows<0, false, false>); break;
    case 1: go(k_energy_rows<0, false, true>); break;
    case 2: go(k_energy_rows<0, true, false>); break;
    case 3: go(k_energy_rows<0, true, true>); break;
    case 4: go(k_energy_rows<1, false, false>); break;
    case 5: go(k_energy_rows<1, false, true>); break;
    case 6: go(k_energy_rows<1, true, false>); break;
    default: go(k_energy_rows<1, true, true>); break;
    }
    if (e != cudaSuccess) return e;
    *nblocks = grid;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_jacobi(const GridDesc<T> &g, const Coeffs<T> &c, T omega, const T *vx, const T *vy, T *ox, T *oy,
                          int fused, cudaStream_t s)
{
    if (fused) return jacobi_pass<T, true, true>(g, c, omega, vx, vy, ox, oy, s);
    cudaError_t e = jacobi_pass<T, true, false>(g, c, omega, vx, vy, ox, oy, s);
    if (e == cudaSuccess) e = jacobi_pass<T, false, true>(g, c, omega, vx, vy, ox, oy, s);
    return e;
}

template <typename T>
cudaError_t launch_rbgs_sweep(const GridDesc<T> &g, const Coeffs<T> &c, T omega, const T *vx, const T *vy, T *ox,
                              T *oy, cudaStream_t s)
{
    const dim3 grid((unsigned)((g.nx + GS_TX - 1) / GS_TX), (unsigned)((g.ny + GS_TY - 1) / GS_TY));
    // FP64 reads 1/diag (FP64 reciprocals are slow); FP32 forms it
    auto run = [&](auto kern, size_t smem) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) kern<<<grid, GS_THREADS, smem, s>>>(g, c, omega, vx, vy, ox, oy);
        return e;
    };
    cudaError_t e;
    if (sizeof(T) == 8 && c.inv_dx && c.inv_dy)
        e = g.square ? run(k_rbgs_tile<T, true, 1>, sizeof(GsSmem<T, true>))
                     : run(k_rbgs_tile<T, true, 0>, sizeof(GsSmem<T, true>));
    else
        e = g.square ? run(k_rbgs_tile<T, false, 1>, sizeof(GsSmem<T, false>))
                     : run(k_rbgs_tile<T, false, 0>, sizeof(GsSmem<T, false>));
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

#define STOKES_SWEEP_INST(T)                                                                                       \
    template cudaError_t launch_jacobi<T>(const GridDesc<T> &, const Coeffs<T> &, T, const T *, const T *, T *,    \
                                          T *, int, cudaStream_t);                                                 \
    template cudaError_t launch_rbgs_sweep<T>(const GridDesc<T> &, const Coeffs<T> &, T, const T *, const T *,     \
                                              T *, T *, cudaStream_t);
STOKES_SWEEP_INST(float)
STOKES_SWEEP_INST(double)
#undef STOKES_SWEEP_INST

} // namespace stokes
