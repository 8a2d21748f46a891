// ras_kernels.cu -- RAS-type temporally blocked Jacobi (Sec. 4.3 and
// Algorithm 2 of arXiv 2509.19061) and, as its one-sweep case, the spatially
// blocked fused Jacobi smoother (Sec. 4.2, Sec. 5 (iv)).
//
// A CTA works on one tile of the shifted tiling at a time: the tile grown by
// h = overlap + 1 cells (the overlap plus the Dirichlet ring, the "window").
// It runs the local Jacobi sweeps on chip and writes back only the unknowns of
// the tile's own cells.  All tiles read the snapshot (vx, vy) and write
// (ox, oy), so the result does not depend on the order in which tiles run
// and every unknown has one writer (the in-place benign race of the CPU
// original is gone).
//
// Sweep s of ks only updates the cells within min(overlap, ks - s) of the
// tile: the owned unknowns after ks sweeps depend on sweep s only through
// that region (the stencil reaches one cell per sweep), so skipping the rest
// leaves the result unchanged.
//
// Kernels, all with the arithmetic of stencil.cuh and so identical results:
//  k_ras_tma  persistent: each CTA loops over tiles; the window of the next
//             tile is staged into shared memory by 2D bulk tensor copies (TMA,
//             cp.async.bulk.tensor) while the current tile is swept.  Thread
//             (column, strip) owns R cells of one window column; their
//             coefficients (2 eta_c/h^2, eta_n, omega/diag, b) and velocities
//             stay in registers for all sweeps.  Per sweep, phase A computes
//             each cell's fluxes (Txx, Tyy and the shear at its node), phase B
//             forms M v from own and neighbour fluxes and updates; shared
//             memory holds only velocities and fluxes.
//  k_ras_reg  the same compute with the window read straight from global
//             memory (used when the staging buffers do not fit).
//  k_ras      general kernel for windows too large for the register layout:
//             every field of the window lives in shared memory.
#include <algorithm>
#include <type_traits>
#include <cstring>

#include "internal.h"
#include "stencil.cuh"
#include "tma.h"

namespace stokes {

namespace {

constexpr int RAS_THREADS = 256;
constexpr int RAS_PLANES = 8;  // vx, vy ping-pong (4), eta_c, eta_n, bx, by
constexpr int REG_MAX_THREADS = 512;
constexpr int SMALL_THREADS = 320;
constexpr int REG_PLANES = 6;  // vx, vy, Txx, Sy, Tyy (strip ends), Sx (strip ends)

// Per-precision shape of the register-resident kernels.
//  R     cells per thread (strip height)
//  TRAP  sweep s updates only the region that still matters (per-cell tests);
//        otherwise every cell of the window is swept (no tests, ring and
//        non-unknown cells have weight 0), which costs more arithmetic but
//        far fewer instructions: FP32 is issue-bound, FP64 is FP64-pipe-bound
//  INVD  1/diag(M) is staged from the library's precomputed arrays instead
//        of being computed per tile (two more fields to read, but the
//        per-tile reciprocals cost more issue slots than the bytes cost)
template <typename T>
struct KCfg;
template <>
struct KCfg<float> {
    static constexpr int R = 5;
    static constexpr bool TRAP = false;
    static constexpr bool INVD = true;
};
template <>
struct KCfg<double> {
    static constexpr int R = 4;
    static constexpr bool TRAP = true;
    static constexpr bool INVD = true;
};

// Tile b of the tiling of [0, n) cut at s + m T.
__host__ __device__ __forceinline__ void tile_interval(int n, int T, int s, int b, int &lo, int &hi)
{
    const int first = s > 0 ? s : T;
    lo = b == 0 ? 0 : first + (b - 1) * T;
    hi = first + b * T;
    if (hi > n) hi = n;
}

template <typename T>
struct RasArgs {
    GridDesc<T> g;
    Coeffs<T> c;
    T omega;
    const T *vx, *vy;
    T *ox, *oy;
    TileGrid tg;
    int ks, overlap;
    int wxm, wym; // largest window extent (cells)
    int strips;   // strips per column (register kernels)
    int wp;       // shared-memory row pitch of the compute planes (elements)
    int spad;     // extra elements between consecutive strips of a plane
    int plane;    // compute-plane size (elements)
    int bw;       // staging box width (elements); box height is wym
    int stage;    // staging-plane size (elements, 128-byte multiple)
    int *status;  // device status word (timeout)
    long long wait_limit; // cycles a TMA wait may take before giving up
};

constexpr int MAX_STAGE_FIELDS = 8;
struct TmaMaps {
    CUtensorMap m[MAX_STAGE_FIELDS]; // vx, vy, eta_c, eta_n, bx, by[, 1/dx, 1/dy]
};

// geometry of one tile's window
struct Window {
    int x0, x1, y0, y1; // owned cells
    int ox0, oy0;       // window origin (global cell index)
    int WX, WY;         // window extent
};

template <typename T>
__device__ __forceinline__ Window window_of(const RasArgs<T> &a, int tile)
{
    Window w;
    tile_interval(a.g.nx, a.tg.ti, a.tg.si, tile % a.tg.ntx, w.x0, w.x1);
    tile_interval(a.g.ny, a.tg.tj, a.tg.sj, tile / a.tg.ntx, w.y0, w.y1);
    const int h = a.overlap + 1;
    w.ox0 = w.x0 - h;
    w.oy0 = w.y0 - h;
    w.WX = w.x1 - w.x0 + 2 * h;
    w.WY = w.y1 - w.y0 + 2 * h;
    return w;
}

// per-thread state of the register-resident layout
template <typename T, int R>
struct CellRegs {
    T vx[R], vy[R], ax[R], ay[R], en[R], bx[R], by[R], wx[R], wy[R];
    unsigned ux, uy; // bit r: cell r is a vx / vy unknown inside the ring
};

// Compute planes: Vx, Vy, Fxx, Fsy, Fyy, Fsx, each (rows + 2) x WP with a
// one-cell border; index (wy, wx), -1 <= wy <= rows, -1 <= wx <= wp - 2.
// Element (wy, wx) sits at wy * WP + floor(wy / R) * SPAD + wx: the pad after
// every strip of R rows makes the stride from one strip to the next congruent
// to the window width modulo 32 banks, so a warp whose threads straddle two
// strips (thread = strip * width + column) reads 32 consecutive banks.
template <typename T>
struct Planes {
    T *Vx, *Vy, *Fxx, *Fsy, *Fyy, *Fsx;
    __device__ Planes(T *raw, int WP, int SPAD, int PL)
    {
        T *b = raw + WP + SPAD + 1;
        Vx = b;
        Vy = b + PL;
        Fxx = b + 2 * PL;
        Fsy = b + 3 * PL;
        Fyy = b + 4 * PL;
        Fsx = b + 5 * PL;
    }
};

// Plane geometry of a register-kernel launch.  For the window widths and
// strip counts the launcher specialises (WXM > 0) every plane offset is a
// compile-time constant, which lets shared-memory accesses use immediate
// offsets; otherwise the values come from the launch arguments.  Both follow
// the formulas of plan_ras.
template <typename T, int WXM, int NS>
struct Geo {
    static constexpr int R = KCfg<T>::R;
    static constexpr bool FIXED = WXM > 0;
    static constexpr int WPC = WXM + 2;
    static constexpr int SPC = (((WXM - R * WPC) % 32) + 32) % 32;
    static constexpr int PLC = WPC * (NS * R + 2) + (NS + 1) * SPC;
    int wxm, wp, spad, plane, strips;
    __device__ __forceinline__ explicit Geo(const RasArgs<T> &a)
        : wxm(FIXED ? WXM : a.wxm), wp(FIXED ? WPC : a.wp), spad(FIXED ? SPC : a.spad),
          plane(FIXED ? PLC : a.plane), strips(FIXED ? NS : a.strips)
    {
    }
};

// Zero the one-cell border of every compute plane (it is never written
// afterwards): the fluxes of window-edge cells then read finite values.
template <typename T, int WXM, int NS>
__device__ __forceinline__ void zero_borders(const Geo<T, WXM, NS> &G, const Planes<T> &pl)
{
    constexpr int R = KCfg<T>::R;
    const int rows = G.strips * R, WP = G.wp, cols = G.wxm;
    const int n = 2 * (cols + 2) + 2 * rows;
    T *const ps[REG_PLANES] = {pl.Vx, pl.Vy, pl.Fxx, pl.Fsy, pl.Fyy, pl.Fsx};
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        int wy, wx;
        if (t < cols + 2) {
            wy = -1;
            wx = t - 1;
        } else if (t < 2 * (cols + 2)) {
            wy = rows;
            wx = t - (cols + 2) - 1;
        } else {
            wy = (t - 2 * (cols + 2)) >> 1;
            wx = (t & 1) ? cols : -1;
        }
        const int q = wy * WP + (wy < 0 ? -1 : wy / R) * G.spad + wx;
#pragma unroll
        for (int f = 0; f < REG_PLANES; ++f) ps[f][q] = T(0);
    }
}

// Fill the own cells' registers and the velocity planes; `ld(field, wy, wx)`
// returns the window value of field 0..7 (vx, vy, eta_c, eta_n, bx, by,
// 1/dx, 1/dy), zero outside the field's extent.  Cells outside the window get
// zero state.
template <typename T, int R, int WXM, int NS, class LD>
__device__ __forceinline__ void setup_cells(const RasArgs<T> &a, const Geo<T, WXM, NS> &G, const Window &w,
                                            CellRegs<T, R> &c, int col, int strip, bool active, const Planes<T> &pl,
                                            LD &&ld)
{
    const GridDesc<T> &g = a.g;
    const int WP = G.wp;
    const int gx = w.ox0 + col;
    c.ux = 0;
    c.uy = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int wy = strip * R + r, gy = w.oy0 + wy;
        T vxv = T(0), vyv = T(0), ec = T(0), env = T(0), bxv = T(0), byv = T(0), wxv = T(0), wyv = T(0);
        if (active && col < w.WX && wy < w.WY) {
            vxv = ld(0, wy, col);
            vyv = ld(1, wy, col);
            ec = ld(2, wy, col);
            env = ld(3, wy, col);
            bxv = ld(4, wy, col);
            byv = ld(5, wy, col);
            const bool inner = col >= 1 && col < w.WX - 1 && wy >= 1 && wy < w.WY - 1;
            if (inner && gy >= 0 && gy < g.ny && gx >= 1 && gx <= g.nx - 1) {
                c.ux |= 1u << r;
                const T inv = KCfg<T>::INVD ? ld(6, wy, col)
                                            : inv_diag(diag_x(g, ec, ld(2, wy, col - 1), ld(3, wy + 1, col), env));
                wxv = jacobi_weight(a.omega, inv);
            }
            if (inner && gx >= 0 && gx < g.nx && gy >= 1 && gy <= g.ny - 1) {
                c.uy |= 1u << r;
                const T inv = KCfg<T>::INVD ? ld(7, wy, col)
                                            : inv_diag(diag_y(g, ec, ld(2, wy - 1, col), ld(3, wy, col + 1), env));
                wyv = jacobi_weight(a.omega, inv);
            }
        }
        if (active) {
            pl.Vx[wy * WP + strip * G.spad + col] = vxv;
            pl.Vy[wy * WP + strip * G.spad + col] = vyv;
        }
        c.vx[r] = vxv;
        c.vy[r] = vyv;
        c.ax[r] = coef_x(g, ec);
        c.ay[r] = coef_y(g, ec);
        c.en[r] = env;
        c.bx[r] = bxv;
        c.by[r] = byv;
        c.wx[r] = wxv;
        c.wy[r] = wyv;
    }
}

// phase A for one cell: its fluxes into registers and the planes
// (q: the cell's plane index; SW: the index step from the last row of a strip
// to the first row of the next)
template <typename T, int R>
__device__ __forceinline__ void cell_fluxes(const GridDesc<T> &g, const CellRegs<T, R> &c, const Planes<T> &pl,
                                            int r, int q, int SW, T *txx, T *tyy, T *sx, T *sy)
{
    const T vx_s = r > 0 ? c.vx[r - 1] : pl.Vx[q - SW];
    const T vy_n = r < R - 1 ? c.vy[r + 1] : pl.Vy[q + SW];
    txx[r] = flux_n(c.ax[r], pl.Vx[q + 1], c.vx[r]);
    tyy[r] = flux_n(c.ay[r], vy_n, c.vy[r]);
    shear_xy(g, c.en[r], c.vx[r], vx_s, c.vy[r], pl.Vy[q - 1], sx[r], sy[r]);
    pl.Fxx[q] = txx[r];
    pl.Fsy[q] = sy[r];
    if (r == R - 1) pl.Fyy[q] = tyy[r];
    if (r == 0) pl.Fsx[q] = sx[r];
}

// ks local sweeps on the window (registers + shared planes), then write back
// the unknowns of the tile's own cells.  Ends with a barrier.
template <typename T, int R, int WXM, int NS>
__device__ __forceinline__ void sweep_and_store(const RasArgs<T> &a, const Geo<T, WXM, NS> &G, const Window &w,
                                                CellRegs<T, R> &c, int col, int strip, bool active,
                                                const Planes<T> &pl)
{
    const GridDesc<T> &g = a.g;
    const int WP = G.wp, SW = G.wp + G.spad, q0 = strip * (R * WP + G.spad) + col;
    T txx[R], tyy[R], sx[R], sy[R];
    for (int s = 1; s <= a.ks; ++s) {
        if (!KCfg<T>::TRAP) {
            // every cell of the window; non-updatable cells have weight 0
            if (active) {
#pragma unroll
                for (int r = 0; r < R; ++r)
                    cell_fluxes<T, R>(g, c, pl, r, q0 + r * WP, SW, txx, tyy, sx, sy);
            }
            __syncthreads();
            if (active) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int q = q0 + r * WP;
                    const T sx_n = r < R - 1 ? sx[r + 1] : pl.Fsx[q + SW];
                    const T tyy_s = r > 0 ? tyy[r - 1] : pl.Fyy[q - SW];
                    c.vx[r] = jacobi_update(c.vx[r], c.bx[r], m_x(txx[r], pl.Fxx[q - 1], sx_n, sx[r]), c.wx[r]);
                    c.vy[r] = jacobi_update(c.vy[r], c.by[r], m_y(pl.Fsy[q + 1], sy[r], tyy[r], tyy_s), c.wy[r]);
                    pl.Vx[q] = c.vx[r];
                    pl.Vy[q] = c.vy[r];
                }
            }
            __syncthreads();
        } else {
            const int rr = min(a.overlap, a.ks - s);
            // updated region, window coordinates; fluxes are needed one cell further
            const int rx0 = max(w.x0 - rr, 0) - w.ox0, rx1 = min(w.x1 + rr, g.nx) - w.ox0;
            const int ry0 = max(w.y0 - rr, 0) - w.oy0, ry1 = min(w.y1 + rr, g.ny) - w.oy0;
            const bool cx_in = active && col >= rx0 && col < rx1;
            const bool cx_flux = active && col >= rx0 - 1 && col <= rx1;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int wy = strip * R + r;
                if (cx_flux && wy >= ry0 - 1 && wy <= ry1)
                    cell_fluxes<T, R>(g, c, pl, r, q0 + r * WP, SW, txx, tyy, sx, sy);
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int wy = strip * R + r;
                if (cx_in && wy >= ry0 && wy < ry1) {
                    const int q = q0 + r * WP;
                    if (c.ux & (1u << r)) {
                        const T sx_n = r < R - 1 ? sx[r + 1] : pl.Fsx[q + SW];
                        c.vx[r] = jacobi_update(c.vx[r], c.bx[r], m_x(txx[r], pl.Fxx[q - 1], sx_n, sx[r]), c.wx[r]);
                        pl.Vx[q] = c.vx[r];
                    }
                    if (c.uy & (1u << r)) {
                        const T tyy_s = r > 0 ? tyy[r - 1] : pl.Fyy[q - SW];
                        c.vy[r] = jacobi_update(c.vy[r], c.by[r], m_y(pl.Fsy[q + 1], sy[r], tyy[r], tyy_s), c.wy[r]);
                        pl.Vy[q] = c.vy[r];
                    }
                }
            }
            __syncthreads();
        }
    }
    // ---- write back the unknowns of the tile's own cells
    const int gx = w.ox0 + col;
    if (active && gx >= w.x0 && gx < w.x1) {
        const size_t P = (size_t)g.pitch;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int gy = w.oy0 + strip * R + r;
            if (gy >= w.y0 && gy < w.y1) {
                const size_t q = (size_t)gy * P + (size_t)gx;
                if (c.ux & (1u << r)) a.ox[q] = c.vx[r];
                if (c.uy & (1u << r)) a.oy[q] = c.vy[r];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// persistent TMA-staged kernel
// ---------------------------------------------------------------------------
template <typename T, int MAXT, int MINB, int WXM, int NS>
__global__ void __launch_bounds__(MAXT, MINB) k_ras_tma(const __grid_constant__ TmaMaps maps, RasArgs<T> a)
{
    constexpr int R = KCfg<T>::R;
    constexpr int NF = KCfg<T>::INVD ? 8 : 6;
    constexpr int ALIGN = 16 / (int)sizeof(T); // TMA x coordinates are multiples of 16 bytes
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    // TMA destinations must be 128-byte aligned shared addresses
    const uint32_t off = (128u - (smem_addr(smem_raw) & 127u)) & 127u;
    T *const stage = reinterpret_cast<T *>(smem_raw + off);
    const int BW = a.bw, SP = a.stage;
    const Geo<T, WXM, NS> G(a);
    const Planes<T> pl(stage + NF * SP, G.wp, G.spad, G.plane);

    const int ntiles = a.tg.ntx * a.tg.nty;
    const int col = (int)threadIdx.x % G.wxm, strip = (int)threadIdx.x / G.wxm;
    const bool active = (int)threadIdx.x < G.wxm * G.strips;
    const uint32_t box_bytes = (uint32_t)(BW * a.wym * (int)sizeof(T));

    auto issue = [&](int tile) {
        const Window w = window_of(a, tile);
        const int xs = w.ox0 & ~(ALIGN - 1);
        fence_proxy_async();
        mbar_arrive_expect_tx(&bar, NF * box_bytes);
#pragma unroll
        for (int f = 0; f < NF; ++f) tma_load_2d(stage + f * SP, &maps.m[f], xs, w.oy0, &bar);
    };

    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_proxy_async();
    }
    zero_borders(G, pl);
    __syncthreads();
    int tile = blockIdx.x;
    if (threadIdx.x == 0 && tile < ntiles) issue(tile);
    uint32_t phase = 0;
    while (tile < ntiles) {
        const bool ok = mbar_wait_bounded(&bar, phase, a.wait_limit);
        if (!__syncthreads_and(ok)) {
            // give up: record the timeout, let the copy in flight land, leave
            if (threadIdx.x == 0) {
                atomicExch(a.status, 1);
                mbar_wait_bounded(&bar, phase, 4000000000LL);
            }
            __syncthreads();
            return;
        }
        const Window w = window_of(a, tile);
        const int dx = w.ox0 - (w.ox0 & ~(ALIGN - 1));
        CellRegs<T, R> c;
        setup_cells<T, R>(a, G, w, c, col, strip, active, pl,
                          [&](int f, int wy, int wx) { return stage[f * SP + wy * BW + wx + dx]; });
        __syncthreads(); // staging consumed: refill it with the next tile
        const int next = tile + (int)gridDim.x;
        if (threadIdx.x == 0 && next < ntiles) issue(next);
        phase ^= 1u;
        sweep_and_store<T, R>(a, G, w, c, col, strip, active, pl);
        tile = next;
    }
}

// ---------------------------------------------------------------------------
// packed-pair FP32 kernel
// ---------------------------------------------------------------------------
// sm_100-class GPUs execute two FP32 additions, multiplications or fused
// multiply-adds of one thread as one instruction on a 64-bit register pair
// (add/sub/mul/fma.rn.f32x2).  Each lane of this kernel owns two adjacent
// window columns (c0 = 2 lane, c1 = c0 + 1) of PR rows, so every stencil
// operation of stencil.cuh runs once per column pair, lane for lane the same
// rounded operation: the results are those of the scalar kernels, bit for bit
// up to the sign of exact zeros.
// One warp spans a whole window row strip (up to 64 columns): horizontal
// neighbours come from the neighbouring lane by shuffles, and the only
// shared-memory traffic of a sweep is the first and last row of each strip.
// A strip computes the two neighbour fluxes it needs (Tyy of the row above
// it, the shear of the row below it) from those rows itself, so a sweep
// needs one barrier, with the edge rows double-buffered by sweep parity.
// Window columns 64 and -1 do not exist: the shuffles of lanes 31 and 0 then
// return the lane's own value, which only reaches the fluxes of the window's
// ring cells (never updated: weight 0) and stays finite.
struct f2 {
    unsigned long long u;
};
__device__ __forceinline__ f2 pk(float lo, float hi)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.u) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float f2lo(f2 a)
{
    float x, y;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a.u));
    return x;
}
__device__ __forceinline__ float f2hi(f2 a)
{
    float x, y;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a.u));
    return y;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b)
{
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.u) : "l"(a.u), "l"(b.u));
    return r;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b)
{
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.u) : "l"(a.u), "l"(b.u));
    return r;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b)
{
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.u) : "l"(a.u), "l"(b.u));
    return r;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.u) : "l"(a.u), "l"(b.u), "l"(c.u));
    return r;
}
// a * b rounded once and never fused into a following addition: the code
// generator contracts mul.rn.f32x2 followed by add/sub.rn.f32x2 into one
// fused multiply-add despite the rounding modifier (measured: a packed
// product minus a nearly equal value differs from the scalar rounded
// sequence in almost every case), so the product is formed as
// fma(a, b, +0), which rounds a * b once and is not contracted.  Its only
// difference from a plain product is the sign of an exact zero (+0 for -0).
__device__ __forceinline__ f2 mul2r(f2 a, f2 b)
{
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.u) : "l"(a.u), "l"(b.u), "l"(0ull));
    return r;
}
// (x(c0 - 1), x(c0)) and (x(c1), x(c1 + 1)) of a pair (x(c0), x(c1))
__device__ __forceinline__ f2 west_pair(f2 a) { return pk(__shfl_up_sync(0xffffffffu, f2hi(a), 1), f2lo(a)); }
__device__ __forceinline__ f2 east_pair(f2 a) { return pk(f2hi(a), __shfl_down_sync(0xffffffffu, f2lo(a), 1)); }

// rows per lane: with five, the 64 x 80 window takes 16 warps of up to 128
// registers (measured at 8192^2, 48 x 64 tiles, k = 8: 0.96 ms per launch,
// against 1.01 with four rows in 20 warps at 96 registers, 1.09 with six
// and 1.07 with eight)
constexpr int PR = 5;
constexpr int PAIR_COLS = 64;  // window columns of one warp
constexpr int PAIR_EDGE_KINDS = 4; // first-row vx, first-row vy, last-row vx, last-row vy
// edge rows per kind and buffer of a kernel of at most maxt threads: its
// strips plus the two zero strips -1 and ns
__host__ __device__ constexpr int pair_edge_stride(int maxt) { return maxt / 32 + 2; }

struct PairCells {
    f2 vx[PR], vy[PR], ax[PR], ay[PR], en[PR], bx[PR], by[PR], wx[PR], wy[PR];
    f2 en_below, ay_above; // eta_n of the next strip's first row, ay of the previous strip's last row
};

// fluxes of one row pair
struct PairFlux {
    f2 txx, tyy, sx, sy;
};

// Cell fields of one window cell from the staged boxes (zero outside the
// window), in the form setup_cells uses.
struct PairCell {
    float vx, vy, ec, en, bx, by, wx, wy;
    bool ux, uy;
};

template <class LD>
__device__ __forceinline__ PairCell pair_cell(const RasArgs<float> &a, const Window &w, int wy, int col, LD &&ld)
{
    const GridDesc<float> &g = a.g;
    PairCell p = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, false, false};
    if (wy < 0 || wy >= w.WY || col >= w.WX) return p;
    const int gx = w.ox0 + col, gy = w.oy0 + wy;
    p.vx = ld(0, wy, col);
    p.vy = ld(1, wy, col);
    p.ec = ld(2, wy, col);
    p.en = ld(3, wy, col);
    p.bx = ld(4, wy, col);
    p.by = ld(5, wy, col);
    const bool inner = col >= 1 && col < w.WX - 1 && wy >= 1 && wy < w.WY - 1;
    if (inner && gy >= 0 && gy < g.ny && gx >= 1 && gx <= g.nx - 1) {
        p.ux = true;
        p.wx = jacobi_weight(a.omega, ld(6, wy, col));
    }
    if (inner && gx >= 0 && gx < g.nx && gy >= 1 && gy <= g.ny - 1) {
        p.uy = true;
        p.wy = jacobi_weight(a.omega, ld(7, wy, col));
    }
    return p;
}

// SQ: square cells (1/hx = 1/hy and 1/hx^2 = 1/hy^2 bit for bit), where the
// coefficient of Tyy equals that of Txx and Sy equals Sx: the kernel keeps
// one of each (fewer registers, one packed multiply less per row).
// Staging row width of the pair kernels (elements): a 64-column window plus
// room for the alignment shift of its first column, for every pair window,
// so that every staged read is the lane's pointer plus a constant.
constexpr int PAIR_BW = 68;

// Registers of one strip from the staged window.  lp points at field 0, the
// strip's first row and column 2 lane of the window; field f starts SP
// elements after field f - 1.
template <bool SQ>
__device__ __forceinline__ void pair_setup(const RasArgs<float> &a, const Window &w, PairCells &c, int lane, int strip,
                                           const float *lp, int SP)
{
    const GridDesc<float> &g = a.g;
    const int c0 = 2 * lane;
    // Columns inside the window (the others read as zero) and inside its
    // ring (updated).  Row tests are the same for the whole warp.  A cell
    // inside the ring that is not an unknown (a wall, or outside the domain)
    // gets the weight omega x 0 = 0 from its staged 1/diag, which is zero
    // there (written so on the walls, zero-filled outside each array), so
    // no per-cell unknown test is needed.
    const bool in0 = c0 < w.WX, in1 = c0 + 1 < w.WX;
    const bool up0 = c0 >= 1 && c0 < w.WX - 1, up1 = c0 + 1 < w.WX - 1;
    const f2 om = pk(a.omega, a.omega), cx = pk(g.ihx2, g.ihx2), cy = pk(g.ihy2, g.ihy2);
    const bool sqc = SQ || g.square; // the square-cell shear (per grid, also in the general form)
    auto ld2 = [&](bool row, int f, int r) {
        const float *p = lp + f * SP + r * PAIR_BW;
        return pk(row && in0 ? p[0] : 0.f, row && in1 ? p[1] : 0.f);
    };
#pragma unroll
    for (int r = 0; r < PR; ++r) {
        const int wy = strip * PR + r;
        const bool row_in = wy < w.WY, row_up = wy >= 1 && wy < w.WY - 1;
        f2 v[8];
#pragma unroll
        for (int f = 0; f < 8; ++f) v[f] = ld2(row_in, f, r);
        c.vx[r] = v[0];
        c.vy[r] = v[1];
        // coef_x, coef_y and jacobi_weight of stencil.cuh, lane for lane
        const f2 e2 = add2(v[2], v[2]);
        c.ax[r] = mul2(e2, cx);
        c.ay[r] = SQ ? c.ax[r] : mul2(e2, cy);
        c.en[r] = sqc ? mul2(v[3], cx) : v[3]; // square cells: eta_n / h^2 (shear_sq)
        c.bx[r] = v[4];
        c.by[r] = v[5];
        const f2 wx = mul2(om, v[6]), wy2 = mul2(om, v[7]);
        c.wx[r] = pk(row_up && up0 ? f2lo(wx) : 0.f, row_up && up1 ? f2hi(wx) : 0.f);
        c.wy[r] = pk(row_up && up0 ? f2lo(wy2) : 0.f, row_up && up1 ? f2hi(wy2) : 0.f);
    }
    // eta_c of the row above the strip and eta_n of the row below it
    const f2 ea = ld2(strip > 0, 2, -1);
    c.ay_above = mul2(add2(ea, ea), cy);
    const f2 eb = ld2(strip * PR + PR < w.WY, 3, PR);
    c.en_below = sqc ? mul2(eb, cx) : eb;
}

// fluxes of row r: Txx, Tyy, Sx, Sy (vy_n: the vy pair of the row below r,
// vx_s: the vx pair of the row above it, both before this sweep)
template <bool SQ>
__device__ __forceinline__ PairFlux pair_flux(f2 ax, f2 ay, f2 en, f2 vx, f2 vy, f2 vy_n, f2 vx_s, f2 ihx, f2 ihy,
                                              bool sqc)
{
    PairFlux F;
    F.txx = mul2r(ax, sub2(east_pair(vx), vx));
    F.tyy = mul2r(SQ ? ax : ay, sub2(vy_n, vy));
    if (SQ || sqc) {
        // shear_sq of stencil.cuh; en holds eta_n / h^2
        F.sx = mul2r(en, add2(sub2(vx, vx_s), sub2(vy, west_pair(vy))));
        F.sy = F.sx;
    } else {
        const f2 sh = mul2(en, fma2(sub2(vx, vx_s), ihy, mul2(sub2(vy, west_pair(vy)), ihx)));
        F.sx = mul2r(sh, ihy);
        F.sy = mul2r(sh, ihx);
    }
    return F;
}

// ks local sweeps of the window in registers, then the write-back of the
// tile's own cells.  Ends with a barrier.  Edge rows: own = this lane's entry
// of its strip in buffer 0, kind 0; kind k of buffer b sits (4 b + k) ES 32
// pairs further and the strips above and below 32 pairs before and after
// (strips -1 and ns all zero).  ES is the kernel's maximum strips + 2, so
// every edge address is the lane's pointer plus a constant.
template <bool SQ, int ES>
__device__ __forceinline__ void pair_sweeps(const RasArgs<float> &a, const Window &w, PairCells &c, int lane, int strip,
                                            f2 *own)
{
    const GridDesc<float> &g = a.g;
    const f2 ihx = pk(g.ihx, g.ihx), ihy = pk(g.ihy, g.ihy);
    const bool sqc = SQ || g.square;
    constexpr int KS = ES * 32;
    // one sweep reading edge buffer RB and writing the other one
    auto sweep = [&](auto rbc) {
        constexpr int RB = decltype(rbc)::value, WB = RB ^ 1;
        const f2 vx_above = own[(RB * PAIR_EDGE_KINDS + 2) * KS - 32], vy_above = own[(RB * PAIR_EDGE_KINDS + 3) * KS - 32];
        const f2 vx_below = own[(RB * PAIR_EDGE_KINDS + 0) * KS + 32], vy_below = own[(RB * PAIR_EDGE_KINDS + 1) * KS + 32];
        // Tyy of the row above the strip and Sx of the row below it
        const f2 tyy_above = mul2r(c.ay_above, sub2(c.vy[0], vy_above));
        f2 sx_below;
        if (sqc) {
            sx_below = mul2r(c.en_below, add2(sub2(vx_below, c.vx[PR - 1]), sub2(vy_below, west_pair(vy_below))));
        } else {
            const f2 sh_below = mul2(c.en_below, fma2(sub2(vx_below, c.vx[PR - 1]), ihy,
                                                      mul2(sub2(vy_below, west_pair(vy_below)), ihx)));
            sx_below = mul2r(sh_below, ihy);
        }
        PairFlux F0 = pair_flux<SQ>(c.ax[0], c.ay[0], c.en[0], c.vx[0], c.vy[0], PR > 1 ? c.vy[1] : vy_below, vx_above,
                                    ihx, ihy, sqc);
        f2 tyy_s = tyy_above;
#pragma unroll
        for (int r = 0; r < PR; ++r) {
            // fluxes of row r + 1 read the old vx of row r: form them before row r moves
            PairFlux F1 = F0;
            if (r + 1 < PR)
                F1 = pair_flux<SQ>(c.ax[r + 1], c.ay[r + 1], c.en[r + 1], c.vx[r + 1], c.vy[r + 1],
                                   r + 2 < PR ? c.vy[r + 2] : vy_below, c.vx[r], ihx, ihy, sqc);
            const f2 sx_n = r + 1 < PR ? F1.sx : sx_below;
            const f2 mx = add2(sub2(F0.txx, west_pair(F0.txx)), sub2(sx_n, F0.sx));
            const f2 my = add2(sub2(east_pair(F0.sy), F0.sy), sub2(F0.tyy, tyy_s));
            c.vx[r] = fma2(sub2(c.bx[r], mx), c.wx[r], c.vx[r]);
            c.vy[r] = fma2(sub2(c.by[r], my), c.wy[r], c.vy[r]);
            tyy_s = F0.tyy;
            F0 = F1;
        }
        own[(WB * PAIR_EDGE_KINDS + 0) * KS] = c.vx[0];
        own[(WB * PAIR_EDGE_KINDS + 1) * KS] = c.vy[0];
        own[(WB * PAIR_EDGE_KINDS + 2) * KS] = c.vx[PR - 1];
        own[(WB * PAIR_EDGE_KINDS + 3) * KS] = c.vy[PR - 1];
        __syncthreads();
    };
    // sweep s (from 1) reads buffer (s - 1) mod 2
    int s = 0;
    for (; s + 2 <= a.ks; s += 2) {
        sweep(std::integral_constant<int, 0>());
        sweep(std::integral_constant<int, 1>());
    }
    if (s < a.ks) sweep(std::integral_constant<int, 0>());
    // ---- write back the tile's own cells.  Both components of every owned
    // cell are stored: the cells a sweep does not update (walls) keep their
    // staged value, which is the value already there (the walls of both
    // buffers of a ping-pong pair are the same), and an owned cell lies
    // inside both arrays' extents.
    const long long P = (long long)g.pitch;
    const int gx0 = w.ox0 + 2 * lane, gy0 = w.oy0 + strip * PR;
    const bool own0 = gx0 >= w.x0 && gx0 < w.x1, own1 = gx0 + 1 >= w.x0 && gx0 + 1 < w.x1;
    long long q = (long long)gy0 * P + gx0;
#pragma unroll
    for (int r = 0; r < PR; ++r, q += P) {
        if (gy0 + r < w.y0 || gy0 + r >= w.y1) continue;
        if (own0) {
            a.ox[q] = f2lo(c.vx[r]);
            a.oy[q] = f2lo(c.vy[r]);
        }
        if (own1) {
            a.ox[q + 1] = f2hi(c.vx[r]);
            a.oy[q + 1] = f2hi(c.vy[r]);
        }
    }
}

// Persistent TMA-staged kernel of the pair layout: one warp per strip of PR
// window rows, a.strips warps.  NST staging buffers: with two, the windows of
// the next two tiles are in flight while a tile is swept (one tile of
// prefetch leaves short sweeps waiting on HBM latency).  The timeout
// handling is that of k_ras_tma, waiting for every copy in flight.
template <int MAXT, int NST, bool SQ>
__global__ void __launch_bounds__(MAXT, 1) k_ras_pair(const __grid_constant__ TmaMaps maps, RasArgs<float> a)
{
    constexpr int NF = 8;
    constexpr int ALIGN = 4; // TMA x coordinates are multiples of 16 bytes
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[NST];
    __shared__ Window win[NST]; // window of the tile staged in buffer j, written by the thread that issues it
    const uint32_t off = (128u - (smem_addr(smem_raw) & 127u)) & 127u;
    float *const stage0 = reinterpret_cast<float *>(smem_raw + off);
    const int SP = a.stage;
    constexpr int ES = pair_edge_stride(MAXT);
    f2 *const edge = reinterpret_cast<f2 *>(stage0 + NST * NF * SP);
    const int ntiles = a.tg.ntx * a.tg.nty;
    const int grid = (int)gridDim.x;
    const int lane = (int)threadIdx.x & 31, strip = (int)threadIdx.x >> 5;
    const uint32_t box_bytes = (uint32_t)(PAIR_BW * a.wym * (int)sizeof(float));
    f2 *const own = edge + (strip + 1) * 32 + lane;

    auto issue = [&](int tile, int j) {
        const Window w = window_of(a, tile);
        win[j] = w;
        const int xs = w.ox0 & ~(ALIGN - 1);
        float *const st = stage0 + j * NF * SP;
        fence_proxy_async();
        mbar_arrive_expect_tx(&bar[j], NF * box_bytes);
#pragma unroll
        for (int f = 0; f < NF; ++f) tma_load_2d(st + f * SP, &maps.m[f], xs, w.oy0, &bar[j]);
    };

    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < NST; ++j) mbar_init(&bar[j], 1);
        fence_proxy_async();
    }
    // edge rows of the missing strips -1 and ns stay zero (the window's zero border)
    for (int t = (int)threadIdx.x; t < 2 * PAIR_EDGE_KINDS * ES * 32; t += (int)blockDim.x) edge[t].u = 0ull;
    __syncthreads();
    int tile = blockIdx.x;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < NST; ++j)
            if (tile + j * grid < ntiles) issue(tile + j * grid, j);
    }
    __syncthreads(); // the first windows are visible
    uint32_t phases = 0; // bit j: parity of the next completion of bar[j]
    int j = 0;           // staging buffer of `tile`
    while (tile < ntiles) {
        // Each thread waits for the window itself and goes on to its setup: a
        // warp that finished the previous tile's write-back early overlaps its
        // staged reads with the other warps' stores.  The edge rows it writes
        // are no longer read (the last sweep ended with a barrier).  The
        // threads agree on a timeout at the barrier after the setup; values
        // read from a window whose copy had not landed are then discarded.
        const bool ok = mbar_wait_bounded(&bar[j], (phases >> j) & 1u, a.wait_limit);
        const float *const stage = stage0 + j * NF * SP;
        const Window w = win[j];
        const int dx = w.ox0 - (w.ox0 & ~(ALIGN - 1));
        PairCells c;
        pair_setup<SQ>(a, w, c, lane, strip, stage + strip * PR * PAIR_BW + 2 * lane + dx, SP);
        own[0 * ES * 32] = c.vx[0];
        own[1 * ES * 32] = c.vy[0];
        own[2 * ES * 32] = c.vx[PR - 1];
        own[3 * ES * 32] = c.vy[PR - 1];
        if (!__syncthreads_and(ok)) { // staging buffer j consumed, edge rows visible
            // give up: record the timeout, let every copy in flight land, leave
            if (threadIdx.x == 0) {
                atomicExch(a.status, 1);
#pragma unroll
                for (int d = 0; d < NST; ++d) {
                    const int jj = (j + d) % NST;
                    if (tile + d * grid < ntiles) mbar_wait_bounded(&bar[jj], (phases >> jj) & 1u, 4000000000LL);
                }
            }
            __syncthreads();
            return;
        }
        const int refill = tile + NST * grid;
        if (threadIdx.x == 0 && refill < ntiles) issue(refill, j);
        phases ^= 1u << j;
        pair_sweeps<SQ, ES>(a, w, c, lane, strip, own);
        tile += grid;
        j = NST > 1 ? (j + 1) % NST : 0;
    }
}

// ---------------------------------------------------------------------------
// register-resident kernel reading the window from global memory
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(REG_MAX_THREADS) k_ras_reg(RasArgs<T> a)
{
    constexpr int R = KCfg<T>::R;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const Geo<T, 0, 0> G(a);
    const Planes<T> pl(reinterpret_cast<T *>(smem_raw), G.wp, G.spad, G.plane);
    const GridDesc<T> &g = a.g;
    const Window w = window_of(a, (int)blockIdx.x);
    const int col = threadIdx.x % a.wxm, strip = threadIdx.x / a.wxm;
    const bool active = (int)threadIdx.x < a.wxm * a.strips;
    const size_t P = (size_t)g.pitch;
    const T *const src[8] = {a.vx, a.vy, a.c.eta_c, a.c.eta_n, a.c.bx, a.c.by, a.c.inv_dx, a.c.inv_dy};
    zero_borders(G, pl);
    CellRegs<T, R> c;
    setup_cells<T, R>(a, G, w, c, col, strip, active, pl, [&](int f, int wy, int wx) {
        const int gy = w.oy0 + wy, gx = w.ox0 + wx;
        // extents: vx, bx, 1/dx ny x (nx+1); vy, by, 1/dy (ny+1) x nx; eta_c ny x nx; eta_n (ny+1) x (nx+1)
        const int ey = (f == 0 || f == 2 || f == 4 || f == 6) ? g.ny : g.ny + 1;
        const int ex = (f == 1 || f == 2 || f == 5 || f == 7) ? g.nx : g.nx + 1;
        return (gy >= 0 && gy < ey && gx >= 0 && gx < ex) ? src[f][(size_t)gy * P + (size_t)gx] : T(0);
    });
    __syncthreads();
    sweep_and_store<T, R>(a, G, w, c, col, strip, active, pl);
}

// entry of the launch's table that owns tile t: from the per-tile map when
// the launch has one, else by binary search on tile_begin
template <typename T>
__device__ __forceinline__ int batch_entry(const BatchTiles<T> *__restrict__ tab, const int *__restrict__ tmap,
                                           int count, int t)
{
    if (tmap) return tmap[t];
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tab[mid].tile_begin <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// batched persistent kernel: the tiles of many instances in one launch
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(REG_MAX_THREADS) k_ras_batched(const BatchTiles<T> *__restrict__ tab,
                                                                 const int *__restrict__ tmap, int count,
                                                                 int total, const int *__restrict__ live,
                                                                 RasArgs<T> shape)
{
    constexpr int R = KCfg<T>::R;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const Geo<T, 0, 0> G(shape);
    const Planes<T> pl(reinterpret_cast<T *>(smem_raw), G.wp, G.spad, G.plane);
    const int col = threadIdx.x % shape.wxm, strip = threadIdx.x / shape.wxm;
    const bool active = (int)threadIdx.x < shape.wxm * shape.strips;
    zero_borders(G, pl);
    __syncthreads();
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const BatchTiles<T> &e = tab[batch_entry(tab, tmap, count, t)];
        if (live && !live[e.inst]) continue;
        RasArgs<T> a = shape;
        a.g = e.g;
        a.c = e.c;
        a.vx = e.vx;
        a.vy = e.vy;
        a.ox = e.ox;
        a.oy = e.oy;
        a.tg = e.tg;
        const Window w = window_of(a, t - e.tile_begin);
        const GridDesc<T> &g = a.g;
        const size_t P = (size_t)g.pitch;
        const T *const src[8] = {a.vx, a.vy, a.c.eta_c, a.c.eta_n, a.c.bx, a.c.by, a.c.inv_dx, a.c.inv_dy};
        CellRegs<T, R> c;
        setup_cells<T, R>(a, G, w, c, col, strip, active, pl, [&](int f, int wy, int wx) {
            const int gy = w.oy0 + wy, gx = w.ox0 + wx;
            const int ey = (f == 0 || f == 2 || f == 4 || f == 6) ? g.ny : g.ny + 1;
            const int ex = (f == 1 || f == 2 || f == 5 || f == 7) ? g.nx : g.nx + 1;
            return (gy >= 0 && gy < ey && gx >= 0 && gx < ex) ? src[f][(size_t)gy * P + (size_t)gx] : T(0);
        });
        __syncthreads();
        sweep_and_store<T, R>(a, G, w, c, col, strip, active, pl);
    }
}

// batched persistent TMA-staged kernel: tile t of the launch belongs to the
// last instance whose tile_begin <= t; instance e's windows are staged
// through its own tensor maps maps[e] (global memory), the next tile's copy
// overlapping the current tile's sweeps as in k_ras_tma

template <typename T>
__device__ __forceinline__ RasArgs<T> batch_args(const RasArgs<T> &shape, const BatchTiles<T> &e)
{
    RasArgs<T> a = shape;
    a.g = e.g;
    a.c = e.c;
    a.vx = e.vx;
    a.vy = e.vy;
    a.ox = e.ox;
    a.oy = e.oy;
    a.tg = e.tg;
    return a;
}

template <typename T, int MAXT, int MINB, int WXM, int NS>
__global__ void __launch_bounds__(MAXT, MINB) k_ras_batched_tma(const BatchTiles<T> *__restrict__ tab,
                                                                const int *__restrict__ tmap,
                                                                const TmaMaps *__restrict__ maps, int count,
                                                                int total, const int *__restrict__ live,
                                                                RasArgs<T> shape)
{
    constexpr int R = KCfg<T>::R;
    constexpr int NF = KCfg<T>::INVD ? 8 : 6;
    constexpr int ALIGN = 16 / (int)sizeof(T);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    const uint32_t off = (128u - (smem_addr(smem_raw) & 127u)) & 127u;
    T *const stage = reinterpret_cast<T *>(smem_raw + off);
    const int BW = shape.bw, SP = shape.stage;
    const Geo<T, WXM, NS> G(shape);
    const Planes<T> pl(stage + NF * SP, G.wp, G.spad, G.plane);
    const int col = (int)threadIdx.x % G.wxm, strip = (int)threadIdx.x / G.wxm;
    const bool active = (int)threadIdx.x < G.wxm * G.strips;
    const uint32_t box_bytes = (uint32_t)(BW * shape.wym * (int)sizeof(T));

    // Each CTA takes chunks of CH consecutive tiles, chunk c, c + gridDim.x,
    // ...: consecutive tiles mostly belong to one instance, so the cursor
    // (e, tb, te) = (entry, its first tile, one past its last) usually just
    // steps on and the instance's arguments are reloaded only when it
    // changes, while the round-robin over chunks keeps the CTAs balanced when
    // finished instances drop out.
    constexpr int CH = 8;
    const int stride = (int)gridDim.x * CH;
    auto end_of = [&](int e) { return tab[e].tile_begin + tab[e].tg.ntx * tab[e].tg.nty; };
    int e = 0, tb = 0, te = 0;
    auto seek = [&](int t) {
        if (t < tb || t >= te) {
            e = batch_entry(tab, tmap, count, t);
            tb = tab[e].tile_begin;
            te = end_of(e);
        }
    };
    // this CTA's position after t in its sequence of chunks
    auto step = [&](int t) { return (t + 1) % CH ? t + 1 : t + 1 - CH + stride; };
    // first position >= t (in this CTA's sequence) whose instance is live
    auto advance = [&](int t) {
        while (t < total) {
            seek(t);
            if (live && !live[tab[e].inst]) {
                // skip the rest of this instance within the chunk
                const int cend = (t / CH + 1) * CH;
                t = te < cend ? te : cend - CH + stride;
                continue;
            }
            break;
        }
        return t;
    };

    int ea = -1; // entry whose arguments `a` holds
    RasArgs<T> a = shape;
    // tensor maps are acquired once per instance by the issuing thread
    int acquired = -1;
    auto issue = [&](int t, int e, int tb) {
        Window w;
        if (e == ea) {
            w = window_of(a, t - tb);
        } else {
            const RasArgs<T> b = batch_args(shape, tab[e]);
            w = window_of(b, t - tb);
        }
        const int xs = w.ox0 & ~(ALIGN - 1);
        if (e != acquired) {
#pragma unroll
            for (int f = 0; f < NF; ++f) fence_tensormap_acquire(&maps[e].m[f]);
            acquired = e;
        }
        fence_proxy_async();
        mbar_arrive_expect_tx(&bar, NF * box_bytes);
#pragma unroll
        for (int f = 0; f < NF; ++f) tma_load_2d(stage + f * SP, &maps[e].m[f], xs, w.oy0, &bar);
    };

    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_proxy_async();
    }
    zero_borders(G, pl);
    __syncthreads();
    int tile = advance((int)blockIdx.x * CH);
    if (threadIdx.x == 0 && tile < total) issue(tile, e, tb);
    uint32_t phase = 0;
    while (tile < total) {
        const bool ok = mbar_wait_bounded(&bar, phase, shape.wait_limit);
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) {
                atomicExch(shape.status, 1);
                mbar_wait_bounded(&bar, phase, 4000000000LL);
            }
            __syncthreads();
            return;
        }
        if (e != ea) {
            a = batch_args(shape, tab[e]);
            ea = e;
        }
        const Window w = window_of(a, tile - tb);
        const int dx = w.ox0 - (w.ox0 & ~(ALIGN - 1));
        CellRegs<T, R> c;
        setup_cells<T, R>(a, G, w, c, col, strip, active, pl,
                          [&](int f, int wy, int wx) { return stage[f * SP + wy * BW + wx + dx]; });
        __syncthreads();
        const int next = advance(step(tile));
        if (threadIdx.x == 0 && next < total) issue(next, e, tb);
        phase ^= 1u;
        sweep_and_store<T, R>(a, G, w, c, col, strip, active, pl);
        tile = next;
    }
}

// Batched form of the packed-pair FP32 kernel: the tile walk, per-instance
// tensor maps and live-instance skipping of k_ras_batched_tma, the window
// setup and sweeps of k_ras_pair (one staging buffer: the next tile's copy is
// issued once the current window is in registers and lands while it is swept).
template <int MAXT, bool SQ>
__global__ void __launch_bounds__(MAXT, 1) k_ras_batched_pair(const BatchTiles<float> *__restrict__ tab,
                                                              const int *__restrict__ tmap,
                                                              const TmaMaps *__restrict__ maps, int count, int total,
                                                              const int *__restrict__ live, RasArgs<float> shape)
{
    constexpr int NF = 8;
    constexpr int ALIGN = 4; // TMA x coordinates are multiples of 16 bytes
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    const uint32_t off = (128u - (smem_addr(smem_raw) & 127u)) & 127u;
    float *const stage = reinterpret_cast<float *>(smem_raw + off);
    const int SP = shape.stage;
    constexpr int ES = pair_edge_stride(MAXT);
    f2 *const edge = reinterpret_cast<f2 *>(stage + NF * SP);
    const int lane = (int)threadIdx.x & 31, strip = (int)threadIdx.x >> 5;
    const uint32_t box_bytes = (uint32_t)(PAIR_BW * shape.wym * (int)sizeof(float));
    f2 *const own = edge + (strip + 1) * 32 + lane;

    constexpr int CH = 8; // chunks of consecutive tiles per CTA, as in k_ras_batched_tma
    const int stride = (int)gridDim.x * CH;
    auto end_of = [&](int e) { return tab[e].tile_begin + tab[e].tg.ntx * tab[e].tg.nty; };
    int e = 0, tb = 0, te = 0;
    auto seek = [&](int t) {
        if (t < tb || t >= te) {
            e = batch_entry(tab, tmap, count, t);
            tb = tab[e].tile_begin;
            te = end_of(e);
        }
    };
    auto step = [&](int t) { return (t + 1) % CH ? t + 1 : t + 1 - CH + stride; };
    auto advance = [&](int t) {
        while (t < total) {
            seek(t);
            if (live && !live[tab[e].inst]) {
                const int cend = (t / CH + 1) * CH;
                t = te < cend ? te : cend - CH + stride;
                continue;
            }
            break;
        }
        return t;
    };

    int ea = -1;
    RasArgs<float> a = shape;
    int acquired = -1;
    auto issue = [&](int t, int e, int tb) {
        Window w;
        if (e == ea) {
            w = window_of(a, t - tb);
        } else {
            const RasArgs<float> b = batch_args(shape, tab[e]);
            w = window_of(b, t - tb);
        }
        const int xs = w.ox0 & ~(ALIGN - 1);
        if (e != acquired) {
#pragma unroll
            for (int f = 0; f < NF; ++f) fence_tensormap_acquire(&maps[e].m[f]);
            acquired = e;
        }
        fence_proxy_async();
        mbar_arrive_expect_tx(&bar, NF * box_bytes);
#pragma unroll
        for (int f = 0; f < NF; ++f) tma_load_2d(stage + f * SP, &maps[e].m[f], xs, w.oy0, &bar);
    };

    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_proxy_async();
    }
    // edge rows of the missing strips -1 and ns stay zero (the window's zero border)
    for (int t = (int)threadIdx.x; t < 2 * PAIR_EDGE_KINDS * ES * 32; t += (int)blockDim.x) edge[t].u = 0ull;
    __syncthreads();
    int tile = advance((int)blockIdx.x * CH);
    if (threadIdx.x == 0 && tile < total) issue(tile, e, tb);
    uint32_t phase = 0;
    while (tile < total) {
        // as in k_ras_pair: no barrier before the setup, the timeout agreed on
        // at the barrier after it
        const bool ok = mbar_wait_bounded(&bar, phase, shape.wait_limit);
        if (e != ea) {
            a = batch_args(shape, tab[e]);
            ea = e;
        }
        const Window w = window_of(a, tile - tb);
        const int dx = w.ox0 - (w.ox0 & ~(ALIGN - 1));
        PairCells c;
        pair_setup<SQ>(a, w, c, lane, strip, stage + strip * PR * PAIR_BW + 2 * lane + dx, SP);
        own[0 * ES * 32] = c.vx[0];
        own[1 * ES * 32] = c.vy[0];
        own[2 * ES * 32] = c.vx[PR - 1];
        own[3 * ES * 32] = c.vy[PR - 1];
        if (!__syncthreads_and(ok)) { // staging buffer consumed, edge rows visible
            if (threadIdx.x == 0) {
                atomicExch(shape.status, 1);
                mbar_wait_bounded(&bar, phase, 4000000000LL);
            }
            __syncthreads();
            return;
        }
        const int next = advance(step(tile));
        if (threadIdx.x == 0 && next < total) issue(next, e, tb);
        phase ^= 1u;
        pair_sweeps<SQ, ES>(a, w, c, lane, strip, own);
        tile = next;
    }
}

// ---------------------------------------------------------------------------
// general kernel: every field of the window in shared memory
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void ras_smem_tile(const RasArgs<T> &a, int tile, T *sm)
{
    const int plane = a.plane, W = a.wp;
    T *Ax = sm, *Ay = sm + plane, *Bx = sm + 2 * plane, *By = sm + 3 * plane;
    T *Ec = sm + 4 * plane, *En = sm + 5 * plane, *Rx = sm + 6 * plane, *Ry = sm + 7 * plane;

    const GridDesc<T> &g = a.g;
    const int nx = g.nx, ny = g.ny;
    const size_t P = (size_t)g.pitch;
    const Window win = window_of(a, tile);
    const int x0 = win.x0, x1 = win.x1, y0 = win.y0, y1 = win.y1, ox0 = win.ox0, oy0 = win.oy0;
    const int wx = win.WX, wy = win.WY;

    for (int p = threadIdx.x; p < wx * wy; p += RAS_THREADS) {
        const int ly = p / wx, lx = p - ly * wx;
        const int gy = oy0 + ly, gx = ox0 + lx;
        T vxv = T(0), vyv = T(0), ecv = T(0), env = T(0), bxv = T(0), byv = T(0);
        if (gx >= 0 && gx <= nx && gy >= 0 && gy <= ny) {
            const size_t q = (size_t)gy * P + (size_t)gx;
            if (gy < ny) {
                vxv = a.vx[q];
                bxv = a.c.bx[q];
                if (gx < nx) ecv = a.c.eta_c[q];
            }
            if (gx < nx) {
                vyv = a.vy[q];
                byv = a.c.by[q];
            }
            env = a.c.eta_n[q];
        }
        const int s = ly * W + lx;
        Ax[s] = vxv;
        Bx[s] = vxv;
        Ay[s] = vyv;
        By[s] = vyv;
        Ec[s] = ecv;
        En[s] = env;
        Rx[s] = bxv;
        Ry[s] = byv;
    }
    __syncthreads();

    T *cx = Ax, *cy = Ay, *nxv = Bx, *nyv = By;
    for (int s = 1; s <= a.ks; ++s) {
        const int r = min(a.overlap, a.ks - s);
        const int cx0 = max(x0 - r, 0), cx1 = min(x1 + r, nx);
        const int cy0 = max(y0 - r, 0), cy1 = min(y1 + r, ny);
        const int w = cx1 - cx0, npts = w * (cy1 - cy0);
        for (int p = threadIdx.x; p < npts; p += RAS_THREADS) {
            const int yy = p / w;
            const int gx = cx0 + (p - yy * w), gy = cy0 + yy;
            const int q = (gy - oy0) * W + (gx - ox0);
            if (gx >= 1 && gx <= nx - 1) { // vx unknown (gy < ny holds)
                const T vc = cx[q];
                const T txx_c = flux_n(coef_x(g, Ec[q]), cx[q + 1], vc);
                const T txx_w = flux_n(coef_x(g, Ec[q - 1]), vc, cx[q - 1]);
                const T sx_n = shear_x(g, En[q + W], cx[q + W], vc, cy[q + W], cy[q + W - 1]);
                const T sx_c = shear_x(g, En[q], vc, cx[q - W], cy[q], cy[q - 1]);
                const T d = diag_x(g, Ec[q], Ec[q - 1], En[q + W], En[q]);
                nxv[q] = jacobi_update(vc, Rx[q], m_x(txx_c, txx_w, sx_n, sx_c), jacobi_weight(a.omega, inv_diag(d)));
            }
            if (gy >= 1 && gy <= ny - 1) { // vy unknown (gx < nx holds)
                const T vc = cy[q];
                const T tyy_c = flux_n(coef_y(g, Ec[q]), cy[q + W], vc);
                const T tyy_s = flux_n(coef_y(g, Ec[q - W]), vc, cy[q - W]);
                const T sy_e = shear_y(g, En[q + 1], cx[q + 1], cx[q + 1 - W], cy[q + 1], vc);
                const T sy_c = shear_y(g, En[q], cx[q], cx[q - W], vc, cy[q - 1]);
                const T d = diag_y(g, Ec[q], Ec[q - W], En[q + 1], En[q]);
                nyv[q] = jacobi_update(vc, Ry[q], m_y(sy_e, sy_c, tyy_c, tyy_s), jacobi_weight(a.omega, inv_diag(d)));
            }
        }
        __syncthreads();
        T *t0 = cx;
        cx = nxv;
        nxv = t0;
        T *t1 = cy;
        cy = nyv;
        nyv = t1;
    }

    const int tw = x1 - x0, npts = tw * (y1 - y0);
    for (int p = threadIdx.x; p < npts; p += RAS_THREADS) {
        const int yy = p / tw;
        const int gx = x0 + (p - yy * tw), gy = y0 + yy;
        const int q = (gy - oy0) * W + (gx - ox0);
        const size_t gq = (size_t)gy * P + (size_t)gx;
        if (gx >= 1 && gx <= nx - 1) a.ox[gq] = cx[q];
        if (gy >= 1 && gy <= ny - 1) a.oy[gq] = cy[q];
    }
}

template <typename T>
__global__ void __launch_bounds__(RAS_THREADS) k_ras(RasArgs<T> a)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    ras_smem_tile(a, (int)blockIdx.x, reinterpret_cast<T *>(smem_raw));
}

// batched form of the general kernel: one CTA per tile of the launch's list
template <typename T>
__global__ void __launch_bounds__(RAS_THREADS) k_ras_batched_smem(const BatchTiles<T> *__restrict__ tab,
                                                                  const int *__restrict__ tmap, int count,
                                                                  const int *__restrict__ live, RasArgs<T> shape)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int t = (int)blockIdx.x;
    const BatchTiles<T> &e = tab[batch_entry(tab, tmap, count, t)];
    if (live && !live[e.inst]) return;
    RasArgs<T> a = shape;
    a.g = e.g;
    a.c = e.c;
    a.vx = e.vx;
    a.vy = e.vy;
    a.ox = e.ox;
    a.oy = e.oy;
    a.tg = e.tg;
    ras_smem_tile(a, t - e.tile_begin, reinterpret_cast<T *>(smem_raw));
}

// which kernel a configuration uses, and its launch shape
enum { PLAN_TMA = 0, PLAN_REG = 1, PLAN_SMEM = 2, PLAN_PAIR = 3 };
struct RasPlan {
    int kind;
    int wxm, wym, strips, wp, spad, plane, threads, bw, stage;
    int nstage = 1; // staging buffers (pair kernel)
    size_t smem;
};

constexpr int PAIR_MAX_THREADS = 512;
constexpr int PAIR_SMALL_THREADS = 384; // the smaller pair kernel instance
// Narrower windows leave lanes idle; up to this width the one-column kernel is
// as fast or faster (measured at 8192^2: 40 columns 264 vs 177 Gcell/s, 48
// columns equal)
constexpr int PAIR_MIN_COLS = 48;

// pair_mode: 0 never the pair kernel, 1 for windows of PAIR_MIN_COLS + 1 to
// PAIR_COLS columns, 2 for any window of at most PAIR_COLS columns
RasPlan plan_ras(int nx, int ny, int ti, int tj, int overlap, size_t elem, bool allow_tma, int pair_mode = 0)
{
    RasPlan p;
    const int h = overlap + 1;
    const int R = elem == 8 ? KCfg<double>::R : KCfg<float>::R;
    const int nf = (elem == 8 ? KCfg<double>::INVD : KCfg<float>::INVD) ? 8 : 6;
    // a tile never spans more than min(T, n) cells
    p.wxm = std::min(ti, nx) + 2 * h;
    p.wym = std::min(tj, ny) + 2 * h;
    p.strips = (p.wym + R - 1) / R;
    const long threads = (long)p.wxm * p.strips;
    const size_t maxs = (size_t)ras_max_smem();
    p.wp = p.wxm + 2;
    // strip stride congruent to the window width modulo 32 banks
    p.spad = (((p.wxm - R * p.wp) % 32) + 32) % 32;
    p.plane = p.wp * (p.strips * R + 2) + (p.strips + 1) * p.spad;
    const int align = 16 / (int)elem;
    p.bw = (p.wxm + align - 1 + align - 1) / align * align; // room for the alignment shift of x
    p.stage = (int)((((size_t)p.bw * p.wym * elem + 127) / 128 * 128) / elem);
    const size_t reg_smem = (size_t)REG_PLANES * (size_t)p.plane * elem;
    const size_t tma_smem = (size_t)nf * (size_t)p.stage * elem + reg_smem + 128;
    p.threads = (int)((threads + 31) / 32 * 32);
    if (elem == 4 && allow_tma && pair_mode > 0 && p.wxm <= PAIR_COLS && (pair_mode > 1 || p.wxm > PAIR_MIN_COLS) &&
        p.bw <= 256 && p.wym <= 256) {
        // packed-pair layout: one warp per strip of PR rows, edge rows double-buffered,
        // two staging buffers when they fit
        const int strips = (p.wym + PR - 1) / PR;
        const int maxt = 32 * strips <= PAIR_SMALL_THREADS ? PAIR_SMALL_THREADS : PAIR_MAX_THREADS; // the kernel instance that runs it
        const size_t edge = (size_t)2 * PAIR_EDGE_KINDS * pair_edge_stride(maxt) * 32 * sizeof(f2);
        const int bw = PAIR_BW, stage = (int)((((size_t)bw * p.wym * elem + 127) / 128 * 128) / elem);
        const size_t one = (size_t)nf * (size_t)stage * elem;
        if (32 * strips <= PAIR_MAX_THREADS && one + edge + 128 <= maxs) {
            p.kind = PLAN_PAIR;
            p.bw = bw;
            p.stage = stage;
            p.strips = strips;
            p.threads = 32 * strips;
            p.nstage = 2 * one + edge + 128 <= maxs ? 2 : 1;
            p.smem = p.nstage * one + edge + 128;
            return p;
        }
    }
    if (threads <= REG_MAX_THREADS && allow_tma && p.bw <= 256 && p.wym <= 256 && tma_smem <= maxs) {
        p.kind = PLAN_TMA;
        p.smem = tma_smem;
    } else if (threads <= REG_MAX_THREADS && reg_smem <= maxs) {
        p.kind = PLAN_REG;
        p.smem = reg_smem;
    } else {
        p.kind = PLAN_SMEM;
        p.wp = p.wxm;
        p.spad = 0;
        p.plane = p.wxm * p.wym;
        p.smem = (size_t)RAS_PLANES * (size_t)p.plane * elem;
        p.threads = RAS_THREADS;
    }
    return p;
}

int sm_count()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v;
}

} // namespace

TileGrid make_tiles(int nx, int ny, int ti, int tj, int si, int sj)
{
    TileGrid t;
    t.ti = ti;
    t.tj = tj;
    t.si = si;
    t.sj = sj;
    const int fx = si > 0 ? si : ti, fy = sj > 0 ? sj : tj;
    t.ntx = fx >= nx ? 1 : 1 + (nx - fx + ti - 1) / ti;
    t.nty = fy >= ny ? 1 : 1 + (ny - fy + tj - 1) / tj;
    return t;
}

void ras_kernel_plan(int nx, int ny, int ti, int tj, int overlap, size_t elem, bool allow_tma, int pair_mode,
                     int *kind, int *threads, size_t *smem)
{
    const RasPlan p = plan_ras(nx, ny, ti, tj, overlap, elem, allow_tma, pair_mode);
    *kind = p.kind;
    *threads = p.threads;
    *smem = p.smem;
}

bool ras_whole_level_tile(int nx, int ny, size_t elem)
{
    // one tile of the whole level, overlap 0: worth it when the window fits a
    // register layout (a single CTA of the general kernel is slower than the
    // level's regular tiling)
    return nx <= 64 && ny <= 64 && plan_ras(nx, ny, nx, ny, 0, elem, true, 0).kind != PLAN_SMEM;
}

size_t ras_smem_bytes(int nx, int ny, int ti, int tj, int overlap, size_t elem)
{
    return plan_ras(nx, ny, ti, tj, overlap, elem, false).smem;
}

int ras_max_smem()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

// Kernel instance for a TMA plan.  FP32 windows of up to 320 threads cap
// registers so that two CTAs share an SM (FP64 is bound by its FP64 pipe and
// keeps 128 registers).  The window shapes of the common tiles (32 x 32 and
// 56 x 32 with overlap 0 or 3 in FP32, 32 x 32 with overlap 3 in FP64) get
// instances with compile-time plane geometry; the others use the generic one.
template <int WXM, int NS, typename T>
bool geo_matches(const RasPlan &p)
{
    using G = Geo<T, WXM, NS>;
    return p.wxm == WXM && p.strips == NS && p.wp == G::WPC && p.spad == G::SPC && p.plane == G::PLC;
}

template <typename T>
void (*pick_tma(const RasPlan &p))(TmaMaps, RasArgs<T>)
{
    if constexpr (sizeof(T) == 4) {
        if (geo_matches<64, 8, T>(p)) return k_ras_tma<T, REG_MAX_THREADS, 1, 64, 8>;
        if (geo_matches<58, 7, T>(p)) return k_ras_tma<T, REG_MAX_THREADS, 1, 58, 7>;
        if (geo_matches<40, 8, T>(p)) return k_ras_tma<T, SMALL_THREADS, 2, 40, 8>;
        if (geo_matches<34, 7, T>(p)) return k_ras_tma<T, SMALL_THREADS, 2, 34, 7>;
        if (p.threads <= SMALL_THREADS) return k_ras_tma<T, SMALL_THREADS, 2, 0, 0>;
    } else {
        if (geo_matches<40, 10, T>(p)) return k_ras_tma<T, REG_MAX_THREADS, 1, 40, 10>;
    }
    return k_ras_tma<T, REG_MAX_THREADS, 1, 0, 0>;
}

template <typename T>
void (*pick_batched_tma(const RasPlan &p))(const BatchTiles<T> *, const int *, const TmaMaps *, int, int, const int *,
                                           RasArgs<T>)
{
    if constexpr (sizeof(T) == 4) {
        if (geo_matches<64, 8, T>(p)) return k_ras_batched_tma<T, REG_MAX_THREADS, 1, 64, 8>;
        if (geo_matches<58, 7, T>(p)) return k_ras_batched_tma<T, REG_MAX_THREADS, 1, 58, 7>;
        if (geo_matches<40, 8, T>(p)) return k_ras_batched_tma<T, SMALL_THREADS, 2, 40, 8>;
        if (geo_matches<34, 7, T>(p)) return k_ras_batched_tma<T, SMALL_THREADS, 2, 34, 7>;
        if (p.threads <= SMALL_THREADS) return k_ras_batched_tma<T, SMALL_THREADS, 2, 0, 0>;
    } else {
        if (geo_matches<40, 10, T>(p)) return k_ras_batched_tma<T, REG_MAX_THREADS, 1, 40, 10>;
    }
    return k_ras_batched_tma<T, REG_MAX_THREADS, 1, 0, 0>;
}

template <typename T>
cudaError_t launch_ras(const GridDesc<T> &g, const Coeffs<T> &c, T omega, const TileGrid &tg, int ksweeps,
                       int overlap, const T *vx, const T *vy, T *ox, T *oy, const RasRun &run, cudaStream_t s)
{
    constexpr int NF = KCfg<T>::INVD ? 8 : 6;
    const bool have_inv = c.inv_dx && c.inv_dy;
    const RasPlan p = plan_ras(g.nx, g.ny, tg.ti, tg.tj, overlap, sizeof(T), run.allow_tma, run.pair_mode);
    RasArgs<T> a;
    a.g = g;
    a.c = c;
    a.omega = omega;
    a.vx = vx;
    a.vy = vy;
    a.ox = ox;
    a.oy = oy;
    a.tg = tg;
    a.ks = ksweeps;
    a.overlap = overlap;
    a.wxm = p.wxm;
    a.wym = p.wym;
    a.strips = p.strips;
    a.wp = p.wp;
    a.spad = p.spad;
    a.plane = p.plane;
    a.bw = p.bw;
    a.stage = p.stage;
    a.status = run.status;
    a.wait_limit = run.wait_limit;
    const int ntiles = tg.ntx * tg.nty;
    cudaError_t e;
    if (KCfg<T>::INVD && !have_inv && p.kind != PLAN_SMEM) return cudaErrorInvalidValue;
    if (p.kind == PLAN_TMA || p.kind == PLAN_PAIR) {
        TmaMaps m;
        const int es = (int)sizeof(T);
        const long pb = (long)g.pitch * es;
        const void *ptrs[8] = {vx, vy, c.eta_c, c.eta_n, c.bx, c.by, c.inv_dx, c.inv_dy};
        const int widths[8] = {g.nx + 1, g.nx, g.nx, g.nx + 1, g.nx + 1, g.nx, g.nx + 1, g.nx};
        const int heights[8] = {g.ny, g.ny + 1, g.ny, g.ny + 1, g.ny, g.ny + 1, g.ny, g.ny + 1};
        for (int f = 0; f < NF; ++f) {
            e = make_tmap_2d(&m.m[f], ptrs[f], es, widths[f], heights[f], pb, p.bw, p.wym);
            if (e != cudaSuccess) return e;
        }
        void (*kern)(TmaMaps, RasArgs<T>) = pick_tma<T>(p);
        if constexpr (sizeof(T) == 4) {
            if (p.kind == PLAN_PAIR) {
                const bool sq = g.square != 0;
                if (sq) {
                    if (p.nstage == 2)
                        kern = p.threads <= PAIR_SMALL_THREADS ? k_ras_pair<PAIR_SMALL_THREADS, 2, true> : k_ras_pair<PAIR_MAX_THREADS, 2, true>;
                    else
                        kern = p.threads <= PAIR_SMALL_THREADS ? k_ras_pair<PAIR_SMALL_THREADS, 1, true> : k_ras_pair<PAIR_MAX_THREADS, 1, true>;
                } else {
                    if (p.nstage == 2)
                        kern = p.threads <= PAIR_SMALL_THREADS ? k_ras_pair<PAIR_SMALL_THREADS, 2, false> : k_ras_pair<PAIR_MAX_THREADS, 2, false>;
                    else
                        kern = p.threads <= PAIR_SMALL_THREADS ? k_ras_pair<PAIR_SMALL_THREADS, 1, false> : k_ras_pair<PAIR_MAX_THREADS, 1, false>;
                }
            }
        }
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, p.threads, p.smem);
        if (e != cudaSuccess) return e;
        const int grid = std::min(ntiles, std::max(per_sm, 1) * sm_count());
        kern<<<grid, p.threads, p.smem, s>>>(m, a);
    } else if (p.kind == PLAN_REG) {
        e = cudaFuncSetAttribute(k_ras_reg<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
        if (e != cudaSuccess) return e;
        k_ras_reg<T><<<ntiles, p.threads, p.smem, s>>>(a);
    } else {
        e = cudaFuncSetAttribute(k_ras<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
        if (e != cudaSuccess) return e;
        k_ras<T><<<ntiles, RAS_THREADS, p.smem, s>>>(a);
    }
    return cudaGetLastError();
}

size_t ras_batched_smem_bytes(int ti, int tj, int overlap, size_t elem)
{
    return plan_ras(ti, tj, ti, tj, overlap, elem, false).smem;
}

bool ras_batched_tma(int ti, int tj, int overlap, size_t elem, int pair_mode)
{
    const int kind = plan_ras(ti, tj, ti, tj, overlap, elem, true, pair_mode).kind;
    return kind == PLAN_TMA || kind == PLAN_PAIR;
}

size_t ras_batched_maps_bytes() { return sizeof(TmaMaps); }

template <typename T>
cudaError_t ras_batched_encode(const BatchTiles<T> *tab, int count, int ti, int tj, int overlap, int pair_mode,
                               void *out)
{
    constexpr int NF = KCfg<T>::INVD ? 8 : 6;
    // the pair and the one-column plans stage the same boxes
    const RasPlan p = plan_ras(ti, tj, ti, tj, overlap, sizeof(T), true, pair_mode);
    if (p.kind != PLAN_TMA && p.kind != PLAN_PAIR) return cudaErrorInvalidValue;
    TmaMaps *m = reinterpret_cast<TmaMaps *>(out);
    const int es = (int)sizeof(T);
    for (int i = 0; i < count; ++i) {
        const BatchTiles<T> &e = tab[i];
        const GridDesc<T> &g = e.g;
        if (NF == 8 && (!e.c.inv_dx || !e.c.inv_dy)) return cudaErrorInvalidValue;
        const void *ptrs[8] = {e.vx, e.vy, e.c.eta_c, e.c.eta_n, e.c.bx, e.c.by, e.c.inv_dx, e.c.inv_dy};
        const int widths[8] = {g.nx + 1, g.nx, g.nx, g.nx + 1, g.nx + 1, g.nx, g.nx + 1, g.nx};
        const int heights[8] = {g.ny, g.ny + 1, g.ny, g.ny + 1, g.ny, g.ny + 1, g.ny, g.ny + 1};
        std::memset(&m[i], 0, sizeof(TmaMaps));
        for (int f = 0; f < NF; ++f) {
            const cudaError_t r =
                make_tmap_2d(&m[i].m[f], ptrs[f], es, widths[f], heights[f], (long)g.pitch * es, p.bw, p.wym);
            if (r != cudaSuccess) return r;
        }
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_ras_batched(const BatchTiles<T> *tab, const int *tmap, const void *maps, int count, int total,
                               int ti, int tj, int ksweeps, int overlap, T omega, const int *live, const RasRun &run,
                               bool square, cudaStream_t s)
{
    // launch shape sized for the largest window (tile ti x tj grown by the
    // overlap): TMA staging through per-instance tensor maps when `maps` is
    // given (the FP32 pair layout for windows it takes, in its square-cell
    // form when every instance has square cells), else the register layout
    // reading global memory, else the general kernel with one CTA per tile
    const RasPlan p = plan_ras(ti, tj, ti, tj, overlap, sizeof(T), maps != nullptr, maps ? run.pair_mode : 0);
    if (p.smem > (size_t)ras_max_smem()) return cudaErrorInvalidValue;
    if (maps && p.kind != PLAN_TMA && p.kind != PLAN_PAIR) return cudaErrorInvalidValue;
    RasArgs<T> a{};
    a.omega = omega;
    a.ks = ksweeps;
    a.overlap = overlap;
    a.wxm = p.wxm;
    a.wym = p.wym;
    a.strips = p.strips;
    a.wp = p.wp;
    a.spad = p.spad;
    a.plane = p.plane;
    a.bw = p.bw;
    a.stage = p.stage;
    a.status = run.status;
    a.wait_limit = run.wait_limit;
    if (total <= 0) return cudaSuccess;
    cudaError_t e;
    if constexpr (sizeof(T) == 4) {
        if (p.kind == PLAN_PAIR) {
            // one staging buffer beside the edge rows
            const size_t one = (size_t)8 * (size_t)p.stage * sizeof(float);
            const size_t smem =
                one + (size_t)2 * PAIR_EDGE_KINDS * pair_edge_stride(p.threads <= PAIR_SMALL_THREADS ? PAIR_SMALL_THREADS : PAIR_MAX_THREADS) * 32 * sizeof(f2) + 128;
            void (*kern)(const BatchTiles<float> *, const int *, const TmaMaps *, int, int, const int *,
                         RasArgs<float>);
            if (square) kern = p.threads <= PAIR_SMALL_THREADS ? k_ras_batched_pair<PAIR_SMALL_THREADS, true> : k_ras_batched_pair<PAIR_MAX_THREADS, true>;
            else kern = p.threads <= PAIR_SMALL_THREADS ? k_ras_batched_pair<PAIR_SMALL_THREADS, false> : k_ras_batched_pair<PAIR_MAX_THREADS, false>;
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            const int grid = std::min(total, sm_count());
            kern<<<grid, p.threads, smem, s>>>(tab, tmap, reinterpret_cast<const TmaMaps *>(maps), count, total, live,
                                               a);
            return cudaGetLastError();
        }
    }
    if (p.kind == PLAN_TMA) {
        void (*kern)(const BatchTiles<T> *, const int *, const TmaMaps *, int, int, const int *, RasArgs<T>) =
            pick_batched_tma<T>(p);
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, p.threads, p.smem);
        if (e != cudaSuccess) return e;
        const int grid = std::min(total, std::max(per_sm, 1) * sm_count());
        kern<<<grid, p.threads, p.smem, s>>>(tab, tmap, reinterpret_cast<const TmaMaps *>(maps), count, total, live,
                                             a);
        return cudaGetLastError();
    }
    if (p.kind == PLAN_SMEM) {
        e = cudaFuncSetAttribute(k_ras_batched_smem<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
        if (e != cudaSuccess) return e;
        k_ras_batched_smem<T><<<total, RAS_THREADS, p.smem, s>>>(tab, tmap, count, live, a);
        return cudaGetLastError();
    }
    e = cudaFuncSetAttribute(k_ras_batched<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ras_batched<T>, p.threads, p.smem);
    if (e != cudaSuccess) return e;
    const int grid = std::min(total, std::max(per_sm, 1) * sm_count());
    k_ras_batched<T><<<grid, p.threads, p.smem, s>>>(tab, tmap, count, total, live, a);
    return cudaGetLastError();
}

template cudaError_t launch_ras_batched<float>(const BatchTiles<float> *, const int *, const void *, int, int, int,
                                               int, int, int, float, const int *, const RasRun &, bool, cudaStream_t);
template cudaError_t launch_ras_batched<double>(const BatchTiles<double> *, const int *, const void *, int, int, int,
                                                int, int, int, double, const int *, const RasRun &, bool,
                                                cudaStream_t);
template cudaError_t ras_batched_encode<float>(const BatchTiles<float> *, int, int, int, int, int, void *);
template cudaError_t ras_batched_encode<double>(const BatchTiles<double> *, int, int, int, int, int, void *);

template cudaError_t launch_ras<float>(const GridDesc<float> &, const Coeffs<float> &, float, const TileGrid &, int,
                                       int, const float *, const float *, float *, float *, const RasRun &,
                                       cudaStream_t);
template cudaError_t launch_ras<double>(const GridDesc<double> &, const Coeffs<double> &, double, const TileGrid &,
                                        int, int, const double *, const double *, double *, double *, const RasRun &,
                                        cudaStream_t);

} // namespace stokes
