// stencil_kernels.cu -- global-memory kernels of libstokes: copies, right-hand
// side, operator apply and the energy residual norm (the Jacobi and
// Gauss-Seidel sweeps are in sweep_kernels.cu).
//
// The operator is the flux form of Eq. (1)-(3) of arXiv 2509.19061 on the
// fully staggered grid of Sec. 2.1: deviatoric stresses at cell centres
// (sigma'_xx, sigma'_yy) and nodes (sigma'_xy), their divided differences at
// the velocity points.  Every field is a (ny+1) x pitch array; the library's
// copy of eta_n holds zero on boundary nodes, which makes the shear stress
// vanish there (free slip) without a branch.
#include "internal.h"
#include "stencil.cuh"
#include "gstencil.cuh"

namespace stokes {

namespace {

constexpr int BX = 32, BY = 8;

inline dim3 grid2d(int w, int h) { return dim3((unsigned)((w + BX - 1) / BX), (unsigned)((h + BY - 1) / BY)); }

// ---------------------------------------------------------------------------
// The per-cell setup kernels below give each thread EL_ROWS rows of one
// column (a warp reads 32 consecutive entries of a row per field), so that
// enough bytes are in flight to approach the HBM bandwidth.
constexpr int EL_ROWS = 4;

inline dim3 grid_rows(int w, int h)
{
    return dim3((unsigned)((w + BX - 1) / BX), (unsigned)((h + BY * EL_ROWS - 1) / (BY * EL_ROWS)));
}

template <typename T>
__global__ void k_copy_eta(GridDesc<T> g, const T *__restrict__ ec_in, const T *__restrict__ en_in,
                           T *__restrict__ ec, T *__restrict__ en)
{
    const int i = blockIdx.x * BX + threadIdx.x, j0 = (blockIdx.y * BY + threadIdx.y) * EL_ROWS;
    if (i > g.nx) return;
#pragma unroll
    for (int r = 0; r < EL_ROWS; ++r) {
        const int j = j0 + r;
        if (j > g.ny) break;
        const size_t q = (size_t)j * g.pitch + i;
        if (i < g.nx && j < g.ny) ec[q] = ec_in[q];
        const bool interior = i >= 1 && i <= g.nx - 1 && j >= 1 && j <= g.ny - 1;
        en[q] = interior ? en_in[q] : T(0);
    }
}

// 1 / diag(M) at the unknowns, zero elsewhere
template <typename T>
__global__ void k_inv_diag(GridDesc<T> g, const T *__restrict__ ec, const T *__restrict__ en, T *__restrict__ ix,
                           T *__restrict__ iy)
{
    const int i = blockIdx.x * BX + threadIdx.x, j0 = (blockIdx.y * BY + threadIdx.y) * EL_ROWS;
    if (i > g.nx) return;
    const size_t P = (size_t)g.pitch;
#pragma unroll
    for (int r = 0; r < EL_ROWS; ++r) {
        const int j = j0 + r;
        if (j > g.ny) break;
        const size_t q = (size_t)j * P + i;
        if (j < g.ny) ix[q] = vx_unknown(g, j, i) ? inv_diag(diag_x(g, ec[q], ec[q - 1], en[q + P], en[q])) : T(0);
        if (i < g.nx) iy[q] = vy_unknown(g, j, i) ? inv_diag(diag_y(g, ec[q], ec[q - P], en[q + 1], en[q])) : T(0);
    }
}

// k_copy_eta and k_inv_diag in one pass: the copies of eta_c (cells) and
// eta_n (zero on boundary nodes), and 1/diag(M) formed from the inputs with
// the same masking, so the values equal those of the two kernels bit for
// bit.  Every load of a thread's rows is issued before the first store.
template <typename T>
__global__ void k_set_eta(GridDesc<T> g, const T *__restrict__ ec_in, const T *__restrict__ en_in,
                          T *__restrict__ ec, T *__restrict__ en, T *__restrict__ ix, T *__restrict__ iy)
{
    const int i = blockIdx.x * BX + threadIdx.x, j0 = (blockIdx.y * BY + threadIdx.y) * EL_ROWS;
    if (i > g.nx) return;
    const size_t P = (size_t)g.pitch;
    auto cell = [&](int j, int c) -> T { return (c >= 0 && c < g.nx && j >= 0 && j < g.ny) ? ec_in[(size_t)j * P + c] : T(0); };
    auto node = [&](int j, int c) -> T {
        return (c >= 1 && c <= g.nx - 1 && j >= 1 && j <= g.ny - 1) ? en_in[(size_t)j * P + c] : T(0);
    };
    T ecs[EL_ROWS + 1], enr[EL_ROWS + 1], ecw[EL_ROWS], ene[EL_ROWS]; // eta_c rows j0 - 1 .., eta_n rows j0 ..
#pragma unroll
    for (int r = 0; r <= EL_ROWS; ++r) {
        ecs[r] = cell(j0 - 1 + r, i);
        enr[r] = node(j0 + r, i);
    }
#pragma unroll
    for (int r = 0; r < EL_ROWS; ++r) {
        ecw[r] = cell(j0 + r, i - 1);
        ene[r] = node(j0 + r, i + 1);
    }
#pragma unroll
    for (int r = 0; r < EL_ROWS; ++r) {
        const int j = j0 + r;
        if (j > g.ny) break;
        const size_t q = (size_t)j * P + i;
        const T ecC = ecs[r + 1], enC = enr[r];
        if (i < g.nx && j < g.ny) ec[q] = ecC;
        en[q] = enC;
        if (j < g.ny) ix[q] = vx_unknown(g, j, i) ? inv_diag(diag_x(g, ecC, ecw[r], enr[r + 1], enC)) : T(0);
        if (i < g.nx) iy[q] = vy_unknown(g, j, i) ? inv_diag(diag_y(g, ecC, ecs[r], ene[r], enC)) : T(0);
    }
}

// b = f - G p with (G p) = -grad p; zero on walls.  Every load of a thread's
// rows is issued before the first store.
template <typename T>
__global__ void k_rhs(GridDesc<T> g, const T *__restrict__ fx, const T *__restrict__ fy, const T *__restrict__ p,
                      T *__restrict__ bx, T *__restrict__ by)
{
    const int i = blockIdx.x * BX + threadIdx.x, j0 = (blockIdx.y * BY + threadIdx.y) * EL_ROWS;
    if (i > g.nx) return;
    const size_t P = (size_t)g.pitch;
    T fxr[EL_ROWS], fyr[EL_ROWS], pc[EL_ROWS], pw[EL_ROWS], ps[EL_ROWS];
#pragma unroll
    for (int r = 0; r < EL_ROWS; ++r) {
        const int j = j0 + r;
        const size_t q = (size_t)j * P + i;
        const bool ux = vx_unknown(g, j, i), uy = vy_unknown(g, j, i);
        fxr[r] = ux ? fx[q] : T(0);
        fyr[r] = uy ? fy[q] : T(0);
        pc[r] = (p && (ux || uy)) ? p[q] : T(0);
        pw[r] = (p && ux) ? p[q - 1] : T(0);
        ps[r] = (p && uy) ? p[q - P] : T(0);
    }
#pragma unroll
    for (int r = 0; r < EL_ROWS; ++r) {
        const int j = j0 + r;
        if (j > g.ny) break;
        const size_t q = (size_t)j * P + i;
        if (j < g.ny) {
            T b = T(0);
            if (vx_unknown(g, j, i)) b = p ? r_fma(r_sub(pc[r], pw[r]), g.ihx, fxr[r]) : fxr[r];
            bx[q] = b;
        }
        if (i < g.nx) {
            T b = T(0);
            if (vy_unknown(g, j, i)) b = p ? r_fma(r_sub(pc[r], ps[r]), g.ihy, fyr[r]) : fyr[r];
            by[q] = b;
        }
    }
}

// out = M v + G p at unknowns; zero on walls and padding.
template <typename T>
__global__ void k_apply(GridDesc<T> g, const T *__restrict__ eta_c, const T *__restrict__ eta_n,
                        const T *__restrict__ vx, const T *__restrict__ vy, const T *__restrict__ p,
                        T *__restrict__ ox, T *__restrict__ oy)
{
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    if (i >= g.pitch || j > g.ny) return;
    const size_t P = (size_t)g.pitch, q = (size_t)j * P + i;
    T m, d, vc;
    T rx = T(0), ry = T(0);
    if (vx_unknown(g, j, i)) {
        op_x(g, eta_c, eta_n, vx, vy, j, i, m, d, vc);
        rx = m - (p ? (p[q] - p[q - 1]) * g.ihx : T(0));
    }
    if (vy_unknown(g, j, i)) {
        op_y(g, eta_c, eta_n, vx, vy, j, i, m, d, vc);
        ry = m - (p ? (p[q] - p[q - P]) * g.ihy : T(0));
    }
    ox[q] = rx;
    oy[q] = ry;
}

template <typename T>
__global__ void k_copy_velocity(GridDesc<T> g, const T *__restrict__ vx, const T *__restrict__ vy,
                                T *__restrict__ ox, T *__restrict__ oy)
{
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    if (i > g.nx || j > g.ny) return;
    const size_t q = (size_t)j * g.pitch + i;
    if (j < g.ny) ox[q] = vx[q];
    if (i < g.nx) oy[q] = vy[q];
}

template <typename T>
__global__ void k_copy_walls(GridDesc<T> g, const T *__restrict__ vx, const T *__restrict__ vy, T *__restrict__ ox,
                             T *__restrict__ oy)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const size_t P = (size_t)g.pitch;
    if (t < g.ny) { // vx walls of row t
        ox[t * P] = vx[t * P];
        ox[t * P + g.nx] = vx[t * P + g.nx];
    }
    if (t < g.nx) { // vy walls of column t
        oy[t] = vy[t];
        oy[(size_t)g.ny * P + t] = vy[(size_t)g.ny * P + t];
    }
}

// ---------------------------------------------------------------------------
// energy norm, Sec. 6.4 (FP64 accumulation, fixed reduction order)
constexpr int EN_THREADS = 256;
constexpr int EN_BLOCKS = 152 * 4;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Compensated FP32 sum (Knuth's TwoSum: the rounding error of every addition
// is carried in lo), for the FP32 terms of one row of cells; added to an FP64
// sum once per row, which keeps the FP64 pipe (1/64 of the FP32 rate on this
// GPU) out of the per-cell work.  The error of hi + lo is of the order of
// 2^-44 of the row sum, far below the 2^-24 rounding of each FP32 term.
struct CompF {
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

// The FP32 energy sums: per cell the terms of CellSq<float> (a cell's vx and vy
// terms added in FP32), per row a compensated FP32 sum, per thread an FP64 sum.
template <bool MASK, int SQM>
__device__ __forceinline__ void energy_rows_f32(const GridDesc<float> &g, const float *__restrict__ eta_c,
                                                const float *__restrict__ eta_n, const float *__restrict__ inv_dx,
                                                const float *__restrict__ inv_dy, const float *__restrict__ fx,
                                                const float *__restrict__ fy, const float *__restrict__ p,
                                                const float *__restrict__ vx, const float *__restrict__ vy,
                                                double &s_rv, double &s_rp, double &s_ff)
{
    const float ilap = (float)(1.0 / g.lap);
    for (int j = blockIdx.x; j <= g.ny; j += gridDim.x) {
        CompF rv, rp, ff;
        for (int i = threadIdx.x; i <= g.nx; i += EN_THREADS) {
            const size_t q = (size_t)j * g.pitch + i;
            float m, d, vc;
            float trv = 0.f, tff = 0.f;
            bool any = false;
            if (vx_unknown(g, j, i)) {
                op_x<float, MASK, SQM>(g, eta_c, eta_n, vx, vy, j, i, m, d, vc);
                const float b = p ? r_fma(r_sub(p[q], p[q - 1]), g.ihx, fx[q]) : fx[q];
                const float wi = -(inv_dx ? inv_dx[q] : inv_diag(d));
                const float r = r_sub(b, m);
                trv = r_mul(r_mul(r, r), wi);
                tff = r_mul(r_mul(fx[q], fx[q]), wi);
                any = true;
            }
            if (vy_unknown(g, j, i)) {
                op_y<float, MASK, SQM>(g, eta_c, eta_n, vx, vy, j, i, m, d, vc);
                const float b = p ? r_fma(r_sub(p[q], p[q - g.pitch]), g.ihy, fy[q]) : fy[q];
                const float wi = -(inv_dy ? inv_dy[q] : inv_diag(d));
                const float r = r_sub(b, m);
                const float a = r_mul(r_mul(r, r), wi), c = r_mul(r_mul(fy[q], fy[q]), wi);
                trv = any ? r_add(trv, a) : a;
                tff = any ? r_add(tff, c) : c;
                any = true;
            }
            if (any) {
                rv.add(trv);
                ff.add(tff);
            }
            if (i < g.nx && j < g.ny) {
                const float dv = r_fma(r_sub(vx[q + 1], vx[q]), g.ihx, r_mul(r_sub(vy[q + g.pitch], vy[q]), g.ihy));
                rp.add(r_mul(r_mul(dv, dv), r_mul(eta_c[q], ilap)));
            }
        }
        rv.flush(s_rv);
        rp.flush(s_rp);
        ff.flush(s_ff);
    }
}

// Per-thread accumulation of the energy terms: FP64 fma per term (FP64
// contexts, as CellSq<double>), compensated FP32 sums flushed to FP64 once
// (FP32 contexts).
template <typename T>
struct EnergyAcc;
template <>
struct EnergyAcc<double> {
    double rv = 0.0, rp = 0.0, ff = 0.0;
    __device__ __forceinline__ void add_v(double r, double f, double w)
    {
        rv = fma(r * r, w, rv);
        ff = fma(f * f, w, ff);
    }
    __device__ __forceinline__ void add_p(double dv, double w) { rp = fma(dv * dv, w, rp); }
    __device__ __forceinline__ void done(double &a, double &b, double &c) { a = rv; b = rp; c = ff; }
};
template <>
struct EnergyAcc<float> {
    CompF rv, rp, ff;
    float trv = 0.f, tff = 0.f;
    bool any = false;
    // the cell's vx and vy terms are added in FP32 first (as CellSq<float>)
    __device__ __forceinline__ void add_v(float r, float f, float w)
    {
        const float a = r_mul(r_mul(r, r), w), c = r_mul(r_mul(f, f), w);
        trv = any ? r_add(trv, a) : a;
        tff = any ? r_add(tff, c) : c;
        any = true;
    }
    __device__ __forceinline__ void end_cell()
    {
        if (any) {
            rv.add(trv);
            ff.add(tff);
        }
        any = false;
    }
    __device__ __forceinline__ void add_p(float dv, float w) { rp.add(r_mul(r_mul(dv, dv), w)); }
    __device__ __forceinline__ void done(double &a, double &b, double &c)
    {
        rv.flush(a);
        rp.flush(b);
        ff.flush(c);
    }
};

// Energy sums tile by tile (32 x 8 cells): the fluxes of M v are staged once
// per tile in shared memory (flux_tile_stage, the bits of op_x / op_y), the
// residual b - M v and its terms formed per unknown.  Library viscosity
// copies (eta_n zero on boundary nodes); 1/diag(M) from the context's arrays
// when given.
template <typename T>
__global__ void __launch_bounds__(EN_THREADS) k_energy_tile(GridDesc<T> g, const T *__restrict__ eta_c,
                                                            const T *__restrict__ eta_n, const T *__restrict__ inv_dx,
                                                            const T *__restrict__ inv_dy, const T *__restrict__ fx,
                                                            const T *__restrict__ fy, const T *__restrict__ p,
                                                            const T *__restrict__ vx, const T *__restrict__ vy,
                                                            double *__restrict__ partials)
{
    static_assert(AT_X * AT_Y == EN_THREADS, "one thread per tile cell");
    __shared__ ApplyTile<T> sm;
    const T ilap = (T)(1.0 / g.lap);
    const size_t P = (size_t)g.pitch;
    const int tid = (int)threadIdx.x, tx = tid % AT_X, ty = tid / AT_X;
    const int ntx = (g.nx + 1 + AT_X - 1) / AT_X, nty = (g.ny + 1 + AT_Y - 1) / AT_Y;
    EnergyAcc<T> acc;
    for (int t = blockIdx.x; t < ntx * nty; t += gridDim.x) {
        const int i0 = (t % ntx) * AT_X, j0 = (t / ntx) * AT_Y;
        flux_tile_stage<T>(g, eta_c, eta_n, nullptr, nullptr, vx, vy, i0, j0, tid, sm);
        const int j = j0 + ty, i = i0 + tx;
        const size_t q = (size_t)j * P + i;
        if (vx_unknown(g, j, i)) {
            const T m = m_x(sm.txx[ty][tx + 1], sm.txx[ty][tx], sm.sx[ty + 1][tx], sm.sx[ty][tx]);
            const T b = p ? r_fma(r_sub(p[q], p[q - 1]), g.ihx, fx[q]) : fx[q];
            const T wi = -(inv_dx ? inv_dx[q] : inv_diag(diag_x(g, eta_c[q], eta_c[q - 1], eta_n[q + P], eta_n[q])));
            acc.add_v(r_sub(b, m), fx[q], wi);
        }
        if (vy_unknown(g, j, i)) {
            const T m = m_y(sm.sy[ty][tx + 1], sm.sy[ty][tx], sm.tyy[ty + 1][tx], sm.tyy[ty][tx]);
            const T b = p ? r_fma(r_sub(p[q], p[q - P]), g.ihy, fy[q]) : fy[q];
            const T wi = -(inv_dy ? inv_dy[q] : inv_diag(diag_y(g, eta_c[q], eta_c[q - P], eta_n[q + 1], eta_n[q])));
            acc.add_v(r_sub(b, m), fy[q], wi);
        }
        if constexpr (sizeof(T) == 4) acc.end_cell();
        if (i < g.nx && j < g.ny) {
            const T dv = r_fma(r_sub(vx[q + 1], vx[q]), g.ihx, r_mul(r_sub(vy[q + P], vy[q]), g.ihy));
            acc.add_p(dv, r_mul(eta_c[q], ilap));
        }
        __syncthreads(); // the tile's shared fluxes are read before the next tile overwrites them
    }
    double s_rv = 0.0, s_rp = 0.0, s_ff = 0.0;
    acc.done(s_rv, s_rp, s_ff);
    __shared__ double sh[3][EN_THREADS / 32];
    s_rv = warp_sum(s_rv);
    s_rp = warp_sum(s_rp);
    s_ff = warp_sum(s_ff);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][wid] = s_rv;
        sh[1][wid] = s_rp;
        sh[2][wid] = s_ff;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double s = 0.0;
        for (int w = 0; w < EN_THREADS / 32; ++w) s += sh[threadIdx.x][w];
        partials[(size_t)blockIdx.x * 3 + threadIdx.x] = s;
    }
}

template <typename T, bool MASK = false, int SQM = 2>
__global__ void __launch_bounds__(EN_THREADS) k_energy(GridDesc<T> g, const T *__restrict__ eta_c,
                                                       const T *__restrict__ eta_n, const T *__restrict__ inv_dx,
                                                       const T *__restrict__ inv_dy, const T *__restrict__ fx,
                                                       const T *__restrict__ fy, const T *__restrict__ p,
                                                       const T *__restrict__ vx, const T *__restrict__ vy,
                                                       double *__restrict__ partials)
{
    // r_v = f - G p - M v with b = f - G p formed on the fly; the weights
    // 1/(-diag M) come from the context's 1/diag arrays when it has them
    double s_rv = 0.0, s_rp = 0.0, s_ff = 0.0;
    const T ilap = (T)(1.0 / g.lap);
    // rows round-robin over the blocks, columns over the threads (no index division)
    if constexpr (sizeof(T) == 4)
        energy_rows_f32<MASK, SQM>(g, eta_c, eta_n, inv_dx, inv_dy, fx, fy, p, vx, vy, s_rv, s_rp, s_ff);
    else
    for (int j = blockIdx.x; j <= g.ny; j += gridDim.x)
    for (int i = threadIdx.x; i <= g.nx; i += EN_THREADS) {
        const size_t q = (size_t)j * g.pitch + i;
        T m, d, vc;
        CellSq<T> rv(s_rv), ff(s_ff); // the cell's vx and vy terms
        if (vx_unknown(g, j, i)) {
            op_x<T, MASK, SQM>(g, eta_c, eta_n, vx, vy, j, i, m, d, vc);
            const T b = p ? r_fma(r_sub(p[q], p[q - 1]), g.ihx, fx[q]) : fx[q];
            const T wi = -(inv_dx ? inv_dx[q] : inv_diag(d));
            rv.add(r_sub(b, m), wi);
            ff.add(fx[q], wi);
        }
        if (vy_unknown(g, j, i)) {
            op_y<T, MASK, SQM>(g, eta_c, eta_n, vx, vy, j, i, m, d, vc);
            const T b = p ? r_fma(r_sub(p[q], p[q - g.pitch]), g.ihy, fy[q]) : fy[q];
            const T wi = -(inv_dy ? inv_dy[q] : inv_diag(d));
            rv.add(r_sub(b, m), wi);
            ff.add(fy[q], wi);
        }
        rv.done();
        ff.done();
        if (i < g.nx && j < g.ny) {
            const T dv = r_fma(r_sub(vx[q + 1], vx[q]), g.ihx, r_mul(r_sub(vy[q + g.pitch], vy[q]), g.ihy));
            s_rp = acc_sq(s_rp, dv, r_mul(eta_c[q], ilap));
        }
    }
    __shared__ double sh[3][EN_THREADS / 32];
    s_rv = warp_sum(s_rv);
    s_rp = warp_sum(s_rp);
    s_ff = warp_sum(s_ff);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][wid] = s_rv;
        sh[1][wid] = s_rp;
        sh[2][wid] = s_ff;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double s = 0.0;
        for (int q = 0; q < EN_THREADS / 32; ++q) s += sh[threadIdx.x][q];
        partials[(size_t)blockIdx.x * 3 + threadIdx.x] = s;
    }
}

__global__ void k_energy_final(const double *__restrict__ partials, int nblocks, double *__restrict__ out)
{
    // one warp per component, fixed order
    const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double s = 0.0;
    for (int b = lane; b < nblocks; b += 32) s += partials[(size_t)b * 3 + c];
    s = warp_sum(s);
    if (lane == 0) out[c] = s;
}

} // namespace

// ---------------------------------------------------------------------------
// launchers
template <typename T>
cudaError_t launch_copy_eta(const GridDesc<T> &g, const T *eta_c_in, const T *eta_n_in, T *eta_c, T *eta_n,
                            cudaStream_t s)
{
    k_copy_eta<T><<<grid_rows(g.nx + 1, g.ny + 1), dim3(BX, BY), 0, s>>>(g, eta_c_in, eta_n_in, eta_c, eta_n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_set_eta(const GridDesc<T> &g, const T *eta_c_in, const T *eta_n_in, T *eta_c, T *eta_n, T *inv_dx,
                           T *inv_dy, cudaStream_t s)
{
    k_set_eta<T><<<grid_rows(g.nx + 1, g.ny + 1), dim3(BX, BY), 0, s>>>(g, eta_c_in, eta_n_in, eta_c, eta_n, inv_dx,
                                                                        inv_dy);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_inv_diag(const GridDesc<T> &g, const T *eta_c, const T *eta_n, T *inv_dx, T *inv_dy,
                            cudaStream_t s)
{
    k_inv_diag<T><<<grid_rows(g.nx + 1, g.ny + 1), dim3(BX, BY), 0, s>>>(g, eta_c, eta_n, inv_dx, inv_dy);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rhs(const GridDesc<T> &g, const T *fx, const T *fy, const T *p, T *bx, T *by, cudaStream_t s)
{
    k_rhs<T><<<grid_rows(g.nx + 1, g.ny + 1), dim3(BX, BY), 0, s>>>(g, fx, fy, p, bx, by);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_apply(const GridDesc<T> &g, const T *eta_c, const T *eta_n, const T *vx, const T *vy, const T *p,
                         T *ox, T *oy, cudaStream_t s)
{
    k_apply<T><<<grid2d(g.pitch, g.ny + 1), dim3(BX, BY), 0, s>>>(g, eta_c, eta_n, vx, vy, p, ox, oy);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_copy_velocity(const GridDesc<T> &g, const T *vx, const T *vy, T *ox, T *oy, cudaStream_t s)
{
    k_copy_velocity<T><<<grid2d(g.nx + 1, g.ny + 1), dim3(BX, BY), 0, s>>>(g, vx, vy, ox, oy);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_copy_walls(const GridDesc<T> &g, const T *vx, const T *vy, T *ox, T *oy, cudaStream_t s)
{
    const int n = (g.nx > g.ny ? g.nx : g.ny);
    k_copy_walls<T><<<(n + 255) / 256, 256, 0, s>>>(g, vx, vy, ox, oy);
    return cudaGetLastError();
}

int energy_partials() { return EN_BLOCKS; }

template <typename T>
cudaError_t launch_energy(const GridDesc<T> &g, const T *eta_c, const T *eta_n, const T *inv_dx, const T *inv_dy,
                          const T *fx, const T *fy, const T *p, const T *vx, const T *vy, double *partials,
                          double *out, cudaStream_t s)
{
    // FP64: the FP64 pipe is the bound, and the tiled kernel forms every flux
    // once (6.1 instead of 9.7 ms at 8192^2); FP32: row-marching warps that
    // read every field once (`sweep_kernels.cu`)
    int nb = EN_BLOCKS;
    if constexpr (sizeof(T) == 8) {
        k_energy_tile<T><<<EN_BLOCKS, EN_THREADS, 0, s>>>(g, eta_c, eta_n, inv_dx, inv_dy, fx, fy, p, vx, vy,
                                                          partials);
    } else {
        // (forming 1/diag from the viscosity instead of reading it made this
        // kernel slower: 0.566 against 0.481 ms at 8192^2)
        const cudaError_t e = launch_energy_rows(g, eta_c, eta_n, fx, fy, inv_dx, inv_dy, p, vx, vy, partials, &nb, s);
        if (e != cudaSuccess) return e;
    }
    k_energy_final<<<1, 96, 0, s>>>(partials, nb, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_energy_raw(const GridDesc<T> &g, const T *eta_c, const T *eta_n, const T *fx, const T *fy,
                              const T *p, const T *vx, const T *vy, double *partials, double *out, cudaStream_t s)
{
    k_energy<T, true, 0><<<EN_BLOCKS, EN_THREADS, 0, s>>>(g, eta_c, eta_n, nullptr, nullptr, fx, fy, p, vx, vy,
                                                          partials);
    k_energy_final<<<1, 96, 0, s>>>(partials, EN_BLOCKS, out);
    return cudaGetLastError();
}

#define INST(T)                                                                                                    \
    template cudaError_t launch_copy_eta<T>(const GridDesc<T> &, const T *, const T *, T *, T *, cudaStream_t);    \
    template cudaError_t launch_inv_diag<T>(const GridDesc<T> &, const T *, const T *, T *, T *, cudaStream_t);    \
    template cudaError_t launch_set_eta<T>(const GridDesc<T> &, const T *, const T *, T *, T *, T *, T *,          \
                                           cudaStream_t);                                                          \
    template cudaError_t launch_rhs<T>(const GridDesc<T> &, const T *, const T *, const T *, T *, T *,             \
                                       cudaStream_t);                                                              \
    template cudaError_t launch_apply<T>(const GridDesc<T> &, const T *, const T *, const T *, const T *,          \
                                         const T *, T *, T *, cudaStream_t);                                       \
    template cudaError_t launch_copy_velocity<T>(const GridDesc<T> &, const T *, const T *, T *, T *,              \
                                                 cudaStream_t);                                                    \
    template cudaError_t launch_copy_walls<T>(const GridDesc<T> &, const T *, const T *, T *, T *, cudaStream_t);  \
    template cudaError_t launch_energy<T>(const GridDesc<T> &, const T *, const T *, const T *, const T *,         \
                                          const T *, const T *, const T *, const T *, const T *, double *,         \
                                          double *, cudaStream_t);                                                 \
    template cudaError_t launch_energy_raw<T>(const GridDesc<T> &, const T *, const T *, const T *, const T *,     \
                                              const T *, const T *, const T *, double *, double *, cudaStream_t);
INST(float)
INST(double)
#undef INST

} // namespace stokes
