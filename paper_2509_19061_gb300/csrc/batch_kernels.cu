// batch_kernels.cu -- the multigrid level operations and the outer-solve
// vector operations for many independent instances in one launch each.
// Arithmetic per point is the single-instance arithmetic (gstencil.cuh,
// mg_point.cuh, stencil.cuh); per-instance sums are accumulated in FP64 in a
// fixed order.
#include "../../include/stokes.h"
#include "batch.h"
#include "gstencil.cuh"
#include "mg_point.cuh"
#include "stencil.cuh"

namespace stokes {

namespace {

constexpr int NT = BATCH_BX * BATCH_BY;

__device__ __forceinline__ int seg_of(const BSeg *__restrict__ m, int n, int b)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (m[mid].block_begin <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// point of this thread inside its instance's rectangle (valid = inside)
struct Pt {
    int inst, i, j;
    bool valid;
};

__device__ __forceinline__ Pt point_of(const BSeg *__restrict__ m, int n)
{
    const BSeg sg = m[seg_of(m, n, blockIdx.x)];
    const int lb = blockIdx.x - sg.block_begin;
    Pt p;
    p.inst = sg.inst;
    p.i = (lb % sg.bxb) * BATCH_BX + threadIdx.x;
    p.j = (lb / sg.bxb) * BATCH_BY + threadIdx.y;
    p.valid = p.i < sg.w && p.j < sg.h;
    return p;
}

// first point of this thread in a tall map (rows p.j + r BATCH_BY, r <
// BATCH_TALL); valid = the column lies inside the instance's rectangle, the
// rows are checked one by one
__device__ __forceinline__ Pt point_of_tall(const BSeg *__restrict__ m, int n, int &h)
{
    const BSeg sg = m[seg_of(m, n, blockIdx.x)];
    const int lb = blockIdx.x - sg.block_begin;
    Pt p;
    p.inst = sg.inst;
    p.i = (lb % sg.bxb) * BATCH_BX + threadIdx.x;
    p.j = (lb / sg.bxb) * BATCH_BY * BATCH_TALL + threadIdx.y;
    p.valid = p.i < sg.w;
    h = sg.h;
    return p;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void block_store2(double s0, double s1, double *partials)
{
    __shared__ double sh[2][NT / 32];
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    const int t = threadIdx.y * BATCH_BX + threadIdx.x, lane = t & 31, wid = t >> 5;
    if (lane == 0) {
        sh[0][wid] = s0;
        sh[1][wid] = s1;
    }
    __syncthreads();
    if (t < 2) {
        double s = 0.0;
        for (int q = 0; q < NT / 32; ++q) s += sh[t][q];
        partials[2 * blockIdx.x + t] = s;
    }
}

// per-instance totals of the block partials: one warp per segment
__global__ void k_seg_final(const BSeg *__restrict__ m, int n, const double *__restrict__ partials,
                            double *__restrict__ out)
{
    const int seg = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (seg >= n) return;
    const BSeg sg = m[seg];
    const int nb = sg.bxb * ((sg.h + BATCH_BY - 1) / BATCH_BY);
    double s0 = 0.0, s1 = 0.0;
    for (int b = lane; b < nb; b += 32) {
        s0 += partials[2 * (sg.block_begin + b)];
        s1 += partials[2 * (sg.block_begin + b) + 1];
    }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    if (lane == 0) {
        out[2 * sg.inst] = s0;
        out[2 * sg.inst + 1] = s1;
    }
}

template <typename T>
__global__ void kb_rhs(const BRhs<T> *__restrict__ tab, const BSeg *__restrict__ m, int n)
{
    int h;
    const Pt p = point_of_tall(m, n, h);
    if (!p.valid) return;
    const BRhs<T> &r = tab[p.inst];
    const GridDesc<T> &g = r.g;
    const int i = p.i;
    const size_t P = (size_t)g.pitch;
    // every row's loads first, then the stores
    T fxr[BATCH_TALL], fyr[BATCH_TALL], pc[BATCH_TALL], pw[BATCH_TALL], ps[BATCH_TALL];
#pragma unroll
    for (int t = 0; t < BATCH_TALL; ++t) {
        const int j = p.j + t * BATCH_BY;
        const size_t q = (size_t)j * P + i;
        const bool ux = j < h && vx_unknown(g, j, i), uy = j < h && vy_unknown(g, j, i);
        fxr[t] = ux ? r.fx[q] : T(0);
        fyr[t] = uy ? r.fy[q] : T(0);
        pc[t] = (r.p && (ux || uy)) ? r.p[q] : T(0);
        pw[t] = (r.p && ux) ? r.p[q - 1] : T(0);
        ps[t] = (r.p && uy) ? r.p[q - P] : T(0);
    }
#pragma unroll
    for (int t = 0; t < BATCH_TALL; ++t) {
        const int j = p.j + t * BATCH_BY;
        if (j >= h) break;
        const size_t q = (size_t)j * P + i;
        if (j < g.ny) {
            T b = T(0);
            if (vx_unknown(g, j, i)) b = r.p ? r_fma(r_sub(pc[t], pw[t]), g.ihx, fxr[t]) : fxr[t];
            r.bx[q] = b;
        }
        if (i < g.nx) {
            T b = T(0);
            if (vy_unknown(g, j, i)) b = r.p ? r_fma(r_sub(pc[t], ps[t]), g.ihy, fyr[t]) : fyr[t];
            r.by[q] = b;
        }
    }
}

// ---- level operations ----------------------------------------------------------
template <typename T>
__global__ void kb_residual(const BLevel<T> *__restrict__ tab, const BSeg *__restrict__ m, int n,
                            const int *__restrict__ active)
{
    const Pt p = point_of(m, n);
    if (!p.valid || (active && !active[p.inst])) return;
    const BLevel<T> &l = tab[p.inst];
    const GridDesc<T> &g = l.g;
    const int i = p.i, j = p.j;
    const size_t q = (size_t)j * g.pitch + i;
    T mm, d, vc;
    if (j < g.ny) {
        T r = T(0);
        if (vx_unknown(g, j, i)) {
            op_x(g, (const T *)l.ec, (const T *)l.en, (const T *)l.vx, (const T *)l.vy, j, i, mm, d, vc);
            r = r_sub(l.bx[q], mm);
        }
        l.rx[q] = r;
    }
    if (i < g.nx) {
        T r = T(0);
        if (vy_unknown(g, j, i)) {
            op_y(g, (const T *)l.ec, (const T *)l.en, (const T *)l.vx, (const T *)l.vy, j, i, mm, d, vc);
            r = r_sub(l.by[q], mm);
        }
        l.ry[q] = r;
    }
}

template <typename T>
__global__ void kb_restrict(const BLevel<T> *__restrict__ tab, const BSeg *__restrict__ m, int n,
                            const int *__restrict__ active)
{
    const Pt p = point_of(m, n);
    if (!p.valid || (active && !active[p.inst])) return;
    const BLevel<T> &l = tab[p.inst];
    restrict_point(l.g.nx, l.g.ny, l.g.pitch, l.cnx, l.cny, l.cp, (const T *)l.rx, (const T *)l.ry, l.cbx, l.cby,
                   p.j, p.i);
}

template <typename T>
__global__ void kb_prolong(const BLevel<T> *__restrict__ tab, const BSeg *__restrict__ m, int n,
                            const int *__restrict__ active)
{
    const Pt p = point_of(m, n);
    if (!p.valid || (active && !active[p.inst])) return;
    const BLevel<T> &l = tab[p.inst];
    prolong_point(l.g.nx, l.g.ny, l.g.pitch, l.cnx, l.cny, l.cp, (const T *)l.cvx, (const T *)l.cvy, l.vx, l.vy,
                  p.j, p.i);
}

template <typename T>
__global__ void kb_zero_v(const BLevel<T> *__restrict__ tab, const BSeg *__restrict__ m, int n,
                            const int *__restrict__ active)
{
    const Pt p = point_of(m, n);
    if (!p.valid || (active && !active[p.inst])) return;
    const BLevel<T> &l = tab[p.inst];
    const size_t q = (size_t)p.j * l.g.pitch + p.i;
    l.vx[q] = T(0);
    l.vy[q] = T(0);
}

template <typename T>
__global__ void kb_copy(const BLevel<T> *__restrict__ tab, const BSeg *__restrict__ m, int n, bool to_scratch,
                        const int *__restrict__ active)
{
    int h;
    const Pt p = point_of_tall(m, n, h);
    if (!p.valid || (active && !active[p.inst])) return;
    const BLevel<T> &l = tab[p.inst];
    const GridDesc<T> &g = l.g;
    const int i = p.i;
    T *sx = to_scratch ? l.sx : l.vx, *sy = to_scratch ? l.sy : l.vy;
    const T *ax = to_scratch ? l.vx : l.sx, *ay = to_scratch ? l.vy : l.sy;
    T cx[BATCH_TALL], cy[BATCH_TALL];
#pragma unroll
    for (int t = 0; t < BATCH_TALL; ++t) {
        const int j = p.j + t * BATCH_BY;
        const size_t q = (size_t)j * g.pitch + i;
        cx[t] = (j < h && j < g.ny) ? ax[q] : T(0);
        cy[t] = (j < h && i < g.nx) ? ay[q] : T(0);
    }
#pragma unroll
    for (int t = 0; t < BATCH_TALL; ++t) {
        const int j = p.j + t * BATCH_BY;
        if (j >= h) break;
        const size_t q = (size_t)j * g.pitch + i;
        if (j < g.ny) sx[q] = cx[t];
        if (i < g.nx) sy[q] = cy[t];
    }
}

// the wall entries of one instance per block: vx at i = 0 and nx, vy at j = 0 and ny
template <typename T>
__global__ void kb_copy_walls(const BLevel<T> *__restrict__ tab, const BSeg *__restrict__ m,
                              const int *__restrict__ active)
{
    const int inst = m[blockIdx.x].inst;
    if (active && !active[inst]) return;
    const BLevel<T> &l = tab[inst];
    const GridDesc<T> &g = l.g;
    const size_t P = (size_t)g.pitch;
    const int nwx = 2 * g.ny, nwy = 2 * g.nx;
    for (int t = (int)threadIdx.x; t < nwx + nwy; t += (int)blockDim.x) {
        if (t < nwx) {
            const size_t q = (size_t)(t >> 1) * P + ((t & 1) ? g.nx : 0);
            l.sx[q] = l.vx[q];
        } else {
            const int u = t - nwx;
            const size_t q = (size_t)((u & 1) ? g.ny : 0) * P + (u >> 1);
            l.sy[q] = l.vy[q];
        }
    }
}

template <typename T>
__device__ __forceinline__ int dense_of(const BDense<T> *__restrict__ tab, int count, int u)
{
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tab[mid].unk_begin <= u) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// unknown u of an nx x ny grid: vx unknowns row-major, then vy unknowns
__device__ __forceinline__ void unk_pos(int u, int nx, int ny, int &comp, int &j, int &i)
{
    const int nvx = ny * (nx - 1);
    if (u < nvx) {
        comp = 0;
        j = u / (nx - 1);
        i = u - j * (nx - 1) + 1;
    } else {
        u -= nvx;
        comp = 1;
        j = u / nx + 1;
        i = u - (j - 1) * nx;
    }
}

template <typename T>
__global__ void kb_dense_pack(const BDense<T> *__restrict__ tab, int count, int rows,
                                const int *__restrict__ active)
{
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= rows) return;
    const int di = dense_of(tab, count, u);
    if (active && !active[di]) return;
    const BDense<T> &d = tab[di];
    int comp, j, i;
    unk_pos(u - d.unk_begin, d.nx, d.ny, comp, j, i);
    d.bvec[u - d.unk_begin] = (double)(comp == 0 ? d.bx : d.by)[(size_t)j * d.pitch + i];
}

template <typename T>
__global__ void kb_dense_solve(const BDense<T> *__restrict__ tab, int count, int rows,
                                const int *__restrict__ active)
{
    const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (row >= rows) return;
    const int di = dense_of(tab, count, row);
    if (active && !active[di]) return;
    const BDense<T> &d = tab[di];
    const int r = row - d.unk_begin;
    double s = 0.0;
    for (int c = lane; c < d.n; c += 32) s += d.Ainv[(size_t)r * d.n + c] * d.bvec[c];
    s = warp_sum(s);
    if (lane == 0) d.xvec[r] = -s;
}

template <typename T>
__global__ void kb_dense_unpack(const BDense<T> *__restrict__ tab, int count, int rows,
                                const int *__restrict__ active)
{
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= rows) return;
    const int di = dense_of(tab, count, u);
    if (active && !active[di]) return;
    const BDense<T> &d = tab[di];
    int comp, j, i;
    unk_pos(u - d.unk_begin, d.nx, d.ny, comp, j, i);
    (comp == 0 ? d.vx : d.vy)[(size_t)j * d.pitch + i] = (T)d.xvec[u - d.unk_begin];
}

template <typename To, typename Ti>
__global__ void kb_cast_in(const BOuter<To> *__restrict__ out, const BLevel<Ti> *__restrict__ l0,
                           const BSeg *__restrict__ m, int n, const int *__restrict__ active)
{
    const Pt p = point_of(m, n);
    if (!p.valid || (active && !active[p.inst])) return;
    const size_t q = (size_t)p.j * l0[p.inst].g.pitch + p.i;
    l0[p.inst].bx[q] = (Ti)out[p.inst].rx[q];
    l0[p.inst].by[q] = (Ti)out[p.inst].ry[q];
}

template <typename To, typename Ti>
__global__ void kb_cast_out(const BOuter<To> *__restrict__ out, const BLevel<Ti> *__restrict__ l0,
                            const BSeg *__restrict__ m, int n, const int *__restrict__ active)
{
    const Pt p = point_of(m, n);
    if (!p.valid || (active && !active[p.inst])) return;
    const size_t q = (size_t)p.j * l0[p.inst].g.pitch + p.i;
    out[p.inst].zx[q] = (To)l0[p.inst].vx[q];
    out[p.inst].zy[q] = (To)l0[p.inst].vy[q];
}

// ---- outer solve -------------------------------------------------------------------
template <typename T>
__global__ void kb_residual_energy(const BOuter<T> *__restrict__ tab, const BSeg *__restrict__ m, int n,
                                   double *__restrict__ partials)
{
    const Pt p = point_of(m, n);
    double s0 = 0.0, s1 = 0.0;
    if (p.valid) {
        const BOuter<T> &o = tab[p.inst];
        const GridDesc<T> &g = o.g;
        const int i = p.i, j = p.j;
        const size_t q = (size_t)j * g.pitch + i;
        T mm, d, vc;
        CellSq<T> c0(s0), c1(s1); // the cell's vx and vy terms
        if (j < g.ny) {
            T r = T(0);
            if (vx_unknown(g, j, i)) {
                op_x(g, o.ec, o.en, (const T *)o.vx, (const T *)o.vy, j, i, mm, d, vc);
                r = r_sub(o.bx[q], mm);
                c0.add(r, -o.ivx[q]);
                c1.add(o.fx[q], -o.ivx[q]);
            }
            o.rx[q] = r;
        }
        if (i < g.nx) {
            T r = T(0);
            if (vy_unknown(g, j, i)) {
                op_y(g, o.ec, o.en, (const T *)o.vx, (const T *)o.vy, j, i, mm, d, vc);
                r = r_sub(o.by[q], mm);
                c0.add(r, -o.ivy[q]);
                c1.add(o.fy[q], -o.ivy[q]);
            }
            o.ry[q] = r;
        }
        c0.done();
        c1.done();
    }
    block_store2(s0, s1, partials);
}

template <typename T>
__global__ void kb_apply_dot(const BOuter<T> *__restrict__ tab, const BSeg *__restrict__ m, int n,
                             double *__restrict__ partials)
{
    // the blocks of an instance are its 32 x 8 tiles (BATCH_BX x BATCH_BY)
    __shared__ ApplyTile<T> sm;
    const BSeg sg = m[seg_of(m, n, blockIdx.x)];
    const int lb = blockIdx.x - sg.block_begin;
    const BOuter<T> &o = tab[sg.inst];
    double s0 = 0.0, s1 = 0.0;
    static_assert(BATCH_BX == AT_X && BATCH_BY == AT_Y, "batched blocks are apply tiles");
    apply_dot_tile<T>(o.g, o.ec, o.en, o.ax, o.ay, o.px, o.py, o.qx, o.qy, o.rx, o.ry, (lb % sg.bxb) * BATCH_BX,
                      (lb / sg.bxb) * BATCH_BY, (int)(threadIdx.y * BATCH_BX + threadIdx.x), sm, s0, s1);
    block_store2(s0, s1, partials);
}

template <typename T>
__global__ void kb_update(const BOuter<T> *__restrict__ tab, const BSeg *__restrict__ m, int n,
                          const double *__restrict__ alpha, double *__restrict__ partials)
{
    const Pt p = point_of(m, n);
    double s0 = 0.0;
    if (p.valid) {
        const BOuter<T> &o = tab[p.inst];
        const GridDesc<T> &g = o.g;
        const T a = (T)alpha[p.inst];
        const int i = p.i, j = p.j;
        const size_t q = (size_t)j * g.pitch + i;
        if (vx_unknown(g, j, i)) {
            o.vx[q] = r_fma(a, o.px[q], o.vx[q]);
            const T rn = r_fma(-a, o.qx[q], o.rx[q]);
            o.rx[q] = rn;
            s0 = acc_sq(s0, rn, -o.ivx[q]);
        }
        if (vy_unknown(g, j, i)) {
            o.vy[q] = r_fma(a, o.py[q], o.vy[q]);
            const T rn = r_fma(-a, o.qy[q], o.ry[q]);
            o.ry[q] = rn;
            s0 = acc_sq(s0, rn, -o.ivy[q]);
        }
    }
    block_store2(s0, 0.0, partials);
}

template <typename T>
__global__ void kb_dot_zq(const BOuter<T> *__restrict__ tab, const BSeg *__restrict__ m, int n,
                          double *__restrict__ partials)
{
    const Pt p = point_of(m, n);
    double s0 = 0.0;
    if (p.valid) {
        const BOuter<T> &o = tab[p.inst];
        const GridDesc<T> &g = o.g;
        const size_t q = (size_t)p.j * g.pitch + p.i;
        if (vx_unknown(g, p.j, p.i)) s0 = fma((double)o.zx[q], (double)o.qx[q], s0);
        if (vy_unknown(g, p.j, p.i)) s0 = fma((double)o.zy[q], (double)o.qy[q], s0);
    }
    block_store2(s0, 0.0, partials);
}

template <typename T>
__global__ void kb_direction(const BOuter<T> *__restrict__ tab, const BSeg *__restrict__ m, int n,
                             const double *__restrict__ beta)
{
    const Pt p = point_of(m, n);
    if (!p.valid) return;
    const BOuter<T> &o = tab[p.inst];
    const GridDesc<T> &g = o.g;
    const size_t q = (size_t)p.j * g.pitch + p.i;
    const T b = beta ? (T)beta[p.inst] : T(0);
    if (vx_unknown(g, p.j, p.i)) o.px[q] = beta ? r_fma(b, o.px[q], o.zx[q]) : o.zx[q];
    if (vy_unknown(g, p.j, p.i)) o.py[q] = beta ? r_fma(b, o.py[q], o.zy[q]) : o.zy[q];
}

// Flexible CG without casts around the V-cycle: the update also writes r in
// the inner precision into the finest level's right-hand side (l0), and
// <z, q> and p = z + beta p read z in the inner precision where the V-cycle
// leaves it (fin); (To) of an inner value is exact, so the iterates are those
// of the casting form.
template <typename To, typename Ti>
__global__ void kb_update_cast(const BOuter<To> *__restrict__ tab, const BLevel<Ti> *__restrict__ l0,
                               const BSeg *__restrict__ m, int n, const double *__restrict__ alpha,
                               double *__restrict__ partials)
{
    const Pt p = point_of(m, n);
    double s0 = 0.0;
    if (p.valid) {
        const BOuter<To> &o = tab[p.inst];
        const GridDesc<To> &g = o.g;
        const To a = (To)alpha[p.inst];
        const int i = p.i, j = p.j;
        const size_t q = (size_t)j * g.pitch + i;
        if (vx_unknown(g, j, i)) {
            o.vx[q] = r_fma(a, o.px[q], o.vx[q]);
            const To rn = r_fma(-a, o.qx[q], o.rx[q]);
            o.rx[q] = rn;
            l0[p.inst].bx[q] = (Ti)rn;
            s0 = acc_sq(s0, rn, -o.ivx[q]);
        }
        if (vy_unknown(g, j, i)) {
            o.vy[q] = r_fma(a, o.py[q], o.vy[q]);
            const To rn = r_fma(-a, o.qy[q], o.ry[q]);
            o.ry[q] = rn;
            l0[p.inst].by[q] = (Ti)rn;
            s0 = acc_sq(s0, rn, -o.ivy[q]);
        }
    }
    block_store2(s0, 0.0, partials);
}

template <typename To, typename Ti>
__global__ void kb_dot_zq_in(const BOuter<To> *__restrict__ tab, const BLevel<Ti> *__restrict__ fin,
                             const BSeg *__restrict__ m, int n, double *__restrict__ partials)
{
    const Pt p = point_of(m, n);
    double s0 = 0.0;
    if (p.valid) {
        const BOuter<To> &o = tab[p.inst];
        const GridDesc<To> &g = o.g;
        const size_t q = (size_t)p.j * g.pitch + p.i;
        if (vx_unknown(g, p.j, p.i)) s0 = fma((double)fin[p.inst].vx[q], (double)o.qx[q], s0);
        if (vy_unknown(g, p.j, p.i)) s0 = fma((double)fin[p.inst].vy[q], (double)o.qy[q], s0);
    }
    block_store2(s0, 0.0, partials);
}

template <typename To, typename Ti>
__global__ void kb_direction_in(const BOuter<To> *__restrict__ tab, const BLevel<Ti> *__restrict__ fin,
                                const BSeg *__restrict__ m, int n, const double *__restrict__ beta)
{
    const Pt p = point_of(m, n);
    if (!p.valid) return;
    const BOuter<To> &o = tab[p.inst];
    const GridDesc<To> &g = o.g;
    const size_t q = (size_t)p.j * g.pitch + p.i;
    const To b = beta ? (To)beta[p.inst] : To(0);
    if (vx_unknown(g, p.j, p.i)) {
        const To z = (To)fin[p.inst].vx[q];
        o.px[q] = beta ? r_fma(b, o.px[q], z) : z;
    }
    if (vy_unknown(g, p.j, p.i)) {
        const To z = (To)fin[p.inst].vy[q];
        o.py[q] = beta ? r_fma(b, o.py[q], z) : z;
    }
}

template <typename T>
__global__ void kb_add(const BOuter<T> *__restrict__ tab, const BSeg *__restrict__ m, int n,
                       const int *__restrict__ active)
{
    const Pt p = point_of(m, n);
    if (!p.valid || !active[p.inst]) return;
    const BOuter<T> &o = tab[p.inst];
    const GridDesc<T> &g = o.g;
    const size_t q = (size_t)p.j * g.pitch + p.i;
    if (vx_unknown(g, p.j, p.i)) o.vx[q] = r_add(o.vx[q], o.zx[q]);
    if (vy_unknown(g, p.j, p.i)) o.vy[q] = r_add(o.vy[q], o.zy[q]);
}

__global__ void k_scalars(int count, const double *__restrict__ pq_pr, const double *__restrict__ zq,
                          const int *__restrict__ active, double *__restrict__ alpha, double *__restrict__ beta)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const bool on = active[i] != 0;
    if (alpha) alpha[i] = on ? pq_pr[2 * i + 1] / pq_pr[2 * i] : 0.0;
    if (beta) beta[i] = on ? -zq[2 * i] / pq_pr[2 * i] : 0.0;
}

inline unsigned nblk(int nb) { return (unsigned)(nb > 0 ? nb : 1); }

} // namespace

#define BLOCK dim3(BATCH_BX, BATCH_BY)

template <typename T>
cudaError_t batch_rhs(const BRhs<T> *tab, const BSeg *map, int nseg, int nblocks, cudaStream_t s)
{
    if (nblocks > 0) kb_rhs<T><<<nblocks, BLOCK, 0, s>>>(tab, map, nseg);
    return cudaGetLastError();
}
template <typename T>
cudaError_t batch_residual(const BLevel<T> *tab, const BSeg *map, int nseg, int nblocks, const int *active,
                           cudaStream_t s)
{
    if (nblocks > 0) kb_residual<T><<<nblocks, BLOCK, 0, s>>>(tab, map, nseg, active);
    return cudaGetLastError();
}
template <typename T>
cudaError_t batch_restrict(const BLevel<T> *tab, const BSeg *map, int nseg, int nblocks, const int *active,
                           cudaStream_t s)
{
    if (nblocks > 0) kb_restrict<T><<<nblocks, BLOCK, 0, s>>>(tab, map, nseg, active);
    return cudaGetLastError();
}
template <typename T>
cudaError_t batch_prolong(const BLevel<T> *tab, const BSeg *map, int nseg, int nblocks, const int *active,
                          cudaStream_t s)
{
    if (nblocks > 0) kb_prolong<T><<<nblocks, BLOCK, 0, s>>>(tab, map, nseg, active);
    return cudaGetLastError();
}
template <typename T>
cudaError_t batch_zero_v(const BLevel<T> *tab, const BSeg *map, int nseg, int nblocks, const int *active,
                         cudaStream_t s)
{
    if (nblocks > 0) kb_zero_v<T><<<nblocks, BLOCK, 0, s>>>(tab, map, nseg, active);
    return cudaGetLastError();
}
template <typename T>
cudaError_t batch_copy(const BLevel<T> *tab, const BSeg *map, int nseg, int nblocks, bool to_scratch,
                       const int *active, cudaStream_t s)
{
    if (nblocks > 0) kb_copy<T><<<nblocks, BLOCK, 0, s>>>(tab, map, nseg, to_scratch, active);
    return cudaGetLastError();
}
template <typename T>
cudaError_t batch_copy_walls(const BLevel<T> *tab, const BSeg *map, int nseg, const int *active, cudaStream_t s)
{
    if (nseg > 0) kb_copy_walls<T><<<nseg, 256, 0, s>>>(tab, map, active);
    return cudaGetLastError();
}
template <typename T>
cudaError_t batch_dense(const BDense<T> *tab, int count, int rows, const int *active, cudaStream_t s)
{
    if (count <= 0 || rows <= 0) return cudaSuccess;
    kb_dense_pack<T><<<(rows + 255) / 256, 256, 0, s>>>(tab, count, rows, active);
    kb_dense_solve<T><<<(rows + 7) / 8, 256, 0, s>>>(tab, count, rows, active);
    kb_dense_unpack<T><<<(rows + 255) / 256, 256, 0, s>>>(tab, count, rows, active);
    return cudaGetLastError();
}
template <typename To, typename Ti>
cudaError_t batch_cast_in(const BOuter<To> *out, const BLevel<Ti> *l0, const BSeg *map, int nseg, int nblocks,
                          const int *active, cudaStream_t s)
{
    if (nblocks > 0) kb_cast_in<To, Ti><<<nblocks, BLOCK, 0, s>>>(out, l0, map, nseg, active);
    return cudaGetLastError();
}
template <typename To, typename Ti>
cudaError_t batch_cast_out(const BOuter<To> *out, const BLevel<Ti> *l0, const BSeg *map, int nseg, int nblocks,
                           const int *active, cudaStream_t s)
{
    if (nblocks > 0) kb_cast_out<To, Ti><<<nblocks, BLOCK, 0, s>>>(out, l0, map, nseg, active);
    return cudaGetLastError();
}

template <typename T>
cudaError_t batch_residual_energy(const BOuter<T> *tab, const BSeg *map, int nseg, int nblocks, double *partials,
                                  double *out, cudaStream_t s)
{
    kb_residual_energy<T><<<nblk(nblocks), BLOCK, 0, s>>>(tab, map, nseg, partials);
    k_seg_final<<<(nseg + 7) / 8, 256, 0, s>>>(map, nseg, partials, out);
    return cudaGetLastError();
}
template <typename T>
cudaError_t batch_apply_dot(const BOuter<T> *tab, const BSeg *map, int nseg, int nblocks, double *partials,
                            double *out, cudaStream_t s)
{
    kb_apply_dot<T><<<nblk(nblocks), BLOCK, 0, s>>>(tab, map, nseg, partials);
    k_seg_final<<<(nseg + 7) / 8, 256, 0, s>>>(map, nseg, partials, out);
    return cudaGetLastError();
}
template <typename T>
cudaError_t batch_update(const BOuter<T> *tab, const BSeg *map, int nseg, int nblocks, const double *alpha,
                         double *partials, double *out, cudaStream_t s)
{
    kb_update<T><<<nblk(nblocks), BLOCK, 0, s>>>(tab, map, nseg, alpha, partials);
    k_seg_final<<<(nseg + 7) / 8, 256, 0, s>>>(map, nseg, partials, out);
    return cudaGetLastError();
}
template <typename T>
cudaError_t batch_dot_zq(const BOuter<T> *tab, const BSeg *map, int nseg, int nblocks, double *partials,
                         double *out, cudaStream_t s)
{
    kb_dot_zq<T><<<nblk(nblocks), BLOCK, 0, s>>>(tab, map, nseg, partials);
    k_seg_final<<<(nseg + 7) / 8, 256, 0, s>>>(map, nseg, partials, out);
    return cudaGetLastError();
}
template <typename T>
cudaError_t batch_direction(const BOuter<T> *tab, const BSeg *map, int nseg, int nblocks, const double *beta,
                            cudaStream_t s)
{
    if (nblocks > 0) kb_direction<T><<<nblocks, BLOCK, 0, s>>>(tab, map, nseg, beta);
    return cudaGetLastError();
}
template <typename To, typename Ti>
cudaError_t batch_update_cast(const BOuter<To> *tab, const BLevel<Ti> *l0, const BSeg *map, int nseg, int nblocks,
                              const double *alpha, double *partials, double *out, cudaStream_t s)
{
    kb_update_cast<To, Ti><<<nblk(nblocks), BLOCK, 0, s>>>(tab, l0, map, nseg, alpha, partials);
    k_seg_final<<<(nseg + 7) / 8, 256, 0, s>>>(map, nseg, partials, out);
    return cudaGetLastError();
}
template <typename To, typename Ti>
cudaError_t batch_dot_zq_in(const BOuter<To> *tab, const BLevel<Ti> *fin, const BSeg *map, int nseg, int nblocks,
                            double *partials, double *out, cudaStream_t s)
{
    kb_dot_zq_in<To, Ti><<<nblk(nblocks), BLOCK, 0, s>>>(tab, fin, map, nseg, partials);
    k_seg_final<<<(nseg + 7) / 8, 256, 0, s>>>(map, nseg, partials, out);
    return cudaGetLastError();
}
template <typename To, typename Ti>
cudaError_t batch_direction_in(const BOuter<To> *tab, const BLevel<Ti> *fin, const BSeg *map, int nseg, int nblocks,
                               const double *beta, cudaStream_t s)
{
    if (nblocks > 0) kb_direction_in<To, Ti><<<nblocks, BLOCK, 0, s>>>(tab, fin, map, nseg, beta);
    return cudaGetLastError();
}
#define INST_IN(To, Ti)                                                                                            \
    template cudaError_t batch_update_cast<To, Ti>(const BOuter<To> *, const BLevel<Ti> *, const BSeg *, int, int, \
                                                   const double *, double *, double *, cudaStream_t);              \
    template cudaError_t batch_dot_zq_in<To, Ti>(const BOuter<To> *, const BLevel<Ti> *, const BSeg *, int, int,   \
                                                 double *, double *, cudaStream_t);                                \
    template cudaError_t batch_direction_in<To, Ti>(const BOuter<To> *, const BLevel<Ti> *, const BSeg *, int,     \
                                                    int, const double *, cudaStream_t);
INST_IN(double, float)
INST_IN(double, double)
INST_IN(float, float)
INST_IN(float, double)
#undef INST_IN

template <typename T>
cudaError_t batch_add(const BOuter<T> *tab, const BSeg *map, int nseg, int nblocks, const int *active, cudaStream_t s)
{
    if (nblocks > 0) kb_add<T><<<nblocks, BLOCK, 0, s>>>(tab, map, nseg, active);
    return cudaGetLastError();
}
cudaError_t batch_scalars(int count, const double *pq_pr, const double *zq, const int *active, double *alpha,
                          double *beta, cudaStream_t s)
{
    k_scalars<<<(count + 255) / 256, 256, 0, s>>>(count, pq_pr, zq, active, alpha, beta);
    return cudaGetLastError();
}

#define INST(T)                                                                                                    \
    template cudaError_t batch_rhs<T>(const BRhs<T> *, const BSeg *, int, int, cudaStream_t);                      \
    template cudaError_t batch_residual<T>(const BLevel<T> *, const BSeg *, int, int, const int *, cudaStream_t);  \
    template cudaError_t batch_restrict<T>(const BLevel<T> *, const BSeg *, int, int, const int *, cudaStream_t);  \
    template cudaError_t batch_prolong<T>(const BLevel<T> *, const BSeg *, int, int, const int *, cudaStream_t);   \
    template cudaError_t batch_zero_v<T>(const BLevel<T> *, const BSeg *, int, int, const int *, cudaStream_t);    \
    template cudaError_t batch_copy<T>(const BLevel<T> *, const BSeg *, int, int, bool, const int *,               \
                                       cudaStream_t);                                                              \
    template cudaError_t batch_copy_walls<T>(const BLevel<T> *, const BSeg *, int, const int *, cudaStream_t);     \
    template cudaError_t batch_dense<T>(const BDense<T> *, int, int, const int *, cudaStream_t);                   \
    template cudaError_t batch_residual_energy<T>(const BOuter<T> *, const BSeg *, int, int, double *, double *,   \
                                                  cudaStream_t);                                                   \
    template cudaError_t batch_apply_dot<T>(const BOuter<T> *, const BSeg *, int, int, double *, double *,         \
                                            cudaStream_t);                                                         \
    template cudaError_t batch_update<T>(const BOuter<T> *, const BSeg *, int, int, const double *, double *,      \
                                         double *, cudaStream_t);                                                  \
    template cudaError_t batch_dot_zq<T>(const BOuter<T> *, const BSeg *, int, int, double *, double *,            \
                                         cudaStream_t);                                                            \
    template cudaError_t batch_direction<T>(const BOuter<T> *, const BSeg *, int, int, const double *,             \
                                            cudaStream_t);                                                         \
    template cudaError_t batch_add<T>(const BOuter<T> *, const BSeg *, int, int, const int *, cudaStream_t);
INST(float)
INST(double)
#undef INST
template cudaError_t batch_cast_in<double, float>(const BOuter<double> *, const BLevel<float> *, const BSeg *, int, int,
                                                   const int *, cudaStream_t);
template cudaError_t batch_cast_in<double, double>(const BOuter<double> *, const BLevel<double> *, const BSeg *, int, int,
                                                   const int *, cudaStream_t);
template cudaError_t batch_cast_in<float, float>(const BOuter<float> *, const BLevel<float> *, const BSeg *, int, int,
                                                   const int *, cudaStream_t);
template cudaError_t batch_cast_in<float, double>(const BOuter<float> *, const BLevel<double> *, const BSeg *, int, int,
                                                   const int *, cudaStream_t);
template cudaError_t batch_cast_out<double, float>(const BOuter<double> *, const BLevel<float> *, const BSeg *, int, int,
                                                   const int *, cudaStream_t);
template cudaError_t batch_cast_out<double, double>(const BOuter<double> *, const BLevel<double> *, const BSeg *,
                                                    int, int, const int *, cudaStream_t);
template cudaError_t batch_cast_out<float, float>(const BOuter<float> *, const BLevel<float> *, const BSeg *, int, int,
                                                   const int *, cudaStream_t);
template cudaError_t batch_cast_out<float, double>(const BOuter<float> *, const BLevel<double> *, const BSeg *, int, int,
                                                   const int *, cudaStream_t);

} // namespace stokes
