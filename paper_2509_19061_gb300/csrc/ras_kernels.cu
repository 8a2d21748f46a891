// ras_kernels.cu -- RAS-type temporally blocked Jacobi (Sec. 4.3 and
// Algorithm 2 of arXiv 2509.19061) and, as its one-sweep case, the spatially
// blocked fused Jacobi smoother (Sec. 4.2, Sec. 5 (iv)).
//
// One CTA per tile of the shifted tiling.  The CTA stages the tile grown by
// overlap+1 cells (the overlap plus the Dirichlet ring) of every field into
// shared memory, runs the local Jacobi sweeps there with a shared-memory
// ping-pong, and writes back only the unknowns of the tile's own cells.  All
// tiles read the snapshot (vx, vy) and write (ox, oy), so the result does not
// depend on the order in which tiles run and every unknown has one writer
// (the in-place benign race of the CPU original is gone).
//
// Sweep s of ks only updates the cells within min(overlap, ks - s) of the
// tile: the owned unknowns after ks sweeps depend on sweep s only through
// that region (the stencil reaches one cell per sweep), so skipping the rest
// leaves the result unchanged.
#include <algorithm>

#include "internal.h"
#include "stencil.cuh"

namespace stokes {

namespace {

constexpr int RAS_THREADS = 256;
constexpr int RAS_PLANES = 8; // vx, vy ping-pong (4), eta_c, eta_n, bx, by

struct TileRange {
    int x0, x1, y0, y1;
};

// Tile (bx, by) of the tiling cut at s + m T, clipped to [0, n).
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
    int wxp; // shared-memory row pitch (elements)
    int plane;
};

template <typename T>
__global__ void __launch_bounds__(RAS_THREADS) k_ras(RasArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    const int plane = a.plane, W = a.wxp;
    T *Ax = sm, *Ay = sm + plane, *Bx = sm + 2 * plane, *By = sm + 3 * plane;
    T *Ec = sm + 4 * plane, *En = sm + 5 * plane, *Rx = sm + 6 * plane, *Ry = sm + 7 * plane;

    const GridDesc<T> &g = a.g;
    const int nx = g.nx, ny = g.ny;
    const size_t P = (size_t)g.pitch;
    const int btx = blockIdx.x % a.tg.ntx, bty = blockIdx.x / a.tg.ntx;
    int x0, x1, y0, y1;
    tile_interval(nx, a.tg.ti, a.tg.si, btx, x0, x1);
    tile_interval(ny, a.tg.tj, a.tg.sj, bty, y0, y1);
    const int h = a.overlap + 1;
    const int ox0 = x0 - h, oy0 = y0 - h;             // window origin (global cell index)
    const int wx = x1 - x0 + 2 * h, wy = y1 - y0 + 2 * h; // window extent

    // ---- stage the window; entries outside each field's extent are zero
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

    // ---- ks local sweeps, shrinking to the region that still matters
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
            T m, d;
            if (gx >= 1 && gx <= nx - 1) { // vx unknown (gy < ny holds)
                stencil_x(g, cx[q], cx[q + 1], cx[q - 1], cx[q + W], cx[q - W], cy[q + W], cy[q + W - 1], cy[q],
                          cy[q - 1], Ec[q], Ec[q - 1], En[q + W], En[q], m, d);
                nxv[q] = jacobi_update(cx[q], Rx[q], m, d, a.omega);
            }
            if (gy >= 1 && gy <= ny - 1) { // vy unknown (gx < nx holds)
                stencil_y(g, cy[q], cy[q + W], cy[q - W], cy[q + 1], cy[q - 1], cx[q + 1], cx[q + 1 - W], cx[q],
                          cx[q - W], Ec[q], Ec[q - W], En[q + 1], En[q], m, d);
                nyv[q] = jacobi_update(cy[q], Ry[q], m, d, a.omega);
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

    // ---- write back the unknowns of the tile's own cells
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

size_t ras_smem_bytes(int ti, int tj, int overlap, size_t elem)
{
    const size_t h = (size_t)overlap + 1;
    return (size_t)RAS_PLANES * ((size_t)ti + 2 * h) * ((size_t)tj + 2 * h) * elem;
}

int ras_max_smem()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

template <typename T>
cudaError_t launch_ras(const GridDesc<T> &g, const Coeffs<T> &c, T omega, const TileGrid &tg, int ksweeps,
                       int overlap, const T *vx, const T *vy, T *ox, T *oy, cudaStream_t s)
{
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
    // a tile never spans more than min(T, n) cells
    const int ex = tg.ti < g.nx ? tg.ti : g.nx, ey = tg.tj < g.ny ? tg.tj : g.ny;
    a.wxp = ex + 2 * (overlap + 1);
    a.plane = a.wxp * (ey + 2 * (overlap + 1));
    const size_t smem = ras_smem_bytes(ex, ey, overlap, sizeof(T));
    cudaError_t e = cudaFuncSetAttribute(k_ras<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned nblocks = (unsigned)tg.ntx * (unsigned)tg.nty;
    k_ras<T><<<nblocks, RAS_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_ras<float>(const GridDesc<float> &, const Coeffs<float> &, float, const TileGrid &, int,
                                       int, const float *, const float *, float *, float *, cudaStream_t);
template cudaError_t launch_ras<double>(const GridDesc<double> &, const Coeffs<double> &, double, const TileGrid &,
                                        int, int, const double *, const double *, double *, double *, cudaStream_t);

} // namespace stokes
