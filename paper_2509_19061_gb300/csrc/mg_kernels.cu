// mg_kernels.cu -- kernels of the geometric-multigrid V-cycle used for the
// velocity solve of the inexact Uzawa method (Sec. 3.2, configuration in
// Sec. 6.2): coarse viscosity, residual, restriction, prolongation, precision
// casts and the dense FP64 coarsest solve.
//
// Transfer operators (the paper does not state them): bilinear prolongation
// P in the staggered coordinates with mirror ghosts for the tangential
// direction and zero walls; restriction R = P^T / 4.
#include "../../include/stokes.h"
#include "gstencil.cuh"
#include "internal.h"
#include "mg.h"
#include "mg_point.cuh"

namespace stokes {

namespace {

constexpr int BX = 32, BY = 8;
inline dim3 grid2d(int w, int h) { return dim3((unsigned)((w + BX - 1) / BX), (unsigned)((h + BY - 1) / BY)); }

// coarse eta_c = mean of the four children; coarse eta_n at an interior node =
// full-weighting mean of the 3 x 3 fine nodes around the coincident node
// (4 centre, 2 edges, 1 corners, over 16), 0 on boundary nodes.  Injecting
// eta_n would make the coarse operator too soft next to stiff inclusions.
template <typename T>
__global__ void k_coarsen_eta(int ncx, int ncy, int fp, int cp, const T *__restrict__ fec, const T *__restrict__ fen,
                              T *__restrict__ cec, T *__restrict__ cen)
{
    const int I = blockIdx.x * BX + threadIdx.x, J = blockIdx.y * BY + threadIdx.y;
    if (I > ncx || J > ncy) return;
    const size_t cq = (size_t)J * cp + I, f0 = (size_t)(2 * J) * fp + 2 * I;
    if (I < ncx && J < ncy) {
        const T s = r_add(r_add(r_add(fec[f0], fec[f0 + 1]), fec[f0 + fp]), fec[f0 + fp + 1]);
        cec[cq] = r_mul(T(0.25), s);
    }
    T v = T(0);
    if (I >= 1 && I <= ncx - 1 && J >= 1 && J <= ncy - 1) {
        const T centre = fen[f0];
        const T edges = r_add(r_add(r_add(fen[f0 - fp], fen[f0 + fp]), fen[f0 - 1]), fen[f0 + 1]);
        const T corners = r_add(r_add(r_add(fen[f0 - fp - 1], fen[f0 - fp + 1]), fen[f0 + fp - 1]), fen[f0 + fp + 1]);
        v = r_mul(r_add(r_add(r_mul(T(4), centre), r_mul(T(2), edges)), corners), T(0.0625));
    }
    cen[cq] = v;
}

template <typename Ts, typename Td>
__global__ void k_cast(size_t n, const Ts *__restrict__ s, Td *__restrict__ d)
{
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        d[t] = (Td)s[t];
}

// r = b - M v at unknowns, zero elsewhere (rows up to ny, columns up to nx)
template <typename T>
__global__ void k_residual(GridDesc<T> g, const T *__restrict__ ec, const T *__restrict__ en,
                           const T *__restrict__ bx, const T *__restrict__ by, const T *__restrict__ vx,
                           const T *__restrict__ vy, T *__restrict__ rx, T *__restrict__ ry)
{
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    if (i > g.nx || j > g.ny) return;
    const size_t q = (size_t)j * g.pitch + i;
    T m, d, vc;
    if (j < g.ny) {
        T r = T(0);
        if (vx_unknown(g, j, i)) {
            op_x(g, ec, en, vx, vy, j, i, m, d, vc);
            r = r_sub(bx[q], m);
        }
        rx[q] = r;
    }
    if (i < g.nx) {
        T r = T(0);
        if (vy_unknown(g, j, i)) {
            op_y(g, ec, en, vx, vy, j, i, m, d, vc);
            r = r_sub(by[q], m);
        }
        ry[q] = r;
    }
}

// fine += P coarse at the fine unknowns
template <typename T>
__global__ void k_prolong_add(int nfx, int nfy, int fp, int ncx, int ncy, int cp, const T *__restrict__ cx,
                              const T *__restrict__ cy, T *__restrict__ fx, T *__restrict__ fy)
{
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    if (i > nfx || j > nfy) return;
    prolong_point(nfx, nfy, fp, ncx, ncy, cp, cx, cy, fx, fy, j, i);
}

// coarse b = P^T r / 4 at the coarse unknowns (gather form), zero elsewhere
template <typename T>
__global__ void k_restrict(int nfx, int nfy, int fp, int ncx, int ncy, int cp, const T *__restrict__ rx,
                           const T *__restrict__ ry, T *__restrict__ bx, T *__restrict__ by)
{
    const int I = blockIdx.x * BX + threadIdx.x, J = blockIdx.y * BY + threadIdx.y;
    if (I > ncx || J > ncy) return;
    restrict_point(nfx, nfy, fp, ncx, ncy, cp, rx, ry, bx, by, J, I);
}

// ---- dense coarsest solve --------------------------------------------------
// Unknown numbering: vx unknowns row-major (j, i = 1..nx-1), then vy unknowns
// row-major (j = 1..ny-1, i).
__device__ __forceinline__ void unknown_pos(int u, int nx, int ny, int &comp, int &j, int &i)
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

// A[r][c] = -(M e_c)_r in FP64 from the level's viscosity (boundary nodes of
// eta_n hold zero)
// (one job per blockIdx.y)
template <typename T>
__global__ void k_assemble(const DenseJob *__restrict__ jobs)
{
    const DenseJob &jb = jobs[blockIdx.y];
    const int nx = jb.nx, ny = jb.ny, pitch = jb.pitch, n = jb.n;
    const double ihx = jb.ihx, ihy = jb.ihy;
    const T *__restrict__ ec = (const T *)jb.ec;
    const T *__restrict__ en = (const T *)jb.en;
    double *__restrict__ A = jb.A;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)n * n) return;
    const int r = (int)(t / n), c = (int)(t - (long)r * n);
    int rc, rj, ri, cc, cj, ci;
    unknown_pos(r, nx, ny, rc, rj, ri);
    unknown_pos(c, nx, ny, cc, cj, ci);
    // value of the unit vector e_c at (component, j, i)
    auto ux = [&](int j, int i) { return (cc == 0 && cj == j && ci == i) ? 1.0 : 0.0; };
    auto uy = [&](int j, int i) { return (cc == 1 && cj == j && ci == i) ? 1.0 : 0.0; };
    auto EC = [&](int j, int i) { return (double)ec[(size_t)j * pitch + i]; };
    auto EN = [&](int j, int i) { return (double)en[(size_t)j * pitch + i]; };
    double m;
    if (rc == 0) {
        const int j = rj, i = ri;
        const double txe = 2.0 * EC(j, i) * (ux(j, i + 1) - ux(j, i)) * ihx;
        const double txw = 2.0 * EC(j, i - 1) * (ux(j, i) - ux(j, i - 1)) * ihx;
        const double sn = EN(j + 1, i) * ((ux(j + 1, i) - ux(j, i)) * ihy + (uy(j + 1, i) - uy(j + 1, i - 1)) * ihx);
        const double ss = EN(j, i) * ((ux(j, i) - ux(j - 1, i)) * ihy + (uy(j, i) - uy(j, i - 1)) * ihx);
        m = (txe - txw) * ihx + (sn - ss) * ihy;
    } else {
        const int j = rj, i = ri;
        const double tyn = 2.0 * EC(j, i) * (uy(j + 1, i) - uy(j, i)) * ihy;
        const double tys = 2.0 * EC(j - 1, i) * (uy(j, i) - uy(j - 1, i)) * ihy;
        const double se = EN(j, i + 1) * ((ux(j, i + 1) - ux(j - 1, i + 1)) * ihy + (uy(j, i + 1) - uy(j, i)) * ihx);
        const double sw = EN(j, i) * ((ux(j, i) - ux(j - 1, i)) * ihy + (uy(j, i) - uy(j, i - 1)) * ihx);
        m = (se - sw) * ihx + (tyn - tys) * ihy;
    }
    A[(size_t)r * n + c] = -m;
}

// In-place Cholesky A = L L^T (lower triangle) by one CTA per job
// (blockIdx.x); status = 1 if a pivot is not positive.  Every entry is
// updated in the order k = 0, 1, ..., whatever the thread layout.
__global__ void k_cholesky(const DenseJob *__restrict__ jobs)
{
    const DenseJob &jb = jobs[blockIdx.x];
    const int n = jb.n;
    double *__restrict__ A = jb.A;
    __shared__ double piv;
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x == 0) {
            const double d = A[(size_t)k * n + k];
            if (!(d > 0.0)) bad = 1;
            piv = d > 0.0 ? sqrt(d) : 1.0;
            A[(size_t)k * n + k] = piv;
        }
        __syncthreads();
        for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) A[(size_t)i * n + k] /= piv;
        __syncthreads();
        // trailing lower triangle, rows/cols k+1..n-1: warp w takes rows
        // k+1+w, k+1+w+nw, ..., its lanes the columns of a row
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int i = k + 1 + w; i < n; i += nw) {
            const double lik = A[(size_t)i * n + k];
            for (int j = k + 1 + lane; j <= i; j += 32) A[(size_t)i * n + j] -= lik * A[(size_t)j * n + k];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && bad) *jb.status = 1;
}

// W = L^{-1}, column c by thread c (forward substitution), lower triangle;
// one job per blockIdx.y
__global__ void k_tri_inverse(const DenseJob *__restrict__ jobs)
{
    const DenseJob &jb = jobs[blockIdx.y];
    const int n = jb.n;
    const double *__restrict__ L = jb.A;
    double *__restrict__ W = jb.W;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    for (int i = 0; i < c; ++i) W[(size_t)i * n + c] = 0.0;
    W[(size_t)c * n + c] = 1.0 / L[(size_t)c * n + c];
    for (int i = c + 1; i < n; ++i) {
        double s = 0.0;
        for (int m = c; m < i; ++m) s += L[(size_t)i * n + m] * W[(size_t)m * n + c];
        W[(size_t)i * n + c] = -s / L[(size_t)i * n + i];
    }
}

// Ainv = W^T W; one job per blockIdx.y
__global__ void k_gram(const DenseJob *__restrict__ jobs)
{
    const DenseJob &jb = jobs[blockIdx.y];
    const int n = jb.n;
    const double *__restrict__ W = jb.W;
    double *__restrict__ Ainv = jb.Ainv;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)n * n) return;
    const int i = (int)(t / n), j = (int)(t - (long)i * n);
    const int m0 = i > j ? i : j;
    double s = 0.0;
    for (int m = m0; m < n; ++m) s += W[(size_t)m * n + i] * W[(size_t)m * n + j];
    Ainv[(size_t)i * n + j] = s;
}

// pack the coarsest right-hand side into a dense FP64 vector
template <typename T>
__global__ void k_pack(int nx, int ny, int pitch, int n, const T *__restrict__ bx, const T *__restrict__ by,
                       double *__restrict__ b)
{
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    int comp, j, i;
    unknown_pos(u, nx, ny, comp, j, i);
    b[u] = (double)(comp == 0 ? bx : by)[(size_t)j * pitch + i];
}

// x = -Ainv b (solution of M x = b), one warp per row
__global__ void k_dense_solve(int n, const double *__restrict__ Ainv, const double *__restrict__ b,
                              double *__restrict__ x)
{
    const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (row >= n) return;
    double s = 0.0;
    for (int c = lane; c < n; c += 32) s += Ainv[(size_t)row * n + c] * b[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) x[row] = -s;
}

template <typename T>
__global__ void k_unpack(int nx, int ny, int pitch, int n, const double *__restrict__ x, T *__restrict__ vx,
                         T *__restrict__ vy)
{
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    int comp, j, i;
    unknown_pos(u, nx, ny, comp, j, i);
    (comp == 0 ? vx : vy)[(size_t)j * pitch + i] = (T)x[u];
}

} // namespace

// ---------------------------------------------------------------------------
template <typename T>
cudaError_t mg_coarsen_eta(const MgLevel &f, const MgLevel &c, cudaStream_t s)
{
    k_coarsen_eta<T><<<grid2d(c.nx + 1, c.ny + 1), dim3(BX, BY), 0, s>>>(
        c.nx, c.ny, f.pitch, c.pitch, (const T *)f.ec, (const T *)f.en, (T *)c.ec, (T *)c.en);
    return cudaGetLastError();
}

template <typename Ts, typename Td>
cudaError_t mg_cast(size_t n, const void *src, void *dst, cudaStream_t s)
{
    k_cast<Ts, Td><<<1216, 256, 0, s>>>(n, (const Ts *)src, (Td *)dst);
    return cudaGetLastError();
}

template <typename T>
cudaError_t mg_residual(const MgLevel &l, cudaStream_t s)
{
    const GridDesc<T> g = make_grid<T>(l.nx, l.ny, l.pitch, l.hx, l.hy);
    k_residual<T><<<grid2d(l.nx + 1, l.ny + 1), dim3(BX, BY), 0, s>>>(g, (const T *)l.ec, (const T *)l.en,
                                                                       (const T *)l.bx, (const T *)l.by,
                                                                       (const T *)l.vx, (const T *)l.vy, (T *)l.rx,
                                                                       (T *)l.ry);
    return cudaGetLastError();
}

template <typename T>
cudaError_t mg_restrict(const MgLevel &f, const MgLevel &c, cudaStream_t s)
{
    k_restrict<T><<<grid2d(c.nx + 1, c.ny + 1), dim3(BX, BY), 0, s>>>(f.nx, f.ny, f.pitch, c.nx, c.ny, c.pitch,
                                                                       (const T *)f.rx, (const T *)f.ry, (T *)c.bx,
                                                                       (T *)c.by);
    return cudaGetLastError();
}

template <typename T>
cudaError_t mg_prolong_add(const MgLevel &f, const MgLevel &c, cudaStream_t s)
{
    k_prolong_add<T><<<grid2d(f.nx + 1, f.ny + 1), dim3(BX, BY), 0, s>>>(f.nx, f.ny, f.pitch, c.nx, c.ny,
                                                                          c.pitch, (const T *)c.vx,
                                                                          (const T *)c.vy, (T *)f.vx, (T *)f.vy);
    return cudaGetLastError();
}

template <typename T>
cudaError_t mg_dense_setup_many(const DenseJob *jobs, int count, int nmax, cudaStream_t s)
{
    const long nn = (long)nmax * nmax;
    for (int j0 = 0; j0 < count; j0 += 65535) {
        const int c = count - j0 < 65535 ? count - j0 : 65535;
        const DenseJob *jb = jobs + j0;
        k_assemble<T><<<dim3((unsigned)((nn + 255) / 256), c), 256, 0, s>>>(jb);
        k_cholesky<<<c, 1024, 0, s>>>(jb);
        k_tri_inverse<<<dim3((nmax + 127) / 128, c), 128, 0, s>>>(jb);
        k_gram<<<dim3((unsigned)((nn + 255) / 256), c), 256, 0, s>>>(jb);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t mg_dense_setup(const MgLevel &l, int n, double *A, double *W, double *Ainv, int *status,
                           cudaStream_t s)
{
    DenseJob h;
    h.nx = l.nx;
    h.ny = l.ny;
    h.pitch = l.pitch;
    h.n = n;
    h.ihx = 1.0 / l.hx;
    h.ihy = 1.0 / l.hy;
    h.ec = l.ec;
    h.en = l.en;
    h.A = A;
    h.W = W;
    h.Ainv = Ainv;
    h.status = status;
    // a one-entry job table in stream-ordered memory, freed after the kernels
    DenseJob *d = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&d, sizeof(DenseJob), s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(d, &h, sizeof(DenseJob), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = mg_dense_setup_many<T>(d, 1, n, s);
    const cudaError_t e2 = cudaStreamSynchronize(s);
    cudaFreeAsync(d, s);
    return e != cudaSuccess ? e : e2;
}

template <typename T>
cudaError_t mg_dense_solve(const MgLevel &l, int n, const double *Ainv, double *bvec, double *xvec, cudaStream_t s)
{
    k_pack<T><<<(n + 255) / 256, 256, 0, s>>>(l.nx, l.ny, l.pitch, n, (const T *)l.bx, (const T *)l.by, bvec);
    k_dense_solve<<<(n + 7) / 8, 256, 0, s>>>(n, Ainv, bvec, xvec);
    k_unpack<T><<<(n + 255) / 256, 256, 0, s>>>(l.nx, l.ny, l.pitch, n, xvec, (T *)l.vx, (T *)l.vy);
    return cudaGetLastError();
}

#define INST(T)                                                                                                    \
    template cudaError_t mg_coarsen_eta<T>(const MgLevel &, const MgLevel &, cudaStream_t);                        \
    template cudaError_t mg_residual<T>(const MgLevel &, cudaStream_t);                                            \
    template cudaError_t mg_restrict<T>(const MgLevel &, const MgLevel &, cudaStream_t);                           \
    template cudaError_t mg_prolong_add<T>(const MgLevel &, const MgLevel &, cudaStream_t);                        \
    template cudaError_t mg_dense_setup<T>(const MgLevel &, int, double *, double *, double *, int *,              \
                                           cudaStream_t);                                                          \
    template cudaError_t mg_dense_setup_many<T>(const DenseJob *, int, int, cudaStream_t);                         \
    template cudaError_t mg_dense_solve<T>(const MgLevel &, int, const double *, double *, double *, cudaStream_t);
INST(float)
INST(double)
#undef INST
template cudaError_t mg_cast<double, float>(size_t, const void *, void *, cudaStream_t);
template cudaError_t mg_cast<float, double>(size_t, const void *, void *, cudaStream_t);
template cudaError_t mg_cast<double, double>(size_t, const void *, void *, cudaStream_t);
template cudaError_t mg_cast<float, float>(size_t, const void *, void *, cudaStream_t);

} // namespace stokes
