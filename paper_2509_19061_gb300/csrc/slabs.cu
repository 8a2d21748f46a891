// slabs.cu -- RAS-Jacobi as a domain decomposition into horizontal slabs
// (Sec. 4.3, Algorithm 2: every tile solves a local problem on its own
// overlapping subdomain and writes only the unknowns it owns), laid out as
// a multi-GPU code would be: each slab keeps its own copy of the fields on
// its rows plus a halo, runs the tile kernel on its own storage, and after
// every outer iteration takes the halo rows of its neighbours' new iterate
// by device-to-device copies, one copy per field and side.  Here all slabs
// live on the calling device and stream.
//
// Slab s owns the cell rows [r0, r1) (a balanced split of ny) and stores
// rows [R0, R1) = [r0 - H, r1 + H) clipped to the grid, H = tile_j +
// overlap + 1: every tile of the global shifted tiling that meets [r0, r1)
// then lies, with its window (overlap plus the Dirichlet ring), strictly
// inside the storage, so the slab computes it exactly as a single context
// does, from the same arithmetic: the slab result equals the single-grid
// result bit for bit.  Tiles that lie in the halo are computed too and
// overwritten by the exchange.  The storage's first and last rows are
// boundaries of the slab's grid (no shear, vy held fixed) but only halo
// tiles, whose results are discarded, ever reach them.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/stokes.h"
#include "internal.h"

using namespace stokes;

namespace {

#define CK(call)                                                                                                   \
    do {                                                                                                           \
        cudaError_t e_ = (call);                                                                                   \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);                                                        \
    } while (0)

struct Slab {
    int r0 = 0, r1 = 0; // own cell rows
    int R0 = 0, R1 = 0; // stored cell rows
    void *ec = nullptr, *en = nullptr, *fx = nullptr, *fy = nullptr, *bx = nullptr, *by = nullptr;
    void *ivx = nullptr, *ivy = nullptr, *p = nullptr;
    void *v[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}}; // two velocity pairs (vx, vy)
};

// own rows of slab s of n: a balanced split
void slab_rows(int ny, int n, int s, int *r0, int *r1)
{
    *r0 = (int)((long long)ny * s / n);
    *r1 = (int)((long long)ny * (s + 1) / n);
}

} // namespace

struct stokes_slabs {
    int nx, ny, dtype, pitch, nslabs;
    double hx, hy;
    size_t esize;
    cudaStream_t stream;
    void *eta_c = nullptr, *eta_n = nullptr, *fx = nullptr, *fy = nullptr; // global copies (library layout)
    bool have_eta = false, have_f = false;
    int halo = -1;          // H of the current slab storage (-1: none)
    bool stale = true;      // slab coefficients need rebuilding
    std::vector<Slab> slabs;
    int *dstatus = nullptr; // bounded-wait status of the tile kernels
    int *hstatus = nullptr;
    long long copies = 0, bytes = 0; // halo exchange counters
};

namespace {

size_t field_bytes(const stokes_slabs *s, int rows) { return (size_t)(rows + 1) * s->pitch * s->esize; }

void free_slab(Slab &b)
{
    void **ps[] = {&b.ec, &b.en, &b.fx, &b.fy, &b.bx, &b.by, &b.ivx, &b.ivy, &b.p,
                   &b.v[0][0], &b.v[0][1], &b.v[1][0], &b.v[1][1]};
    for (void **p : ps) {
        if (*p) cudaFree(*p);
        *p = nullptr;
    }
}

template <typename T>
GridDesc<T> slab_grid(const stokes_slabs *s, const Slab &b)
{
    return make_grid<T>(s->nx, b.R1 - b.R0, s->pitch, s->hx, s->hy);
}

// (Re)allocate every slab's storage for halo H and copy its coefficient rows
// out of the global copies.
template <typename T>
int build(stokes_slabs *s, int H)
{
    const size_t row = (size_t)s->pitch * s->esize;
    if (H != s->halo) {
        for (Slab &b : s->slabs) free_slab(b);
        for (int i = 0; i < s->nslabs; ++i) {
            Slab &b = s->slabs[i];
            slab_rows(s->ny, s->nslabs, i, &b.r0, &b.r1);
            b.R0 = std::max(0, b.r0 - H);
            b.R1 = std::min(s->ny, b.r1 + H);
            const size_t nb = field_bytes(s, b.R1 - b.R0);
            void **ps[] = {&b.ec, &b.en, &b.fx, &b.fy, &b.bx, &b.by, &b.ivx, &b.ivy, &b.p,
                           &b.v[0][0], &b.v[0][1], &b.v[1][0], &b.v[1][1]};
            for (void **p : ps) {
                CK(cudaMalloc(p, nb));
                CK(cudaMemsetAsync(*p, 0, nb, s->stream));
            }
        }
        s->halo = H;
        s->stale = true;
    }
    if (!s->stale) return STOKES_OK;
    for (Slab &b : s->slabs) {
        const int ns = b.R1 - b.R0;
        const GridDesc<T> g = slab_grid<T>(s, b);
        const size_t off = (size_t)b.R0 * row;
        // eta_c rows [R0, R1) and eta_n rows [R0, R1] into the velocity
        // buffers as scratch, then the library copy (boundary nodes of the
        // slab grid zeroed) and 1/diag(M)
        CK(cudaMemcpyAsync(b.v[0][0], (const char *)s->eta_c + off, (size_t)ns * row, cudaMemcpyDeviceToDevice,
                           s->stream));
        CK(cudaMemcpyAsync(b.v[0][1], (const char *)s->eta_n + off, (size_t)(ns + 1) * row, cudaMemcpyDeviceToDevice,
                           s->stream));
        CK(launch_copy_eta<T>(g, (const T *)b.v[0][0], (const T *)b.v[0][1], (T *)b.ec, (T *)b.en, s->stream));
        CK(launch_inv_diag<T>(g, (const T *)b.ec, (const T *)b.en, (T *)b.ivx, (T *)b.ivy, s->stream));
        CK(cudaMemcpyAsync(b.fx, (const char *)s->fx + off, (size_t)ns * row, cudaMemcpyDeviceToDevice, s->stream));
        CK(cudaMemcpyAsync(b.fy, (const char *)s->fy + off, (size_t)(ns + 1) * row, cudaMemcpyDeviceToDevice,
                           s->stream));
    }
    s->stale = false;
    return STOKES_OK;
}

// copy rows [a, b) of a field from slab `src` to slab `dst` (global row
// numbers; both slabs store them)
int copy_rows(stokes_slabs *s, const Slab &src, const void *sp, const Slab &dst, void *dp, int a, int b)
{
    if (b <= a) return STOKES_OK;
    const size_t row = (size_t)s->pitch * s->esize;
    CK(cudaMemcpyAsync((char *)dp + (size_t)(a - dst.R0) * row, (const char *)sp + (size_t)(a - src.R0) * row,
                       (size_t)(b - a) * row, cudaMemcpyDeviceToDevice, s->stream));
    s->copies += 1;
    s->bytes += (long long)((b - a) * row);
    return STOKES_OK;
}

template <typename T>
int smooth_impl(stokes_slabs *s, T *vx, T *vy, const T *p, const stokes_smooth_params *prm)
{
    const int ti = prm->tile_i > 0 ? prm->tile_i : 32, tj = prm->tile_j > 0 ? prm->tile_j : 32;
    const int H = tj + prm->overlap + 1;
    for (int i = 0; i < s->nslabs; ++i) {
        int r0, r1;
        slab_rows(s->ny, s->nslabs, i, &r0, &r1);
        if (r1 - r0 < H + 1) return STOKES_ERR_ARG; // a halo must come from the neighbour's own rows
    }
    int st = build<T>(s, H);
    if (st != STOKES_OK) return st;
    if (prm->sweeps == 0) return STOKES_OK;
    const size_t row = (size_t)s->pitch * s->esize;
    const T omega = (T)prm->omega;
    RasRun run;
    run.allow_tma = true;
    run.pair_mode = 1;
    run.status = s->dstatus;
    run.wait_limit = 2000000000LL;
    // scatter: right-hand side, velocity rows (own and halo) into pair 0, walls into pair 1
    for (Slab &b : s->slabs) {
        const int ns = b.R1 - b.R0;
        const GridDesc<T> g = slab_grid<T>(s, b);
        const size_t off = (size_t)b.R0 * row;
        if (p) {
            CK(cudaMemcpyAsync(b.p, (const char *)p + off, (size_t)ns * row, cudaMemcpyDeviceToDevice, s->stream));
            CK(launch_rhs<T>(g, (const T *)b.fx, (const T *)b.fy, (const T *)b.p, (T *)b.bx, (T *)b.by, s->stream));
        }
        CK(cudaMemcpyAsync(b.v[0][0], (const char *)vx + off, (size_t)ns * row, cudaMemcpyDeviceToDevice, s->stream));
        CK(cudaMemcpyAsync(b.v[0][1], (const char *)vy + off, (size_t)(ns + 1) * row, cudaMemcpyDeviceToDevice,
                           s->stream));
        CK(launch_copy_walls<T>(g, (const T *)b.v[0][0], (const T *)b.v[0][1], (T *)b.v[1][0], (T *)b.v[1][1],
                                s->stream));
    }
    const int n_outer = (prm->sweeps + prm->k - 1) / prm->k;
    int cur = 0;
    for (int t = 0; t < n_outer; ++t) {
        const int ks = (t == n_outer - 1) ? prm->sweeps - (n_outer - 1) * prm->k : prm->k;
        int si = 0, sj = 0;
        if (prm->shift_mode == STOKES_SHIFT_SPLITMIX) {
            si = (int)(splitmix64(prm->seed, 2u * (uint64_t)t) % (uint64_t)ti);
            sj = (int)(splitmix64(prm->seed, 2u * (uint64_t)t + 1u) % (uint64_t)tj);
        } else if (prm->shift_mode == STOKES_SHIFT_LIST) {
            si = prm->shifts[2 * t];
            sj = prm->shifts[2 * t + 1];
            if (si < 0 || si >= ti || sj < 0 || sj >= tj) return STOKES_ERR_ARG;
        }
        // every slab: one outer iteration of the global tiling on its storage
        for (Slab &b : s->slabs) {
            const GridDesc<T> g = slab_grid<T>(s, b);
            Coeffs<T> k;
            k.eta_c = (const T *)b.ec;
            k.eta_n = (const T *)b.en;
            k.bx = (const T *)(p ? b.bx : b.fx);
            k.by = (const T *)(p ? b.by : b.fy);
            k.inv_dx = (const T *)b.ivx;
            k.inv_dy = (const T *)b.ivy;
            // the global cuts sj + m tj in the storage's row numbers
            const int sjs = (int)(((long long)sj - b.R0) % tj + tj) % tj;
            const TileGrid tg = make_tiles(s->nx, b.R1 - b.R0, ti, tj, si, sjs);
            CK(launch_ras<T>(g, k, omega, tg, ks, prm->overlap, (const T *)b.v[cur][0], (const T *)b.v[cur][1],
                             (T *)b.v[cur ^ 1][0], (T *)b.v[cur ^ 1][1], run, s->stream));
        }
        // halo exchange: rows a slab stores but does not own, from the owner
        const int nw = cur ^ 1;
        for (int i = 0; i < s->nslabs; ++i) {
            Slab &b = s->slabs[i];
            if (i > 0) {
                const Slab &lo = s->slabs[i - 1];
                if ((st = copy_rows(s, lo, lo.v[nw][0], b, b.v[nw][0], b.R0, b.r0)) != STOKES_OK) return st;
                if ((st = copy_rows(s, lo, lo.v[nw][1], b, b.v[nw][1], b.R0, b.r0)) != STOKES_OK) return st;
            }
            if (i + 1 < s->nslabs) {
                const Slab &hi = s->slabs[i + 1];
                if ((st = copy_rows(s, hi, hi.v[nw][0], b, b.v[nw][0], b.r1, b.R1)) != STOKES_OK) return st;
                // vy rows r1 .. R1 (row R1 is the storage's last vy row)
                if ((st = copy_rows(s, hi, hi.v[nw][1], b, b.v[nw][1], b.r1, b.R1 + 1)) != STOKES_OK) return st;
            }
        }
        cur = nw;
    }
    // gather the own rows back into the caller's arrays
    for (const Slab &b : s->slabs) {
        const size_t off = (size_t)b.r0 * row, in = (size_t)(b.r0 - b.R0) * row;
        const size_t nb = (size_t)(b.r1 - b.r0) * row;
        CK(cudaMemcpyAsync((char *)vx + off, (const char *)b.v[cur][0] + in, nb, cudaMemcpyDeviceToDevice, s->stream));
        CK(cudaMemcpyAsync((char *)vy + off, (const char *)b.v[cur][1] + in, nb, cudaMemcpyDeviceToDevice, s->stream));
    }
    CK(cudaMemcpyAsync(s->hstatus, s->dstatus, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if (*s->hstatus != 0) {
        CK(cudaMemsetAsync(s->dstatus, 0, sizeof(int), s->stream));
        CK(cudaStreamSynchronize(s->stream));
        return STOKES_ERR_TIMEOUT;
    }
    return STOKES_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

} // namespace

extern "C" {

int stokes_slab_plan(int ny, int nslabs, int tile_j, int overlap, int slab, int out[4])
{
    if (ny < 2 || nslabs < 1 || tile_j < 1 || overlap < 0 || slab < 0 || slab >= nslabs || !out)
        return STOKES_ERR_ARG;
    const int H = tile_j + overlap + 1;
    for (int i = 0; i < nslabs; ++i) {
        int r0, r1;
        slab_rows(ny, nslabs, i, &r0, &r1);
        if (r1 - r0 < H + 1) return STOKES_ERR_ARG;
    }
    int r0, r1;
    slab_rows(ny, nslabs, slab, &r0, &r1);
    out[0] = r0;
    out[1] = r1;
    out[2] = std::max(0, r0 - H);
    out[3] = std::min(ny, r1 + H);
    return STOKES_OK;
}

int stokes_slabs_create(int nx, int ny, double lx, double ly, int dtype, int nslabs, void *cuda_stream,
                        stokes_slabs **out)
{
    if (!out) return STOKES_ERR_ARG;
    *out = nullptr;
    if (nx < 2 || ny < 2 || nx > (1 << 18) || ny > (1 << 18) || !(lx > 0.0) || !(ly > 0.0)) return STOKES_ERR_ARG;
    if (dtype != STOKES_F32 && dtype != STOKES_F64) return STOKES_ERR_ARG;
    if (nslabs < 1 || nslabs > ny / 2) return STOKES_ERR_ARG;
    stokes_slabs *s = new (std::nothrow) stokes_slabs();
    if (!s) return STOKES_ERR_OOM;
    s->nx = nx;
    s->ny = ny;
    s->hx = lx / nx;
    s->hy = ly / ny;
    s->dtype = dtype;
    s->esize = dtype == STOKES_F64 ? 8 : 4;
    s->pitch = ((nx + 1) + 31) / 32 * 32; // the single-context layout
    s->nslabs = nslabs;
    s->stream = (cudaStream_t)cuda_stream;
    s->slabs.resize(nslabs);
    const size_t nb = field_bytes(s, ny);
    cudaError_t e = cudaSuccess;
    void **gs[] = {&s->eta_c, &s->eta_n, &s->fx, &s->fy};
    for (void **p : gs) {
        if (e == cudaSuccess) e = cudaMalloc(p, nb);
        if (e == cudaSuccess) e = cudaMemsetAsync(*p, 0, nb, s->stream);
    }
    if (e == cudaSuccess) e = cudaMalloc(&s->dstatus, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(s->dstatus, 0, sizeof(int), s->stream);
    if (e == cudaSuccess) e = cudaMallocHost(&s->hstatus, sizeof(int));
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        const int st = cuda_fail(e, "stokes_slabs_create");
        stokes_slabs_destroy(s);
        return st;
    }
    *out = s;
    return STOKES_OK;
}

int stokes_slabs_set_viscosity(stokes_slabs *s, const void *eta_c, const void *eta_n)
{
    if (!s || !eta_c || !eta_n) return STOKES_ERR_ARG;
    const size_t nb = field_bytes(s, s->ny);
    CK(cudaMemcpyAsync(s->eta_c, eta_c, nb, cudaMemcpyDeviceToDevice, s->stream));
    CK(cudaMemcpyAsync(s->eta_n, eta_n, nb, cudaMemcpyDeviceToDevice, s->stream));
    s->have_eta = true;
    s->stale = true;
    return STOKES_OK;
}

int stokes_slabs_set_rhs(stokes_slabs *s, const void *fx, const void *fy)
{
    if (!s || !fx || !fy) return STOKES_ERR_ARG;
    // f at the unknowns of the whole grid, zero on walls and padding
    cudaError_t e;
    if (s->dtype == STOKES_F64)
        e = launch_rhs<double>(make_grid<double>(s->nx, s->ny, s->pitch, s->hx, s->hy), (const double *)fx,
                               (const double *)fy, nullptr, (double *)s->fx, (double *)s->fy, s->stream);
    else
        e = launch_rhs<float>(make_grid<float>(s->nx, s->ny, s->pitch, s->hx, s->hy), (const float *)fx,
                              (const float *)fy, nullptr, (float *)s->fx, (float *)s->fy, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "stokes_slabs_set_rhs");
    s->have_f = true;
    s->stale = true;
    return STOKES_OK;
}

int stokes_slabs_smooth(stokes_slabs *s, void *vx, void *vy, const void *p, const stokes_smooth_params *prm)
{
    if (!s || !vx || !vy || !prm) return STOKES_ERR_ARG;
    if (!aligned16(vx) || !aligned16(vy) || !aligned16(p)) return STOKES_ERR_ARG;
    if (prm->variant != STOKES_RAS || prm->sweeps < 0 || prm->k < 1 || prm->overlap < 0 || prm->overlap > 4096 ||
        !(prm->omega > 0.0) || prm->tile_i < 0 || prm->tile_j < 0)
        return STOKES_ERR_ARG;
    if (prm->shift_mode < STOKES_SHIFT_NONE || prm->shift_mode > STOKES_SHIFT_LIST) return STOKES_ERR_ARG;
    if (prm->shift_mode == STOKES_SHIFT_LIST && prm->sweeps > 0 && !prm->shifts) return STOKES_ERR_ARG;
    const int ti = prm->tile_i > 0 ? prm->tile_i : 32, tj = prm->tile_j > 0 ? prm->tile_j : 32;
    if (ras_smem_bytes(s->nx, s->ny, ti, tj, prm->overlap, s->esize) > (size_t)ras_max_smem()) return STOKES_ERR_ARG;
    if (!s->have_eta || !s->have_f) return STOKES_ERR_STATE;
    if (s->dtype == STOKES_F64) return smooth_impl<double>(s, (double *)vx, (double *)vy, (const double *)p, prm);
    return smooth_impl<float>(s, (float *)vx, (float *)vy, (const float *)p, prm);
}

int stokes_slabs_exchanges(const stokes_slabs *s, long long *copies, long long *bytes)
{
    if (!s) return STOKES_ERR_ARG;
    if (copies) *copies = s->copies;
    if (bytes) *bytes = s->bytes;
    return STOKES_OK;
}

int stokes_slabs_destroy(stokes_slabs *s)
{
    if (!s) return STOKES_ERR_ARG;
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (Slab &b : s->slabs) free_slab(b);
    void *gs[] = {s->eta_c, s->eta_n, s->fx, s->fy, s->dstatus};
    for (void *p : gs)
        if (p) cudaFree(p);
    if (s->hstatus) cudaFreeHost(s->hstatus);
    delete s;
    return STOKES_OK;
}

} // extern "C"
