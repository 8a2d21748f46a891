// stokes_api.cu -- the C ABI of libstokes (include/stokes.h): context
// management, argument checks, the smoother schedules (sweep loops, RAS
// outer iterations with their tile shifts, ping-pong buffers) and the energy
// norm.  Every arithmetic step runs in the kernels of stencil_kernels.cu and
// ras_kernels.cu.
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/stokes.h"
#include "internal.h"
#include "mg.h"

using namespace stokes;

namespace {

thread_local char g_cuda_err[256] = "";

int cuda_fail(cudaError_t e, const char *where)
{
    std::snprintf(g_cuda_err, sizeof g_cuda_err, "%s: %s", where, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? STOKES_ERR_OOM : STOKES_ERR_CUDA;
}

#define CK(call)                                                                                                   \
    do {                                                                                                           \
        cudaError_t e_ = (call);                                                                                   \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);                                                        \
    } while (0)

} // namespace

uint64_t stokes::splitmix64(uint64_t seed, uint64_t c)
{
    // state after c+1 golden-gamma increments, then the mix64 finaliser
    uint64_t z = seed + (c + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Launch counts per kernel class and, when enabled, CUDA-event timing of
// every launch group.
struct Profiler {
    struct Rec {
        int kind;
        cudaEvent_t a, b;
    };
    bool timing = false;
    long long kernels[STOKES_K_COUNT] = {};
    long long groups[STOKES_K_COUNT] = {};
    double ms[STOKES_K_COUNT] = {};
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
};

struct stokes_ctx {
    int nx, ny, dtype, pitch, device;
    double lx, ly, hx, hy;
    size_t elems, esize;
    cudaStream_t stream;
    void *eta_c = nullptr, *eta_n = nullptr, *fx = nullptr, *fy = nullptr;
    void *bx = nullptr, *by = nullptr, *sx = nullptr, *sy = nullptr;
    void *ivx = nullptr, *ivy = nullptr; // 1/diag(M) (FP64 contexts: the FP64 pipe is the bottleneck)
    double *partials = nullptr, *dsum = nullptr, *hsum = nullptr;
    bool have_eta = false, have_f = false;
    int *dstatus = nullptr;              // device status word of the bounded waits
    int *hstatus = nullptr;              // pinned host copy
    bool use_tma = true;                 // STOKES_OPT_USE_TMA
    long long wait_limit = 2000000000LL; // STOKES_OPT_WAIT_LIMIT_CYCLES (about 1 s)
    MgHierarchy *mg = nullptr;
    Profiler prof;
};

namespace {

int alloc_field(stokes_ctx *c, void **p)
{
    CK(cudaMalloc(p, c->elems * c->esize));
    CK(cudaMemsetAsync(*p, 0, c->elems * c->esize, c->stream));
    return STOKES_OK;
}

cudaError_t prof_event(stokes_ctx *c, cudaEvent_t *e)
{
    if (!c->prof.pool.empty()) {
        *e = c->prof.pool.back();
        c->prof.pool.pop_back();
        return cudaSuccess;
    }
    return cudaEventCreate(e);
}

// Fold completed timing records into the per-class totals (waits for them).
int prof_flush(stokes_ctx *c)
{
    for (const Profiler::Rec &r : c->prof.pending) {
        float ms = 0.f;
        CK(cudaEventSynchronize(r.b));
        CK(cudaEventElapsedTime(&ms, r.a, r.b));
        c->prof.ms[r.kind] += ms;
        c->prof.groups[r.kind] += 1;
        c->prof.pool.push_back(r.a);
        c->prof.pool.push_back(r.b);
    }
    c->prof.pending.clear();
    return STOKES_OK;
}

// Launch a group of `nk` kernels of class `kind` through `f`, counting them
// and, with timing on, bracketing them with events on the context stream.
template <class F>
int run(stokes_ctx *c, int kind, int nk, F &&f)
{
    cudaEvent_t a = nullptr, b = nullptr;
    if (c->prof.timing) {
        if (c->prof.pending.size() >= 8192) {
            int st = prof_flush(c);
            if (st != STOKES_OK) return st;
        }
        CK(prof_event(c, &a));
        CK(prof_event(c, &b));
        CK(cudaEventRecord(a, c->stream));
    }
    const cudaError_t e = f();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    if (c->prof.timing) {
        CK(cudaEventRecord(b, c->stream));
        c->prof.pending.push_back({kind, a, b});
    }
    c->prof.kernels[kind] += nk;
    return STOKES_OK;
}

#define RUN(kind, nk, expr)                                                                                        \
    do {                                                                                                           \
        const int st_ = run(c, (kind), (nk), [&]() { return (expr); });                                            \
        if (st_ != STOKES_OK) return st_;                                                                          \
    } while (0)

template <typename T>
GridDesc<T> grid_of(const stokes_ctx *c)
{
    return make_grid<T>(c->nx, c->ny, c->pitch, c->hx, c->hy);
}

template <typename T>
Coeffs<T> coeffs_of(const stokes_ctx *c)
{
    Coeffs<T> k;
    k.eta_c = (const T *)c->eta_c;
    k.eta_n = (const T *)c->eta_n;
    k.bx = (const T *)c->bx;
    k.by = (const T *)c->by;
    k.inv_dx = (const T *)c->ivx;
    k.inv_dy = (const T *)c->ivy;
    return k;
}

int check_smooth_params(const stokes_ctx *c, const stokes_smooth_params *p, int *ti, int *tj)
{
    if (!p || p->sweeps < 0 || !(p->omega > 0.0)) return STOKES_ERR_ARG;
    if (p->variant < STOKES_JACOBI || p->variant > STOKES_RAS) return STOKES_ERR_ARG;
    *ti = p->tile_i > 0 ? p->tile_i : 32;
    *tj = p->tile_j > 0 ? p->tile_j : 32;
    if (p->variant == STOKES_RAS || p->variant == STOKES_JACOBI_BLOCKED) {
        const int k = p->variant == STOKES_RAS ? p->k : 1;
        const int o = p->variant == STOKES_RAS ? p->overlap : 0;
        if (k < 1 || o < 0 || o > 4096) return STOKES_ERR_ARG;
        if (ras_smem_bytes(c->nx, c->ny, *ti, *tj, o, c->esize) > (size_t)ras_max_smem()) return STOKES_ERR_ARG;
        if (p->variant == STOKES_RAS) {
            if (p->shift_mode < STOKES_SHIFT_NONE || p->shift_mode > STOKES_SHIFT_LIST) return STOKES_ERR_ARG;
            if (p->shift_mode == STOKES_SHIFT_LIST && p->sweeps > 0 && !p->shifts) return STOKES_ERR_ARG;
        }
    }
    return STOKES_OK;
}

RasRun run_opts(const stokes_ctx *c)
{
    RasRun r;
    r.allow_tma = c->use_tma;
    r.status = c->dstatus;
    r.wait_limit = c->wait_limit;
    return r;
}

// Reads (and clears) the device status word; synchronises the stream.
int device_status(stokes_ctx *c)
{
    CK(cudaMemcpyAsync(c->hstatus, c->dstatus, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (*c->hstatus != 0) {
        CK(cudaMemsetAsync(c->dstatus, 0, sizeof(int), c->stream));
        CK(cudaStreamSynchronize(c->stream));
        return STOKES_ERR_TIMEOUT;
    }
    return STOKES_OK;
}

// Runs the smoother of `p` on (vx, vy) with b already formed.
template <typename T>
int smooth_impl(stokes_ctx *c, T *vx, T *vy, const stokes_smooth_params *p, int ti, int tj)
{
    const GridDesc<T> g = grid_of<T>(c);
    const Coeffs<T> k = coeffs_of<T>(c);
    const T omega = (T)p->omega;
    cudaStream_t s = c->stream;
    if (p->sweeps == 0) return STOKES_OK;
    if (p->variant == STOKES_RBGS) {
        for (int it = 0; it < p->sweeps; ++it) RUN(STOKES_K_RBGS, 4, launch_rbgs_sweep<T>(g, k, omega, vx, vy, s));
        return STOKES_OK;
    }
    // ping-pong between the caller's buffers (A) and the library's (B)
    T *ax = vx, *ay = vy, *bxp = (T *)c->sx, *byp = (T *)c->sy;
    RUN(STOKES_K_COPY, 1, launch_copy_walls<T>(g, vx, vy, bxp, byp, s));
    int passes = 0;
    if (p->variant == STOKES_RAS) {
        const int n_outer = (p->sweeps + p->k - 1) / p->k;
        for (int t = 0; t < n_outer; ++t) {
            const int ks = (t == n_outer - 1) ? p->sweeps - (n_outer - 1) * p->k : p->k;
            int si = 0, sj = 0;
            if (p->shift_mode == STOKES_SHIFT_SPLITMIX) {
                si = (int)(splitmix64(p->seed, 2u * (uint64_t)t) % (uint64_t)ti);
                sj = (int)(splitmix64(p->seed, 2u * (uint64_t)t + 1u) % (uint64_t)tj);
            } else if (p->shift_mode == STOKES_SHIFT_LIST) {
                si = p->shifts[2 * t];
                sj = p->shifts[2 * t + 1];
                if (si < 0 || si >= ti || sj < 0 || sj >= tj) return STOKES_ERR_ARG;
            }
            const TileGrid tg = make_tiles(c->nx, c->ny, ti, tj, si, sj);
            RUN(STOKES_K_RAS, 1, launch_ras<T>(g, k, omega, tg, ks, p->overlap, ax, ay, bxp, byp, run_opts(c), s));
            T *t0 = ax; ax = bxp; bxp = t0;
            T *t1 = ay; ay = byp; byp = t1;
            ++passes;
        }
    } else {
        for (int it = 0; it < p->sweeps; ++it) {
            if (p->variant == STOKES_JACOBI_BLOCKED) {
                const TileGrid tg = make_tiles(c->nx, c->ny, ti, tj, 0, 0);
                RUN(STOKES_K_RAS, 1, launch_ras<T>(g, k, omega, tg, 1, 0, ax, ay, bxp, byp, run_opts(c), s));
            } else {
                RUN(STOKES_K_JACOBI, p->variant == STOKES_JACOBI_FUSED ? 1 : 2,
                    launch_jacobi<T>(g, k, omega, ax, ay, bxp, byp, p->variant == STOKES_JACOBI_FUSED, s));
            }
            T *t0 = ax; ax = bxp; bxp = t0;
            T *t1 = ay; ay = byp; byp = t1;
            ++passes;
        }
    }
    if (passes & 1) RUN(STOKES_K_COPY, 1, launch_copy_velocity<T>(g, ax, ay, vx, vy, s));
    return STOKES_OK;
}

template <typename T>
int energy_impl(stokes_ctx *c, const T *vx, const T *vy, const T *p, double out[3])
{
    const GridDesc<T> g = grid_of<T>(c);
    RUN(STOKES_K_ENERGY, 2,
        launch_energy<T>(g, (const T *)c->eta_c, (const T *)c->eta_n, (const T *)c->ivx, (const T *)c->ivy,
                         (const T *)c->fx, (const T *)c->fy, p, vx, vy, c->partials, c->dsum, c->stream));
    CK(cudaMemcpyAsync(c->hsum, c->dsum, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    const int st = device_status(c);
    std::memcpy(out, c->hsum, 3 * sizeof(double));
    return st;
}

} // namespace

// ---------------------------------------------------------------------------
extern "C" {

const char *stokes_strerror(int status)
{
    switch (status) {
    case STOKES_OK: return "ok";
    case STOKES_ERR_ARG: return "invalid argument";
    case STOKES_ERR_CUDA: return "CUDA error";
    case STOKES_ERR_OOM: return "out of device memory";
    case STOKES_ERR_DIVERGED: return "diverged (NaN/Inf or residual growth)";
    case STOKES_ERR_TIMEOUT: return "device-side wait timed out";
    case STOKES_ERR_NOT_CONVERGED: return "not converged within max_cycles";
    case STOKES_ERR_STATE: return "call out of order";
    default: return "unknown status";
    }
}

const char *stokes_last_cuda_error(void) { return g_cuda_err; }

int stokes_create(int nx, int ny, double lx, double ly, int dtype, void *cuda_stream, stokes_ctx **out)
{
    if (!out) return STOKES_ERR_ARG;
    *out = nullptr;
    if (nx < 2 || ny < 2 || nx > (1 << 20) || ny > (1 << 20) || !(lx > 0.0) || !(ly > 0.0)) return STOKES_ERR_ARG;
    if (dtype != STOKES_F32 && dtype != STOKES_F64) return STOKES_ERR_ARG;
    stokes_ctx *c = new (std::nothrow) stokes_ctx();
    if (!c) return STOKES_ERR_OOM;
    c->nx = nx;
    c->ny = ny;
    c->lx = lx;
    c->ly = ly;
    c->hx = lx / nx;
    c->hy = ly / ny;
    c->dtype = dtype;
    c->esize = dtype == STOKES_F64 ? 8 : 4;
    // rows padded to a multiple of 32 elements (128 B in FP32, 256 B in FP64)
    c->pitch = ((nx + 1) + 31) / 32 * 32;
    c->elems = (size_t)(ny + 1) * (size_t)c->pitch;
    c->stream = (cudaStream_t)cuda_stream;
    cudaGetDevice(&c->device);
    int st = STOKES_OK;
    void **fields[] = {&c->eta_c, &c->eta_n, &c->fx, &c->fy, &c->bx, &c->by, &c->sx, &c->sy};
    for (void **f : fields)
        if ((st = alloc_field(c, f)) != STOKES_OK) break;
    if (st == STOKES_OK && dtype == STOKES_F64) {
        st = alloc_field(c, &c->ivx);
        if (st == STOKES_OK) st = alloc_field(c, &c->ivy);
    }
    if (st == STOKES_OK) {
        cudaError_t e = cudaMalloc(&c->partials, (size_t)energy_partials() * 3 * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&c->dsum, 3 * sizeof(double));
        if (e == cudaSuccess) e = cudaMallocHost(&c->hsum, 3 * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&c->dstatus, sizeof(int));
        if (e == cudaSuccess) e = cudaMemsetAsync(c->dstatus, 0, sizeof(int), c->stream);
        if (e == cudaSuccess) e = cudaMallocHost(&c->hstatus, sizeof(int));
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "stokes_create");
    }
    if (st != STOKES_OK) {
        stokes_destroy(c);
        return st;
    }
    *out = c;
    return STOKES_OK;
}

int stokes_destroy(stokes_ctx *c)
{
    if (!c) return STOKES_OK;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    mg_destroy(c->mg);
    prof_flush(c);
    for (cudaEvent_t e : c->prof.pool) cudaEventDestroy(e);
    void *fields[] = {c->eta_c, c->eta_n, c->fx, c->fy, c->bx, c->by, c->sx, c->sy, c->ivx, c->ivy, c->partials,
                      c->dsum, c->dstatus};
    for (void *f : fields)
        if (f) cudaFree(f);
    if (c->hsum) cudaFreeHost(c->hsum);
    if (c->hstatus) cudaFreeHost(c->hstatus);
    delete c;
    return STOKES_OK;
}

int stokes_get_layout(const stokes_ctx *c, int field, int *rows, int *cols, int *pitch_elems, size_t *alloc_elems)
{
    if (!c) return STOKES_ERR_ARG;
    int r, q;
    switch (field) {
    case STOKES_FIELD_VX: r = c->ny; q = c->nx + 1; break;
    case STOKES_FIELD_VY: r = c->ny + 1; q = c->nx; break;
    case STOKES_FIELD_P:
    case STOKES_FIELD_ETA_C: r = c->ny; q = c->nx; break;
    case STOKES_FIELD_ETA_N: r = c->ny + 1; q = c->nx + 1; break;
    default: return STOKES_ERR_ARG;
    }
    if (rows) *rows = r;
    if (cols) *cols = q;
    if (pitch_elems) *pitch_elems = c->pitch;
    if (alloc_elems) *alloc_elems = c->elems;
    return STOKES_OK;
}

int stokes_set_viscosity(stokes_ctx *c, const void *eta_c, const void *eta_n)
{
    if (!c || !eta_c || !eta_n) return STOKES_ERR_ARG;
    if (c->dtype == STOKES_F64) {
        RUN(STOKES_K_COPY, 1, launch_copy_eta<double>(grid_of<double>(c), (const double *)eta_c, (const double *)eta_n,
                                   (double *)c->eta_c, (double *)c->eta_n, c->stream));
        RUN(STOKES_K_COPY, 1,
            launch_inv_diag<double>(grid_of<double>(c), (const double *)c->eta_c, (const double *)c->eta_n,
                                    (double *)c->ivx, (double *)c->ivy, c->stream));
    }
    else
        RUN(STOKES_K_COPY, 1, launch_copy_eta<float>(grid_of<float>(c), (const float *)eta_c, (const float *)eta_n, (float *)c->eta_c,
                                  (float *)c->eta_n, c->stream));
    c->have_eta = true;
    mg_invalidate(c->mg);
    return STOKES_OK;
}

int stokes_set_rhs(stokes_ctx *c, const void *fx, const void *fy)
{
    if (!c || !fx || !fy) return STOKES_ERR_ARG;
    const size_t bytes = c->elems * c->esize;
    CK(cudaMemcpyAsync(c->fx, fx, bytes, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(c->fy, fy, bytes, cudaMemcpyDeviceToDevice, c->stream));
    c->have_f = true;
    return STOKES_OK;
}

int stokes_apply_operator(stokes_ctx *c, const void *vx, const void *vy, const void *p, void *out_x, void *out_y)
{
    if (!c || !vx || !vy || !out_x || !out_y) return STOKES_ERR_ARG;
    if (!c->have_eta) return STOKES_ERR_STATE;
    if (c->dtype == STOKES_F64)
        RUN(STOKES_K_APPLY, 1, launch_apply<double>(grid_of<double>(c), (const double *)c->eta_c, (const double *)c->eta_n,
                                (const double *)vx, (const double *)vy, (const double *)p, (double *)out_x,
                                (double *)out_y, c->stream));
    else
        RUN(STOKES_K_APPLY, 1, launch_apply<float>(grid_of<float>(c), (const float *)c->eta_c, (const float *)c->eta_n,
                               (const float *)vx, (const float *)vy, (const float *)p, (float *)out_x,
                               (float *)out_y, c->stream));
    return STOKES_OK;
}

int stokes_smooth(stokes_ctx *c, void *vx, void *vy, const void *p, const stokes_smooth_params *params)
{
    if (!c || !vx || !vy) return STOKES_ERR_ARG;
    int ti, tj, st = check_smooth_params(c, params, &ti, &tj);
    if (st != STOKES_OK) return st;
    if (!c->have_eta || !c->have_f) return STOKES_ERR_STATE;
    if (c->dtype == STOKES_F64) {
        RUN(STOKES_K_RHS, 1, launch_rhs<double>(grid_of<double>(c), (const double *)c->fx, (const double *)c->fy, (const double *)p,
                              (double *)c->bx, (double *)c->by, c->stream));
        return smooth_impl<double>(c, (double *)vx, (double *)vy, params, ti, tj);
    }
    RUN(STOKES_K_RHS, 1, launch_rhs<float>(grid_of<float>(c), (const float *)c->fx, (const float *)c->fy, (const float *)p,
                         (float *)c->bx, (float *)c->by, c->stream));
    return smooth_impl<float>(c, (float *)vx, (float *)vy, params, ti, tj);
}

int stokes_residual_energy_norm(stokes_ctx *c, const void *vx, const void *vy, const void *p, double out[3])
{
    if (!c || !vx || !vy || !out) return STOKES_ERR_ARG;
    if (!c->have_eta || !c->have_f) return STOKES_ERR_STATE;
    if (c->dtype == STOKES_F64) return energy_impl<double>(c, (const double *)vx, (const double *)vy, (const double *)p, out);
    return energy_impl<float>(c, (const float *)vx, (const float *)vy, (const float *)p, out);
}

int stokes_vcycle(stokes_ctx *c, void *vx, void *vy, const void *p, const stokes_mg_params *params,
                  double *final_rel_resid, int *cycles)
{
    if (!c || !vx || !vy || !params) return STOKES_ERR_ARG;
    if (!c->have_eta || !c->have_f) return STOKES_ERR_STATE;
    return STOKES_ERR_STATE; // multigrid solve: not yet available
}

int stokes_set_option(stokes_ctx *c, int option, long long value)
{
    if (!c) return STOKES_ERR_ARG;
    switch (option) {
    case STOKES_OPT_USE_TMA: c->use_tma = value != 0; return STOKES_OK;
    case STOKES_OPT_WAIT_LIMIT_CYCLES: c->wait_limit = value; return STOKES_OK;
    default: return STOKES_ERR_ARG;
    }
}

int stokes_synchronize(stokes_ctx *c)
{
    if (!c) return STOKES_ERR_ARG;
    return device_status(c);
}

int stokes_profile_reset(stokes_ctx *c, int enable_timing)
{
    if (!c) return STOKES_ERR_ARG;
    int st = prof_flush(c);
    if (st != STOKES_OK) return st;
    for (int k = 0; k < STOKES_K_COUNT; ++k) {
        c->prof.kernels[k] = 0;
        c->prof.groups[k] = 0;
        c->prof.ms[k] = 0.0;
    }
    c->prof.timing = enable_timing != 0;
    return STOKES_OK;
}

int stokes_profile_read(stokes_ctx *c, int kind, long long *kernels, long long *groups, double *total_ms)
{
    if (!c || kind < 0 || kind >= STOKES_K_COUNT) return STOKES_ERR_ARG;
    CK(cudaStreamSynchronize(c->stream));
    int st = prof_flush(c);
    if (st != STOKES_OK) return st;
    if (kernels) *kernels = c->prof.kernels[kind];
    if (groups) *groups = c->prof.groups[kind];
    if (total_ms) *total_ms = c->prof.ms[kind];
    return STOKES_OK;
}

} // extern "C"
