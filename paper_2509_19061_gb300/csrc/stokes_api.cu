// stokes_api.cu -- the C ABI of libstokes (include/stokes.h): context
// management, argument checks, the smoother schedules (sweep loops, RAS
// outer iterations with their tile shifts, ping-pong buffers) and the energy
// norm.  Every arithmetic step runs in the kernels of stencil_kernels.cu and
// ras_kernels.cu.
#include <algorithm>
#include <cmath>
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
} // namespace

int stokes::cuda_fail(cudaError_t e, const char *where)
{
    std::snprintf(g_cuda_err, sizeof g_cuda_err, "%s: %s", where, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? STOKES_ERR_OOM : STOKES_ERR_CUDA;
}

namespace {

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
    void *sx2 = nullptr, *sy2 = nullptr; // second scratch pair (allocated by the first odd-pass smoothing)
    void *ivx = nullptr, *ivy = nullptr; // 1/diag(M), read by the tile kernels and the energy sums
    // flux coefficients 2 eta_c / hx^2, 2 eta_c / hy^2 of the outer operator
    // apply, formed for viscosity version coef_version (eta_version counts the
    // viscosity changes)
    void *cax = nullptr, *cay = nullptr;
    long long eta_version = 0, coef_version = -1;
    void *eta_c0 = nullptr, *eta_n0 = nullptr; // the caller's viscosity during a continuation
    double *uz_partials = nullptr, *uz_scal = nullptr; // Uzawa reductions; uz_scal: [eta_min, sum]
    std::vector<void *> aa;              // Anderson history: (depth+1) x (F, r) x 3 fields, then x_old (3)
    double *aa_partials = nullptr, *aa_out = nullptr, *aa_hout = nullptr;
    double *partials = nullptr, *dsum = nullptr, *hsum = nullptr;
    bool have_eta = false, have_f = false;
    int *dstatus = nullptr;              // device status word of the bounded waits
    int *hstatus = nullptr;              // pinned host copy
    bool use_tma = true;                 // STOKES_OPT_USE_TMA
    int pair_mode = 1;                   // STOKES_OPT_PAIRED
    long long wait_limit = 2000000000LL; // STOKES_OPT_WAIT_LIMIT_CYCLES (about 1 s)
    MgHierarchy *mg = nullptr;
    Profiler prof;
    // outer solve: work vectors r, z, p, q (x and y each), reduction buffers,
    // and the preconditioner z = B r as a CUDA graph replayed on gstream
    void *kw[8] = {};
    void *iw[10] = {};                   // inner-precision r, z, p, q, e (x, y) of the refinement mode
    int iw_dtype = -1;
    double *kpartials = nullptr, *kout = nullptr, *hout = nullptr;
    cudaStream_t gstream = nullptr;
    cudaEvent_t gev[2] = {nullptr, nullptr};
    cudaGraphExec_t gexec = nullptr;
    const void *gz[2] = {nullptr, nullptr}; // where the captured V-cycle leaves z (inner precision, krylov = 1)
    unsigned char gkey[sizeof(stokes_mg_params)] = {};
    long long gkernels[STOKES_K_COUNT] = {};
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
    // the register tile kernels read 1/diag(M) instead of recomputing it
    k.inv_dx = (const T *)c->ivx;
    k.inv_dy = (const T *)c->ivy;
    return k;
}

int check_smooth_params(int nx, int ny, size_t esize, const stokes_smooth_params *p, int *ti, int *tj)
{
    if (!p || p->sweeps < 0 || !(p->omega > 0.0)) return STOKES_ERR_ARG;
    if (p->variant < STOKES_JACOBI || p->variant > STOKES_RAS) return STOKES_ERR_ARG;
    *ti = p->tile_i > 0 ? p->tile_i : 32;
    *tj = p->tile_j > 0 ? p->tile_j : 32;
    if (p->variant == STOKES_RAS || p->variant == STOKES_JACOBI_BLOCKED) {
        const int k = p->variant == STOKES_RAS ? p->k : 1;
        const int o = p->variant == STOKES_RAS ? p->overlap : 0;
        if (k < 1 || o < 0 || o > 4096) return STOKES_ERR_ARG;
        if (ras_smem_bytes(nx, ny, *ti, *tj, o, esize) > (size_t)ras_max_smem()) return STOKES_ERR_ARG;
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
    r.pair_mode = c->pair_mode;
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

// the context as a launch hook: counts launches, times them when enabled
struct CtxHook : LaunchHook {
    stokes_ctx *c;
    explicit CtxHook(stokes_ctx *cc) : c(cc) {}
    int run(int kind, int nk, const std::function<cudaError_t()> &launch) override
    {
        return ::run(c, kind, nk, launch);
    }
};

SmoothSpec spec_of(const stokes_smooth_params *p, int ti, int tj)
{
    SmoothSpec s;
    s.variant = p->variant;
    s.sweeps = p->sweeps;
    s.ti = ti;
    s.tj = tj;
    s.k = p->k;
    s.overlap = p->overlap;
    s.shift_mode = p->shift_mode;
    s.omega = p->omega;
    s.seed = p->seed;
    s.shifts = p->shifts;
    return s;
}

// Runs the smoother of `p` on (vx, vy) with b already formed.
// without a pressure b = f: the smoothers read f directly (no b = f - G p pass)
template <typename T>
int smooth_impl(stokes_ctx *c, T *vx, T *vy, const stokes_smooth_params *p, int ti, int tj, bool b_is_f)
{
    CtxHook hook(c);
    Coeffs<T> k = coeffs_of<T>(c);
    if (b_is_f) {
        k.bx = (const T *)c->fx;
        k.by = (const T *)c->fy;
    }
    const SmoothSpec spec = spec_of(p, ti, tj);
    const int n_pass = smooth_passes(spec);
    if (n_pass >= 3 && (n_pass & 1) && !c->sx2) { // second scratch pair: odd pass counts end in place
        int st = alloc_field(c, &c->sx2);
        if (st == STOKES_OK) st = alloc_field(c, &c->sy2);
        if (st != STOKES_OK) return st;
    }
    return smooth_buffers<T>(grid_of<T>(c), k, vx, vy, (T *)c->sx, (T *)c->sy, spec, run_opts(c), c->stream, hook,
                             nullptr, (T *)c->sx2, (T *)c->sy2);
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

// counts the kernels of a launch sequence without timing it (graph capture)
struct CountHook : LaunchHook {
    long long k[STOKES_K_COUNT] = {};
    int run(int kind, int nk, const std::function<cudaError_t()> &launch) override
    {
        const cudaError_t e = launch();
        if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
        k[kind] += nk;
        return STOKES_OK;
    }
};

int check_mg_params(const stokes_ctx *c, const stokes_mg_params *p)
{
    if (!p || p->levels < 1 || p->coarsest < 2 || p->nu_pre < 0 || p->nu_post < 0 || !(p->nu_growth > 0.0) ||
        p->nu_max < 0 || p->max_cycles < 0 || !(p->tol >= 0.0))
        return STOKES_ERR_ARG;
    if (p->inner_dtype != STOKES_F32 && p->inner_dtype != STOKES_F64) return STOKES_ERR_ARG;
    if (p->krylov < 0 || p->krylov > 2) return STOKES_ERR_ARG;
    if (p->krylov == 2 && p->inner_its < 1) return STOKES_ERR_ARG;
    stokes_smooth_params sm = p->smoother;
    sm.sweeps = 0;
    sm.shift_mode = STOKES_SHIFT_SPLITMIX;
    sm.shifts = nullptr;
    if (sm.variant == STOKES_MIXED) sm.variant = STOKES_RAS; // its coarse levels use the RAS parameters
    int ti, tj;
    // the window must fit on the finest level in the inner precision
    return check_smooth_params(c->nx, c->ny, p->inner_dtype == STOKES_F64 ? 8 : 4, &sm, &ti, &tj);
}

MgOuter outer_of(const stokes_ctx *c)
{
    MgOuter o;
    o.nx = c->nx;
    o.ny = c->ny;
    o.pitch = c->pitch;
    o.dtype = c->dtype;
    o.hx = c->hx;
    o.hy = c->hy;
    o.eta_c = c->eta_c;
    o.eta_n = c->eta_n;
    o.bx = c->bx;
    o.by = c->by;
    return o;
}

// work vectors of the outer solve, allocated on first use
// The flux coefficients of the current viscosity (allocated on first use).
template <typename T>
int ensure_coef(stokes_ctx *c, const KrylovView &kv)
{
    if (!c->cax) {
        int st = alloc_field(c, &c->cax);
        if (st == STOKES_OK) st = alloc_field(c, &c->cay);
        if (st != STOKES_OK) return st;
        c->coef_version = -1;
    }
    if (c->coef_version != c->eta_version) {
        RUN(STOKES_K_COPY, 1, kry_coef<T>(kv, grid_of<T>(c), (const T *)c->eta_c, (T *)c->cax, (T *)c->cay, c->stream));
        c->coef_version = c->eta_version;
    }
    return STOKES_OK;
}

int ensure_work(stokes_ctx *c)
{
    if (c->kw[0]) return STOKES_OK;
    for (void *&w : c->kw) {
        const int st = alloc_field(c, &w);
        if (st != STOKES_OK) return st;
    }
    CK(cudaMalloc(&c->kpartials, (size_t)krylov_partials() * 2 * sizeof(double)));
    CK(cudaMalloc(&c->kout, 2 * sizeof(double)));
    CK(cudaMallocHost(&c->hout, 2 * sizeof(double)));
    return STOKES_OK;
}

// Inner-precision work vectors of the refinement mode (krylov = 2).
int ensure_inner_work(stokes_ctx *c, int dtype)
{
    if (c->iw[0] && c->iw_dtype == dtype) return STOKES_OK;
    for (void *&w : c->iw)
        if (w) {
            cudaFree(w);
            w = nullptr;
        }
    const size_t es = dtype == STOKES_F64 ? 8 : 4;
    for (void *&w : c->iw) {
        CK(cudaMalloc(&w, c->elems * es));
        CK(cudaMemsetAsync(w, 0, c->elems * es, c->stream));
    }
    c->iw_dtype = dtype;
    return STOKES_OK;
}

// (Re)capture the preconditioner z = B r (fixed work buffers) for these
// parameters: on the outer work vectors, or on the inner-precision ones in
// the refinement mode.
int ensure_graph(stokes_ctx *c, const stokes_mg_params *p)
{
    if (c->gexec && std::memcmp(p, c->gkey, sizeof *p) == 0) return STOKES_OK;
    if (p->krylov == 2) {
        const int st = ensure_inner_work(c, p->inner_dtype);
        if (st != STOKES_OK) return st;
    }
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    if (!c->gstream) {
        CK(cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&c->gev[0], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&c->gev[1], cudaEventDisableTiming));
    }
    CountHook hook;
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal));
    const bool inner = p->krylov == 2;
    // flexible CG (krylov = 1) writes r in the inner precision itself and
    // reads z where the V-cycle leaves it: no casts in the graph
    const bool direct = p->krylov == 1;
    const int st = direct ? mg_enqueue_precond(c->mg, c->dtype, nullptr, nullptr, nullptr, nullptr, p, run_opts(c),
                                               c->gstream, hook)
                          : mg_enqueue_precond(c->mg, inner ? p->inner_dtype : c->dtype, inner ? c->iw[0] : c->kw[0],
                                               inner ? c->iw[1] : c->kw[1], inner ? c->iw[2] : c->kw[2],
                                               inner ? c->iw[3] : c->kw[3], p, run_opts(c), c->gstream, hook);
    const cudaError_t e = cudaStreamEndCapture(c->gstream, &graph);
    if (st == STOKES_OK && direct) mg_result(c->mg, &c->gz[0], &c->gz[1]);
    if (st != STOKES_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    const cudaError_t ei = cudaGraphInstantiate(&c->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        c->gexec = nullptr;
        return cuda_fail(ei, "cudaGraphInstantiate");
    }
    std::memcpy(c->gkey, p, sizeof *p);
    for (int k = 0; k < STOKES_K_COUNT; ++k) c->gkernels[k] = hook.k[k];
    return STOKES_OK;
}

// one replay of the preconditioner, ordered after the context stream's work
int replay_graph(stokes_ctx *c)
{
    CK(cudaEventRecord(c->gev[0], c->stream));
    CK(cudaStreamWaitEvent(c->gstream, c->gev[0], 0));
    CK(cudaGraphLaunch(c->gexec, c->gstream));
    CK(cudaEventRecord(c->gev[1], c->gstream));
    CK(cudaStreamWaitEvent(c->stream, c->gev[1], 0));
    for (int k = 0; k < STOKES_K_COUNT; ++k) c->prof.kernels[k] += c->gkernels[k];
    return STOKES_OK;
}

// the two reduction results, synchronising the context stream
int read2(stokes_ctx *c, double *a, double *b)
{
    CK(cudaMemcpyAsync(c->hout, c->kout, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    const int st = device_status(c);
    if (a) *a = c->hout[0];
    if (b) *b = c->hout[1];
    return st;
}

// Outer solve of M v = f - G p (Sec. 3.2): flexible CG or defect correction
// with the V-cycle preconditioner z = B r.
template <typename T>
int vcycle_impl(stokes_ctx *c, T *vx, T *vy, const T *p, const stokes_mg_params *params, double *final_e,
                int *cycles)
{
    const GridDesc<T> g = grid_of<T>(c);
    RUN(STOKES_K_RHS, 1, launch_rhs<T>(g, (const T *)c->fx, (const T *)c->fy, p, (T *)c->bx, (T *)c->by, c->stream));
    int st = mg_ensure(&c->mg, outer_of(c), params, c->stream);
    if (st == STOKES_OK) st = ensure_work(c);
    if (st == STOKES_OK) st = ensure_graph(c, params);
    if (st != STOKES_OK) return st;
    T *rx = (T *)c->kw[0], *ry = (T *)c->kw[1], *zx = (T *)c->kw[2], *zy = (T *)c->kw[3];
    T *px = (T *)c->kw[4], *py = (T *)c->kw[5], *qx = (T *)c->kw[6], *qy = (T *)c->kw[7];
    const T *ix = (const T *)c->ivx, *iy = (const T *)c->ivy;
    const KrylovView kv{c->nx, c->ny, c->pitch, c->kpartials, c->kout};
    MgLevel top{};
    top.nx = c->nx;
    top.ny = c->ny;
    top.pitch = c->pitch;
    top.elems = c->elems;
    top.hx = c->hx;
    top.hy = c->hy;
    top.ec = c->eta_c;
    top.en = c->eta_n;
    top.bx = c->bx;
    top.by = c->by;
    top.vx = vx;
    top.vy = vy;
    top.rx = rx;
    top.ry = ry;
    // r = b - M v and E_v
    RUN(STOKES_K_MG, 1, mg_residual<T>(top, c->stream));
    RUN(STOKES_K_ENERGY, 2, kry_energy<T>(kv, rx, ry, (const T *)c->fx, (const T *)c->fy, ix, iy, c->stream));
    double num = 0.0, den = 1.0;
    st = read2(c, &num, &den);
    if (st != STOKES_OK) return st;
    double e = std::sqrt(num / den);
    const double e0 = e;
    int it = 0;
    auto check = [&]() -> int {
        if (!std::isfinite(e) || e > 1e6 * e0) return STOKES_ERR_DIVERGED;
        if (e <= params->tol) return 1;
        if (it >= params->max_cycles) return STOKES_ERR_NOT_CONVERGED;
        return 0;
    };
    int verdict = check();
    if (params->krylov == 2) {
        // defect correction around inner-precision flexible CG
        auto refine = [&](auto tag) -> int {
            using Ti = decltype(tag);
            Ti *w[10];
            for (int q = 0; q < 10; ++q) w[q] = (Ti *)c->iw[q];
            Ti *rix = w[0], *riy = w[1], *zix = w[2], *ziy = w[3], *pix = w[4], *piy = w[5], *qix = w[6],
               *qiy = w[7], *eix = w[8], *eiy = w[9];
            const MgLevel &l0 = mg_level(c->mg, 0);
            const GridDesc<Ti> gi = make_grid<Ti>(l0.nx, l0.ny, l0.pitch, l0.hx, l0.hy);
            const Ti *ixi = (const Ti *)l0.ivx, *iyi = (const Ti *)l0.ivy;
            const size_t ib = c->elems * sizeof(Ti);
            while (verdict == 0) {
                RUN(STOKES_K_MG, 1, (mg_cast<T, Ti>(c->elems, rx, rix, c->stream)));
                RUN(STOKES_K_MG, 1, (mg_cast<T, Ti>(c->elems, ry, riy, c->stream)));
                CK(cudaMemsetAsync(eix, 0, ib, c->stream));
                CK(cudaMemsetAsync(eiy, 0, ib, c->stream));
                int st2 = replay_graph(c);
                if (st2 != STOKES_OK) return st2;
                CK(cudaMemcpyAsync(pix, zix, ib, cudaMemcpyDeviceToDevice, c->stream));
                CK(cudaMemcpyAsync(piy, ziy, ib, cudaMemcpyDeviceToDevice, c->stream));
                for (int k = 0; k < params->inner_its; ++k) {
                    RUN(STOKES_K_APPLY, 2,
                        kry_apply_dot<Ti>(kv, gi, (const Ti *)l0.ec, (const Ti *)l0.en, (const Ti *)nullptr,
                                          (const Ti *)nullptr, pix, piy, qix, qiy, rix, riy,
                                          c->stream));
                    double pq = 0.0, pr = 0.0;
                    if ((st2 = read2(c, &pq, &pr)) != STOKES_OK) return st2;
                    RUN(STOKES_K_MG, 2,
                        kry_update<Ti>(kv, pr / pq, pix, piy, qix, qiy, eix, eiy, rix, riy, ixi, iyi, c->stream));
                    if (k == params->inner_its - 1) break;
                    if ((st2 = replay_graph(c)) != STOKES_OK) return st2;
                    RUN(STOKES_K_MG, 2,
                        kry_dot2<Ti>(kv, zix, ziy, qix, qiy, (const Ti *)nullptr, (const Ti *)nullptr, c->stream));
                    double zq = 0.0;
                    if ((st2 = read2(c, &zq, nullptr)) != STOKES_OK) return st2;
                    RUN(STOKES_K_MG, 1, kry_direction<Ti>(kv, -zq / pq, zix, ziy, pix, piy, c->stream));
                }
                RUN(STOKES_K_MG, 1, (kry_add_cast<T, Ti>(kv, eix, eiy, vx, vy, c->stream)));
                it += params->inner_its;
                RUN(STOKES_K_MG, 1, mg_residual<T>(top, c->stream));
                RUN(STOKES_K_ENERGY, 2,
                    kry_energy<T>(kv, rx, ry, (const T *)c->fx, (const T *)c->fy, ix, iy, c->stream));
                if ((st2 = read2(c, &num, nullptr)) != STOKES_OK) return st2;
                e = std::sqrt(num / den);
                verdict = check();
            }
            return STOKES_OK;
        };
        st = params->inner_dtype == STOKES_F64 ? refine(double{}) : refine(float{});
        if (st != STOKES_OK) return st;
    } else if (params->krylov && verdict == 0) {
        // flexible CG: the V-cycle reads r from the finest level's right-hand
        // side in the inner precision (written by the update kernel) and
        // leaves z in the inner precision, read as such by <z, q> and p = z + beta p
        if ((st = ensure_coef<T>(c, kv)) != STOKES_OK) return st;
        auto fcg = [&](auto tag) -> int {
            using Ti = decltype(tag);
            const MgLevel &l0 = mg_level(c->mg, 0);
            Ti *bix = (Ti *)l0.bx, *biy = (Ti *)l0.by;
            const Ti *zix = (const Ti *)c->gz[0], *ziy = (const Ti *)c->gz[1];
            RUN(STOKES_K_MG, 1, (mg_cast<T, Ti>(c->elems, rx, bix, c->stream)));
            RUN(STOKES_K_MG, 1, (mg_cast<T, Ti>(c->elems, ry, biy, c->stream)));
            int s2 = replay_graph(c);
            if (s2 != STOKES_OK) return s2;
            RUN(STOKES_K_MG, 1, (kry_direction_z<T, Ti>(kv, 0.0, zix, ziy, px, py, c->stream)));
            for (;;) {
                RUN(STOKES_K_APPLY, 2,
                    kry_apply_dot<T>(kv, g, (const T *)c->eta_c, (const T *)c->eta_n, (const T *)c->cax,
                                     (const T *)c->cay, px, py, qx, qy, rx, ry, c->stream));
                double pq = 0.0, pr = 0.0;
                if ((s2 = read2(c, &pq, &pr)) != STOKES_OK) return s2;
                const double a = pr / pq;
                RUN(STOKES_K_MG, 2,
                    (kry_update_cast<T, Ti>(kv, a, px, py, qx, qy, vx, vy, rx, ry, ix, iy, bix, biy, c->stream)));
                if ((s2 = read2(c, &num, nullptr)) != STOKES_OK) return s2;
                ++it;
                e = std::sqrt(num / den);
                if ((verdict = check()) != 0) break;
                if ((s2 = replay_graph(c)) != STOKES_OK) return s2;
                RUN(STOKES_K_MG, 2, (kry_dot_z<T, Ti>(kv, zix, ziy, qx, qy, c->stream)));
                double zq = 0.0;
                if ((s2 = read2(c, &zq, nullptr)) != STOKES_OK) return s2;
                RUN(STOKES_K_MG, 1, (kry_direction_z<T, Ti>(kv, -zq / pq, zix, ziy, px, py, c->stream)));
            }
            return STOKES_OK;
        };
        st = mg_dtype(c->mg) == STOKES_F64 ? fcg(double{}) : fcg(float{});
        if (st != STOKES_OK) return st;
    } else {
        while (verdict == 0) {
            if ((st = replay_graph(c)) != STOKES_OK) return st;
            RUN(STOKES_K_MG, 1, kry_add<T>(kv, zx, zy, vx, vy, c->stream));
            RUN(STOKES_K_MG, 1, mg_residual<T>(top, c->stream));
            RUN(STOKES_K_ENERGY, 2, kry_energy<T>(kv, rx, ry, (const T *)c->fx, (const T *)c->fy, ix, iy, c->stream));
            if ((st = read2(c, &num, nullptr)) != STOKES_OK) return st;
            ++it;
            e = std::sqrt(num / den);
            verdict = check();
        }
    }
    if (final_e) *final_e = e;
    if (cycles) *cycles = it;
    return verdict < 0 ? verdict : STOKES_OK;
}

// Solve H y = b (n x n, row-major, n <= AA_MAX) by Gaussian elimination with
// partial pivoting; false if singular.
bool small_solve(int n, double *H, double *b)
{
    for (int k = 0; k < n; ++k) {
        int piv = k;
        for (int i = k + 1; i < n; ++i)
            if (std::fabs(H[i * n + k]) > std::fabs(H[piv * n + k])) piv = i;
        if (!(std::fabs(H[piv * n + k]) > 0.0)) return false;
        if (piv != k) {
            for (int j = 0; j < n; ++j) std::swap(H[k * n + j], H[piv * n + j]);
            std::swap(b[k], b[piv]);
        }
        for (int i = k + 1; i < n; ++i) {
            const double f = H[i * n + k] / H[k * n + k];
            for (int j = k; j < n; ++j) H[i * n + j] -= f * H[k * n + j];
            b[i] -= f * b[k];
        }
    }
    for (int k = n - 1; k >= 0; --k) {
        double v = b[k];
        for (int j = k + 1; j < n; ++j) v -= H[k * n + j] * b[j];
        b[k] = v / H[k * n + k];
    }
    return true;
}

// swap in the viscosity of continuation stage theta (from the saved base)
template <typename T>
int set_stage(stokes_ctx *c, double theta)
{
    const GridDesc<T> g = grid_of<T>(c);
    RUN(STOKES_K_COPY, 1,
        uz_blend<T>(g, theta, c->uz_scal, (const T *)c->eta_c0, (const T *)c->eta_n0, (T *)c->eta_c, (T *)c->eta_n,
                    c->stream));
    RUN(STOKES_K_COPY, 1,
        launch_inv_diag<T>(g, (const T *)c->eta_c, (const T *)c->eta_n, (T *)c->ivx, (T *)c->ivy, c->stream));
    mg_invalidate(c->mg);
    ++c->eta_version;
    if (c->gexec) { // the graph holds the old hierarchy's buffers
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    return STOKES_OK;
}

// Inexact Uzawa iteration (Sec. 3.1-3.2, configuration of Sec. 6.2).
template <typename T>
int uzawa_impl(stokes_ctx *c, T *vx, T *vy, T *p, const stokes_uzawa_params *u, double *hist, int *cycles,
               double *final_e)
{
    const GridDesc<T> g = grid_of<T>(c);
    if (!c->uz_partials) {
        CK(cudaMalloc(&c->uz_partials, (size_t)uzawa_partials() * sizeof(double)));
        CK(cudaMalloc(&c->uz_scal, 2 * sizeof(double)));
    }
    if (u->lithostatic_init)
        RUN(STOKES_K_RHS, 4,
            uz_lithostatic<T>(g, c->hy, (const T *)c->fy, p, c->uz_partials, c->uz_scal + 1, c->stream));
    const bool cont = u->theta_interval > 0 && u->theta_stages > 1;
    if (cont) {
        if (!c->eta_c0) {
            int st = alloc_field(c, &c->eta_c0);
            if (st == STOKES_OK) st = alloc_field(c, &c->eta_n0);
            if (st != STOKES_OK) return st;
        }
        CK(cudaMemcpyAsync(c->eta_c0, c->eta_c, c->elems * c->esize, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(c->eta_n0, c->eta_n, c->elems * c->esize, cudaMemcpyDeviceToDevice, c->stream));
        RUN(STOKES_K_COPY, 2,
            uz_eta_min<T>(g, (const T *)c->eta_c, (const T *)c->eta_n, c->uz_partials, c->uz_scal, c->stream));
    }
    stokes_mg_params mp = u->mg;
    mp.tol = 0.0; // the velocity step always runs its mg.max_cycles V-cycles (unless the residual is 0)
    // Anderson acceleration (Algorithm 1): history of F(x_i) and r_i = F(x_i) - x_i
    const int depth = u->anderson_depth, slots = depth + 1;
    const size_t fbytes = c->elems * c->esize;
    if (depth > 0 && (int)c->aa.size() < 6 * slots + 3) {
        while ((int)c->aa.size() < 6 * slots + 3) {
            void *f = nullptr;
            const int st0 = alloc_field(c, &f);
            if (st0 != STOKES_OK) return st0;
            c->aa.push_back(f);
        }
        if (!c->aa_partials) {
            CK(cudaMalloc(&c->aa_partials, (size_t)uzawa_partials() * AA_MAX * sizeof(double)));
            CK(cudaMalloc(&c->aa_out, AA_MAX * sizeof(double)));
            CK(cudaMallocHost(&c->aa_hout, AA_MAX * sizeof(double)));
        }
    }
    auto fld = [&](int slot, int kind, int comp) { return (T *)c->aa[(size_t)(slot * 6 + kind * 3 + comp)]; };
    T *const xo[3] = {depth > 0 ? (T *)c->aa[6 * slots] : nullptr, depth > 0 ? (T *)c->aa[6 * slots + 1] : nullptr,
                      depth > 0 ? (T *)c->aa[6 * slots + 2] : nullptr};
    T *const xs[3] = {vx, vy, p};
    std::vector<int> order;                 // slots, oldest first
    std::vector<double> H((size_t)slots * slots, 0.0); // <r_s, r_t> by slot
    int stage = -1, st = STOKES_OK, n = 0;
    double e = 0.0;
    for (; n < u->cycles; ++n) {
        double theta = 1.0;
        if (cont) {
            const int sg = std::min(n / u->theta_interval, u->theta_stages - 1);
            theta = (double)sg / (double)(u->theta_stages - 1);
            if (sg != stage) {
                if ((st = set_stage<T>(c, theta)) != STOKES_OK) break;
                stage = sg;
                order.clear(); // the map F changes with theta: restart the history
            }
        }
        if (depth > 0)
            for (int q = 0; q < 3; ++q) CK(cudaMemcpyAsync(xo[q], xs[q], fbytes, cudaMemcpyDeviceToDevice, c->stream));
        // velocity step: M_theta v = f - G p from the current v
        st = vcycle_impl<T>(c, vx, vy, p, &mp, nullptr, nullptr);
        if (st == STOKES_ERR_NOT_CONVERGED) st = STOKES_OK;
        if (st != STOKES_OK) break;
        // pressure step and zero mean
        RUN(STOKES_K_MG, 3,
            uz_pressure_update<T>(g, u->omega_p, (const T *)c->eta_c, vx, vy, p, c->uz_partials, c->uz_scal + 1,
                                  c->stream));
        if (depth > 0) {
            // store F(x) and r = F(x) - x in a free slot, newest last
            int slot = 0;
            if ((int)order.size() == slots) {
                slot = order.front();
                order.erase(order.begin());
            } else {
                std::vector<bool> used(slots, false);
                for (int o : order) used[o] = true;
                while (used[slot]) ++slot;
            }
            for (int q = 0; q < 3; ++q) {
                CK(cudaMemcpyAsync(fld(slot, 0, q), xs[q], fbytes, cudaMemcpyDeviceToDevice, c->stream));
                RUN(STOKES_K_MG, 1, aa_diff<T>(c->elems, xs[q], xo[q], fld(slot, 1, q), c->stream));
            }
            order.push_back(slot);
            // <r_new, r_j> for every stored slot
            AndersonSet<T> a{}, hs{};
            a.x[0] = fld(slot, 1, 0);
            a.y[0] = fld(slot, 1, 1);
            a.p[0] = fld(slot, 1, 2);
            a.n = 1;
            hs.n = (int)order.size();
            for (int j = 0; j < hs.n; ++j) {
                hs.x[j] = fld(order[j], 1, 0);
                hs.y[j] = fld(order[j], 1, 1);
                hs.p[j] = fld(order[j], 1, 2);
            }
            RUN(STOKES_K_MG, 2, aa_multidot<T>(c->elems, a, hs, c->aa_partials, c->aa_out, c->stream));
            CK(cudaMemcpyAsync(c->aa_hout, c->aa_out, AA_MAX * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
            if ((st = device_status(c)) != STOKES_OK) break;
            for (int j = 0; j < hs.n; ++j) {
                H[(size_t)slot * slots + order[j]] = c->aa_hout[j];
                H[(size_t)order[j] * slots + slot] = c->aa_hout[j];
            }
            if (hs.n > 1) {
                // alpha = argmin ||R alpha|| with sum alpha = 1: H y = 1, alpha = y / sum y
                const int m = hs.n;
                double Hm[AA_MAX * AA_MAX], y[AA_MAX], dmax = 0.0;
                for (int i = 0; i < m; ++i) {
                    for (int j = 0; j < m; ++j) Hm[i * m + j] = H[(size_t)order[i] * slots + order[j]];
                    dmax = std::max(dmax, Hm[i * m + i]);
                    y[i] = 1.0;
                }
                for (int i = 0; i < m; ++i) Hm[i * m + i] += 1e-14 * std::max(dmax, 1e-300);
                if (small_solve(m, Hm, y)) {
                    double sy = 0.0;
                    for (int i = 0; i < m; ++i) sy += y[i];
                    AndersonAlpha al{};
                    AndersonSet<T> F{};
                    F.n = m;
                    for (int i = 0; i < m; ++i) {
                        al.a[i] = y[i] / sy;
                        F.x[i] = fld(order[i], 0, 0);
                        F.y[i] = fld(order[i], 0, 1);
                        F.p[i] = fld(order[i], 0, 2);
                    }
                    RUN(STOKES_K_MG, 1, aa_combine<T>(c->elems, F, al, vx, vy, p, c->stream));
                }
            }
        }
        // relative energy residual (Sec. 6.4) with the caller's viscosity
        const bool base = cont && theta != 1.0;
        RUN(STOKES_K_ENERGY, 2,
            launch_energy<T>(g, (const T *)(base ? c->eta_c0 : c->eta_c), (const T *)(base ? c->eta_n0 : c->eta_n),
                             base ? nullptr : (const T *)c->ivx, base ? nullptr : (const T *)c->ivy,
                             (const T *)c->fx, (const T *)c->fy, p, vx, vy, c->partials, c->dsum, c->stream));
        CK(cudaMemcpyAsync(c->hsum, c->dsum, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        if ((st = device_status(c)) != STOKES_OK) break;
        e = std::sqrt((c->hsum[0] + c->hsum[1]) / c->hsum[2]);
        if (hist) hist[n] = e;
        if (!std::isfinite(e)) {
            st = STOKES_ERR_DIVERGED;
            ++n;
            break;
        }
        if (e <= u->tol) {
            ++n;
            break;
        }
    }
    // leave the context with the caller's viscosity
    if (cont && stage != u->theta_stages - 1 && stage >= 0) {
        CK(cudaMemcpyAsync(c->eta_c, c->eta_c0, c->elems * c->esize, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(c->eta_n, c->eta_n0, c->elems * c->esize, cudaMemcpyDeviceToDevice, c->stream));
        RUN(STOKES_K_COPY, 1,
            launch_inv_diag<T>(g, (const T *)c->eta_c, (const T *)c->eta_n, (T *)c->ivx, (T *)c->ivy, c->stream));
        mg_invalidate(c->mg);
        ++c->eta_version;
        if (c->gexec) {
            cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
        }
    }
    if (cycles) *cycles = n;
    if (final_e) *final_e = e;
    if (st != STOKES_OK) return st;
    return (u->tol > 0.0 && !(e <= u->tol)) ? STOKES_ERR_NOT_CONVERGED : STOKES_OK;
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
    if (nx < 2 || ny < 2 || nx > (1 << 18) || ny > (1 << 18) || !(lx > 0.0) || !(ly > 0.0)) return STOKES_ERR_ARG;
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
    if (st == STOKES_OK) st = alloc_field(c, &c->ivx);
    if (st == STOKES_OK) st = alloc_field(c, &c->ivy);
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
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->gstream) cudaStreamSynchronize(c->gstream);
    for (void *w : c->kw)
        if (w) cudaFree(w);
    for (void *w : c->iw)
        if (w) cudaFree(w);
    if (c->kpartials) cudaFree(c->kpartials);
    if (c->kout) cudaFree(c->kout);
    if (c->hout) cudaFreeHost(c->hout);
    if (c->gstream) cudaStreamDestroy(c->gstream);
    for (cudaEvent_t e : c->gev)
        if (e) cudaEventDestroy(e);
    mg_destroy(c->mg);
    prof_flush(c);
    for (cudaEvent_t e : c->prof.pool) cudaEventDestroy(e);
    void *fields[] = {c->eta_c, c->eta_n, c->fx, c->fy, c->bx, c->by, c->sx, c->sy, c->ivx, c->ivy, c->cax, c->cay, c->sx2, c->sy2,
                      c->partials,
                      c->dsum, c->dstatus, c->eta_c0, c->eta_n0, c->uz_partials, c->uz_scal};
    for (void *f : fields)
        if (f) cudaFree(f);
    if (c->hsum) cudaFreeHost(c->hsum);
    if (c->hstatus) cudaFreeHost(c->hstatus);
    for (void *f : c->aa) cudaFree(f);
    if (c->aa_partials) cudaFree(c->aa_partials);
    if (c->aa_out) cudaFree(c->aa_out);
    if (c->aa_hout) cudaFreeHost(c->aa_hout);
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
    if (c->dtype == STOKES_F64)
        RUN(STOKES_K_COPY, 1,
            launch_set_eta<double>(grid_of<double>(c), (const double *)eta_c, (const double *)eta_n,
                                   (double *)c->eta_c, (double *)c->eta_n, (double *)c->ivx, (double *)c->ivy,
                                   c->stream));
    else
        RUN(STOKES_K_COPY, 1,
            launch_set_eta<float>(grid_of<float>(c), (const float *)eta_c, (const float *)eta_n, (float *)c->eta_c,
                                  (float *)c->eta_n, (float *)c->ivx, (float *)c->ivy, c->stream));
    c->have_eta = true;
    mg_invalidate(c->mg);
    ++c->eta_version;
    if (c->gexec) { // the graph holds the old hierarchy's buffers
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    return STOKES_OK;
}

int stokes_set_rhs(stokes_ctx *c, const void *fx, const void *fy)
{
    if (!c || !fx || !fy) return STOKES_ERR_ARG;
    // f at the unknowns, zero on walls and padding: f is then b = f - G p for p = 0
    if (c->dtype == STOKES_F64)
        RUN(STOKES_K_RHS, 1, launch_rhs<double>(grid_of<double>(c), (const double *)fx, (const double *)fy, nullptr,
                                                (double *)c->fx, (double *)c->fy, c->stream));
    else
        RUN(STOKES_K_RHS, 1, launch_rhs<float>(grid_of<float>(c), (const float *)fx, (const float *)fy, nullptr,
                                               (float *)c->fx, (float *)c->fy, c->stream));
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

// field buffers start on a 16-byte boundary (the sweep kernels read and write
// 16-byte vectors; TMA copies need the same)
static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

int stokes_smooth(stokes_ctx *c, void *vx, void *vy, const void *p, const stokes_smooth_params *params)
{
    if (!c || !vx || !vy) return STOKES_ERR_ARG;
    if (!aligned16(vx) || !aligned16(vy) || !aligned16(p)) return STOKES_ERR_ARG;
    int ti, tj, st = check_smooth_params(c->nx, c->ny, c->esize, params, &ti, &tj);
    if (st != STOKES_OK) return st;
    if (!c->have_eta || !c->have_f) return STOKES_ERR_STATE;
    const bool b_is_f = p == nullptr;
    if (c->dtype == STOKES_F64) {
        if (!b_is_f)
            RUN(STOKES_K_RHS, 1, launch_rhs<double>(grid_of<double>(c), (const double *)c->fx, (const double *)c->fy,
                                                    (const double *)p, (double *)c->bx, (double *)c->by, c->stream));
        return smooth_impl<double>(c, (double *)vx, (double *)vy, params, ti, tj, b_is_f);
    }
    if (!b_is_f)
        RUN(STOKES_K_RHS, 1, launch_rhs<float>(grid_of<float>(c), (const float *)c->fx, (const float *)c->fy,
                                               (const float *)p, (float *)c->bx, (float *)c->by, c->stream));
    return smooth_impl<float>(c, (float *)vx, (float *)vy, params, ti, tj, b_is_f);
}

int stokes_residual_energy_norm(stokes_ctx *c, const void *vx, const void *vy, const void *p, double out[3])
{
    if (!c || !vx || !vy || !out) return STOKES_ERR_ARG;
    if (!aligned16(vx) || !aligned16(vy) || !aligned16(p)) return STOKES_ERR_ARG; // vector row loads
    if (!c->have_eta || !c->have_f) return STOKES_ERR_STATE;
    if (c->dtype == STOKES_F64) return energy_impl<double>(c, (const double *)vx, (const double *)vy, (const double *)p, out);
    return energy_impl<float>(c, (const float *)vx, (const float *)vy, (const float *)p, out);
}

int stokes_vcycle(stokes_ctx *c, void *vx, void *vy, const void *p, const stokes_mg_params *params,
                  double *final_rel_resid, int *cycles)
{
    if (!c || !vx || !vy || !params) return STOKES_ERR_ARG;
    if (!aligned16(vx) || !aligned16(vy) || !aligned16(p)) return STOKES_ERR_ARG;
    const int st = check_mg_params(c, params);
    if (st != STOKES_OK) return st;
    if (!c->have_eta || !c->have_f) return STOKES_ERR_STATE;
    if (c->dtype == STOKES_F64)
        return vcycle_impl<double>(c, (double *)vx, (double *)vy, (const double *)p, params, final_rel_resid, cycles);
    return vcycle_impl<float>(c, (float *)vx, (float *)vy, (const float *)p, params, final_rel_resid, cycles);
}

int stokes_uzawa(stokes_ctx *c, void *vx, void *vy, void *p, const stokes_uzawa_params *params, double *history,
                 int *cycles, double *final_rel_resid)
{
    if (!c || !vx || !vy || !p || !params) return STOKES_ERR_ARG;
    if (!aligned16(vx) || !aligned16(vy) || !aligned16(p)) return STOKES_ERR_ARG;
    const stokes_uzawa_params &u = *params;
    if (u.cycles < 0 || !(u.omega_p > 0.0) || !std::isfinite(u.omega_p) || u.theta_interval < 0 ||
        u.theta_stages < 0 || !(u.tol >= 0.0) || u.mg.max_cycles < 1 || u.anderson_depth < 0 ||
        u.anderson_depth >= AA_MAX)
        return STOKES_ERR_ARG;
    int st = check_mg_params(c, &u.mg);
    if (st != STOKES_OK) return st;
    if (!c->have_eta || !c->have_f) return STOKES_ERR_STATE;
    if (c->dtype == STOKES_F64)
        return uzawa_impl<double>(c, (double *)vx, (double *)vy, (double *)p, params, history, cycles,
                                  final_rel_resid);
    return uzawa_impl<float>(c, (float *)vx, (float *)vy, (float *)p, params, history, cycles, final_rel_resid);
}

int stokes_set_option(stokes_ctx *c, int option, long long value)
{
    if (!c) return STOKES_ERR_ARG;
    switch (option) {
    case STOKES_OPT_USE_TMA: c->use_tma = value != 0; return STOKES_OK;
    case STOKES_OPT_WAIT_LIMIT_CYCLES: c->wait_limit = value; return STOKES_OK;
    case STOKES_OPT_PAIRED:
        if (value < 0 || value > 2) return STOKES_ERR_ARG;
        c->pair_mode = (int)value;
        return STOKES_OK;
    default: return STOKES_ERR_ARG;
    }
}

int stokes_tile_kernel_plan(int nx, int ny, int ti, int tj, int overlap, int dtype, int use_tma, int pair_mode,
                            int *kernel, int *threads, size_t *smem_bytes)
{
    if (nx < 1 || ny < 1 || ti < 1 || tj < 1 || overlap < 0 || (dtype != STOKES_F32 && dtype != STOKES_F64) ||
        pair_mode < 0 || pair_mode > 2)
        return STOKES_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return STOKES_ERR_CUDA;
    }
    int kind = 0, thr = 0;
    size_t smem = 0;
    ras_kernel_plan(nx, ny, ti, tj, overlap, dtype == STOKES_F64 ? 8 : 4, use_tma != 0, pair_mode, &kind, &thr, &smem);
    if (kernel) *kernel = kind;
    if (threads) *threads = thr;
    if (smem_bytes) *smem_bytes = smem;
    return STOKES_OK;
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
