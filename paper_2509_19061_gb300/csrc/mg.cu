// mg.cu -- geometric-multigrid hierarchy and V-cycle of a context (Sec. 3.2;
// configuration of Sec. 6.2): level construction, the dense FP64 coarsest
// factorisation (on the GPU), and the enqueue of one V-cycle application.
//
// Level l runs ceil(nu_pre g^l) pre- and ceil(nu_post g^l) post-sweeps of the
// chosen smoother (optionally capped); a RAS smoother on level l, phase ph
// draws its shifts from SplitMix64 seeded with splitmix64(seed, 2 l + ph), so
// every cycle is the same linear map and the caller can replay it as a graph.
// The cycle is used as the preconditioner z = B r of the outer solve.
#include <cmath>
#include <new>
#include <utility>

#include "../../include/stokes.h"
#include "internal.h"
#include "mg.h"

namespace stokes {

constexpr int MG_MAX_LEVELS = 32;
constexpr int MG_MAX_DENSE = 1024; // unknowns of the coarsest level

struct MgHierarchy {
    bool stale = true;
    int dtype = -1, levels_req = -1, coarsest_req = -1;
    int L = 0;
    MgLevel lv[MG_MAX_LEVELS] = {};
    int n = 0; // coarsest unknowns
    double *A = nullptr, *W = nullptr, *Ainv = nullptr, *bvec = nullptr, *xvec = nullptr;
    int *dstatus = nullptr;
    const void *zx = nullptr, *zy = nullptr; // finest-level result of the last enqueued application
};

namespace {

void free_level(MgLevel &l)
{
    void *ps[] = {l.ec, l.en, l.ivx, l.ivy, l.bx, l.by, l.vx, l.vy, l.rx, l.ry, l.sx, l.sy};
    for (void *p : ps)
        if (p) cudaFree(p);
    l = MgLevel{};
}

void free_all(MgHierarchy *h)
{
    for (int l = 0; l < h->L; ++l) free_level(h->lv[l]);
    void *ps[] = {h->A, h->W, h->Ainv, h->bvec, h->xvec, h->dstatus};
    for (void *p : ps)
        if (p) cudaFree(p);
    h->A = h->W = h->Ainv = h->bvec = h->xvec = nullptr;
    h->dstatus = nullptr;
    h->L = 0;
    h->n = 0;
}

int alloc_level(MgLevel &l, int nx, int ny, double hx, double hy, size_t es, bool inv, cudaStream_t s)
{
    l.nx = nx;
    l.ny = ny;
    l.hx = hx;
    l.hy = hy;
    l.pitch = ((nx + 1) + 31) / 32 * 32;
    l.elems = (size_t)(ny + 1) * (size_t)l.pitch;
    void **fs[] = {&l.ec, &l.en, &l.bx, &l.by, &l.vx, &l.vy, &l.rx, &l.ry, &l.sx, &l.sy, &l.ivx, &l.ivy};
    const int nf = inv ? 12 : 10;
    for (int f = 0; f < nf; ++f) {
        cudaError_t e = cudaMalloc(fs[f], l.elems * es);
        if (e == cudaSuccess) e = cudaMemsetAsync(*fs[f], 0, l.elems * es, s);
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? STOKES_ERR_OOM : STOKES_ERR_CUDA;
    }
    return STOKES_OK;
}

template <typename T>
Coeffs<T> level_coeffs(const MgLevel &l)
{
    Coeffs<T> k;
    k.eta_c = (const T *)l.ec;
    k.eta_n = (const T *)l.en;
    k.bx = (const T *)l.bx;
    k.by = (const T *)l.by;
    k.inv_dx = (const T *)l.ivx;
    k.inv_dy = (const T *)l.ivy;
    return k;
}

template <typename T>
GridDesc<T> level_grid(const MgLevel &l)
{
    return make_grid<T>(l.nx, l.ny, l.pitch, l.hx, l.hy);
}

int n_unknowns(int nx, int ny) { return ny * (nx - 1) + (ny - 1) * nx; }

#define CKS(expr)                                                                                                  \
    do {                                                                                                           \
        if ((expr) != cudaSuccess) return STOKES_ERR_CUDA;                                                         \
    } while (0)

template <typename Ti>
int build(MgHierarchy *h, const MgOuter &o, int levels, int coarsest, cudaStream_t s)
{
    const size_t es = sizeof(Ti);
    const bool inv = true; // 1/diag(M) on every level, read by the tile kernels
    // level sizes
    int nx = o.nx, ny = o.ny, L = 1;
    while (L < levels && L < MG_MAX_LEVELS && nx % 2 == 0 && ny % 2 == 0 && nx > coarsest && ny > coarsest) {
        nx /= 2;
        ny /= 2;
        ++L;
    }
    if (n_unknowns(nx, ny) > MG_MAX_DENSE || nx < 2 || ny < 2) return STOKES_ERR_ARG;
    nx = o.nx;
    ny = o.ny;
    double hx = o.hx, hy = o.hy;
    for (int l = 0; l < L; ++l) {
        h->L = l + 1;
        int st = alloc_level(h->lv[l], nx, ny, hx, hy, es, inv, s);
        if (st != STOKES_OK) return st;
        nx /= 2;
        ny /= 2;
        hx *= 2.0;
        hy *= 2.0;
    }
    // level-0 viscosity in the inner precision, then coarser levels
    MgLevel &l0 = h->lv[0];
    if (o.dtype == STOKES_F64) {
        CKS((mg_cast<double, Ti>(l0.elems, o.eta_c, l0.ec, s)));
        CKS((mg_cast<double, Ti>(l0.elems, o.eta_n, l0.en, s)));
    } else {
        CKS((mg_cast<float, Ti>(l0.elems, o.eta_c, l0.ec, s)));
        CKS((mg_cast<float, Ti>(l0.elems, o.eta_n, l0.en, s)));
    }
    for (int l = 1; l < L; ++l) CKS(mg_coarsen_eta<Ti>(h->lv[l - 1], h->lv[l], s));
    if (inv)
        for (int l = 0; l < L; ++l) {
            const MgLevel &v = h->lv[l];
            CKS(launch_inv_diag<Ti>(level_grid<Ti>(v), (const Ti *)v.ec, (const Ti *)v.en, (Ti *)v.ivx,
                                    (Ti *)v.ivy, s));
        }
    // dense inverse of -M on the coarsest level
    const MgLevel &lc = h->lv[L - 1];
    h->n = n_unknowns(lc.nx, lc.ny);
    const size_t nn = (size_t)h->n * h->n;
    if (cudaMalloc(&h->A, nn * 8) != cudaSuccess || cudaMalloc(&h->W, nn * 8) != cudaSuccess ||
        cudaMalloc(&h->Ainv, nn * 8) != cudaSuccess || cudaMalloc(&h->bvec, h->n * 8) != cudaSuccess ||
        cudaMalloc(&h->xvec, h->n * 8) != cudaSuccess || cudaMalloc(&h->dstatus, sizeof(int)) != cudaSuccess)
        return STOKES_ERR_OOM;
    CKS(cudaMemsetAsync(h->dstatus, 0, sizeof(int), s));
    CKS(mg_dense_setup<Ti>(lc, h->n, h->A, h->W, h->Ainv, h->dstatus, s));
    int bad = 0;
    CKS(cudaMemcpyAsync(&bad, h->dstatus, sizeof(int), cudaMemcpyDeviceToHost, s));
    CKS(cudaStreamSynchronize(s));
    cudaFree(h->A);
    cudaFree(h->W);
    h->A = h->W = nullptr;
    return bad ? STOKES_ERR_DIVERGED : STOKES_OK;
}

// smoothing spec of level l and phase ph
SmoothSpec level_spec(const stokes_mg_params *p, const MgLevel &l, int lvl, int ph, size_t es)
{
    const stokes_smooth_params sm = level_smoother(p->smoother, lvl);
    SmoothSpec s;
    s.variant = sm.variant;
    s.sweeps = mg_sweeps(ph == 0 ? p->nu_pre : p->nu_post, p->nu_growth, lvl, p->nu_max);
    s.ti = sm.tile_i > 0 ? sm.tile_i : 32;
    s.tj = sm.tile_j > 0 ? sm.tile_j : 32;
    s.k = sm.k;
    s.overlap = sm.overlap;
    s.omega = sm.omega;
    s.seed = splitmix64(sm.seed, 2u * (uint64_t)lvl + (uint64_t)ph);
    s.shift_mode = STOKES_SHIFT_SPLITMIX;
    s.shifts = nullptr;
    // Jacobi in any schedule (and RAS with overlap >= k-1, which is Jacobi)
    // on a level whose whole-level window fits a register tile kernel: all
    // sweeps in one launch (the same map, so the same values)
    const bool jacobi = sm.variant == STOKES_JACOBI || sm.variant == STOKES_JACOBI_FUSED ||
                        sm.variant == STOKES_JACOBI_BLOCKED ||
                        (sm.variant == STOKES_RAS && sm.overlap >= sm.k - 1);
    if (jacobi && s.sweeps > 0 && ras_whole_level_tile(l.nx, l.ny, es)) {
        s.variant = STOKES_RAS;
        s.ti = l.nx;
        s.tj = l.ny;
        s.k = s.sweeps;
        s.overlap = 0;
        s.shift_mode = STOKES_SHIFT_NONE;
    }
    return s;
}

template <typename Tc, typename Ti>
int enqueue_precond(MgHierarchy *h, const Tc *rx, const Tc *ry, Tc *zx, Tc *zy, const stokes_mg_params *p,
                    const RasRun &run, cudaStream_t s, LaunchHook &hook)
{
    int st = STOKES_OK;
#define LAUNCH(kind, nk, expr)                                                                                     \
    do {                                                                                                           \
        st = hook.run((kind), (nk), [&]() { return (expr); });                                                     \
        if (st != STOKES_OK) return st;                                                                            \
    } while (0)
    const int L = h->L;
    MgLevel &l0 = h->lv[0];
    // A smoothing that ends in a level's scratch pair leaves its result there
    // and the level's (vx, vy) and (sx, sy) pointers trade places for the rest
    // of this enqueue (the launches record the addresses they were given); the
    // guard puts the host-side pointers back when the enqueue ends.
    struct Restore {
        MgHierarchy *h;
        void *p[MG_MAX_LEVELS][4];
        explicit Restore(MgHierarchy *hh) : h(hh)
        {
            for (int l = 0; l < h->L; ++l) {
                p[l][0] = h->lv[l].vx;
                p[l][1] = h->lv[l].vy;
                p[l][2] = h->lv[l].sx;
                p[l][3] = h->lv[l].sy;
            }
        }
        ~Restore()
        {
            for (int l = 0; l < h->L; ++l) {
                h->lv[l].vx = p[l][0];
                h->lv[l].vy = p[l][1];
                h->lv[l].sx = p[l][2];
                h->lv[l].sy = p[l][3];
            }
        }
    } restore(h);
    auto smooth_level = [&](MgLevel &f, int l, int phase) -> int {
        bool swapped = false;
        const int r = smooth_buffers<Ti>(level_grid<Ti>(f), level_coeffs<Ti>(f), (Ti *)f.vx, (Ti *)f.vy, (Ti *)f.sx,
                                         (Ti *)f.sy, level_spec(p, f, l, phase, sizeof(Ti)), run, s, hook, &swapped);
        if (swapped) {
            std::swap(f.vx, f.sx);
            std::swap(f.vy, f.sy);
        }
        return r;
    };
    if (rx) {
        LAUNCH(STOKES_K_MG, 1, (mg_cast<Tc, Ti>(l0.elems, rx, l0.bx, s)));
        LAUNCH(STOKES_K_MG, 1, (mg_cast<Tc, Ti>(l0.elems, ry, l0.by, s)));
    }
    for (int l = 0; l < L; ++l) {
        MgLevel &v = h->lv[l];
        LAUNCH(STOKES_K_COPY, 0, cudaMemsetAsync(v.vx, 0, v.elems * sizeof(Ti), s));
        LAUNCH(STOKES_K_COPY, 0, cudaMemsetAsync(v.vy, 0, v.elems * sizeof(Ti), s));
    }
    // down: smooth, residual, restrict
    for (int l = 0; l < L - 1; ++l) {
        MgLevel &f = h->lv[l];
        st = smooth_level(f, l, 0);
        if (st != STOKES_OK) return st;
        LAUNCH(STOKES_K_MG, 1, mg_residual<Ti>(f, s));
        LAUNCH(STOKES_K_MG, 1, mg_restrict<Ti>(f, h->lv[l + 1], s));
    }
    // coarsest: exact solve
    LAUNCH(STOKES_K_MG, 3, mg_dense_solve<Ti>(h->lv[L - 1], h->n, h->Ainv, h->bvec, h->xvec, s));
    // up: prolong and correct, smooth
    for (int l = L - 2; l >= 0; --l) {
        MgLevel &f = h->lv[l];
        LAUNCH(STOKES_K_MG, 1, mg_prolong_add<Ti>(f, h->lv[l + 1], s));
        st = smooth_level(f, l, 1);
        if (st != STOKES_OK) return st;
    }
    h->zx = l0.vx;
    h->zy = l0.vy;
    if (zx) {
        LAUNCH(STOKES_K_MG, 1, (mg_cast<Ti, Tc>(l0.elems, l0.vx, zx, s)));
        LAUNCH(STOKES_K_MG, 1, (mg_cast<Ti, Tc>(l0.elems, l0.vy, zy, s)));
    }
#undef LAUNCH
    return STOKES_OK;
}

} // namespace

stokes_smooth_params level_smoother(const stokes_smooth_params &sm, int level)
{
    stokes_smooth_params s = sm;
    if (s.variant == STOKES_MIXED) s.variant = level == 0 ? STOKES_JACOBI : STOKES_RAS;
    return s;
}

int mg_sweeps(int nu0, double growth, int l, int nu_max)
{
    double f = (double)nu0;
    for (int q = 0; q < l; ++q) f *= growth;
    const int nu = (int)std::ceil(f);
    return (nu_max > 0 && nu > nu_max) ? nu_max : nu;
}

void mg_invalidate(MgHierarchy *h)
{
    if (h) h->stale = true;
}

void mg_destroy(MgHierarchy *h)
{
    if (!h) return;
    free_all(h);
    delete h;
}

int mg_levels(const MgHierarchy *h) { return h ? h->L : 0; }

int mg_dtype(const MgHierarchy *h) { return h ? h->dtype : -1; }

void mg_result(const MgHierarchy *h, const void **zx, const void **zy)
{
    *zx = h->zx;
    *zy = h->zy;
}

const MgLevel &mg_level(const MgHierarchy *h, int l) { return h->lv[l]; }

int mg_ensure(MgHierarchy **hp, const MgOuter &o, const stokes_mg_params *p, cudaStream_t s)
{
    if (!*hp) {
        *hp = new (std::nothrow) MgHierarchy();
        if (!*hp) return STOKES_ERR_OOM;
    }
    MgHierarchy *h = *hp;
    if (!h->stale && h->dtype == p->inner_dtype && h->levels_req == p->levels && h->coarsest_req == p->coarsest)
        return STOKES_OK;
    if (cudaStreamSynchronize(s) != cudaSuccess) return STOKES_ERR_CUDA;
    free_all(h);
    h->stale = true;
    const int st = p->inner_dtype == STOKES_F64 ? build<double>(h, o, p->levels, p->coarsest, s)
                                                : build<float>(h, o, p->levels, p->coarsest, s);
    if (st != STOKES_OK) {
        cudaStreamSynchronize(s);
        free_all(h);
        return st;
    }
    h->stale = false;
    h->dtype = p->inner_dtype;
    h->levels_req = p->levels;
    h->coarsest_req = p->coarsest;
    return STOKES_OK;
}

int mg_enqueue_precond(MgHierarchy *h, int outer_dtype, const void *rx, const void *ry, void *zx, void *zy,
                       const stokes_mg_params *p, const RasRun &run, cudaStream_t s, LaunchHook &hook)
{
    if (outer_dtype == STOKES_F64) {
        if (h->dtype == STOKES_F64)
            return enqueue_precond<double, double>(h, (const double *)rx, (const double *)ry, (double *)zx,
                                                   (double *)zy, p, run, s, hook);
        return enqueue_precond<double, float>(h, (const double *)rx, (const double *)ry, (double *)zx, (double *)zy,
                                              p, run, s, hook);
    }
    if (h->dtype == STOKES_F64)
        return enqueue_precond<float, double>(h, (const float *)rx, (const float *)ry, (float *)zx, (float *)zy, p,
                                              run, s, hook);
    return enqueue_precond<float, float>(h, (const float *)rx, (const float *)ry, (float *)zx, (float *)zy, p, run,
                                         s, hook);
}

} // namespace stokes
