// batch.cu -- many independent problems of different sizes advanced
// together.  Every step of a smoothing call, of the V-cycle (Sec. 3.2) and of
// the outer iteration runs as one launch over all instances that take part
// in it, and the V-cycle of all instances is captured once as a CUDA graph.
//
// Each instance follows exactly the schedule a context of its own would run
// (same tiles, shifts, sweep counts and per-point arithmetic), so its
// smoothing and V-cycle results equal that context's bit for bit.  Only the
// FP64 sums of the outer iteration (energy residual, CG inner products) are
// accumulated in another fixed order.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <cuda.h>

#include "../../include/stokes.h"
#include "batch.h"
#include "internal.h"
#include "mg.h"

using namespace stokes;

namespace {

#define CK(call)                                                                                                   \
    do {                                                                                                           \
        cudaError_t e_ = (call);                                                                                   \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);                                                        \
    } while (0)
#define ST(call)                                                                                                   \
    do {                                                                                                           \
        const int s_ = (call);                                                                                     \
        if (s_ != STOKES_OK) return s_;                                                                            \
    } while (0)

constexpr int B_MAX_LEVELS = 32;
constexpr int B_MAX_DENSE = 1024; // unknowns of a coarsest level
constexpr size_t B_ALIGN = 64;    // instance offsets in a slab (elements)

// one instance's grid and its place in a slab
struct Dims {
    int nx = 0, ny = 0, pitch = 0; // nx = 0: the instance has no such level
    double hx = 0, hy = 0;
    size_t off = 0, elems = 0;
};

Dims dims_of(int nx, int ny, double hx, double hy)
{
    Dims d;
    d.nx = nx;
    d.ny = ny;
    d.hx = hx;
    d.hy = hy;
    d.pitch = ((nx + 1) + 31) / 32 * 32;
    d.elems = (size_t)(ny + 1) * (size_t)d.pitch;
    return d;
}

// place the present instances back to back; returns the slab size (elements)
size_t place(std::vector<Dims> &d)
{
    size_t off = 0;
    for (Dims &x : d) {
        if (x.nx == 0) continue;
        x.off = off;
        off += (x.elems + B_ALIGN - 1) / B_ALIGN * B_ALIGN;
    }
    return off;
}

// device allocations owned by a batch (tables, maps), freed together
struct Owned {
    std::vector<void *> p;
    void release()
    {
        for (void *q : p) cudaFree(q);
        p.clear();
    }
};

template <typename X>
int upload(Owned &o, const std::vector<X> &h, const X **out, cudaStream_t s)
{
    *out = nullptr;
    if (h.empty()) return STOKES_OK;
    void *d = nullptr;
    CK(cudaMalloc(&d, h.size() * sizeof(X)));
    o.p.push_back(d);
    CK(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(X), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    *out = (const X *)d;
    return STOKES_OK;
}

// the instances of one element-wise launch and the rectangle each covers
struct Sub {
    const BSeg *map = nullptr;
    int nseg = 0, nblocks = 0;
};
struct Rect {
    int inst, w, h;
};

// block_rows = BATCH_BY * BATCH_TALL makes a tall map
int make_sub(Owned &o, const std::vector<Rect> &r, Sub *out, cudaStream_t s, int block_rows = BATCH_BY)
{
    std::vector<BSeg> m;
    int b = 0;
    for (const Rect &x : r) {
        BSeg g;
        g.inst = x.inst;
        g.w = x.w;
        g.h = x.h;
        g.bxb = (x.w + BATCH_BX - 1) / BATCH_BX;
        g.block_begin = b;
        b += g.bxb * ((x.h + block_rows - 1) / block_rows);
        m.push_back(g);
    }
    out->nseg = (int)m.size();
    out->nblocks = b;
    return upload(o, m, &out->map, s);
}

// ---- smoothing groups ----------------------------------------------------------
// A smoothing schedule in RAS form.  The Jacobi variants are run as RAS outer
// iterations with overlap >= k - 1, which reproduce Jacobi exactly.
struct RasForm {
    int sweeps, ti, tj, k, overlap, shift_mode;
    double omega;
    uint64_t seed;
    const int32_t *shifts;
};

template <typename T>
struct TileLaunch {
    const BatchTiles<T> *tab;
    const int *tmap;  // table entry of every tile
    const void *maps; // per-instance tensor maps (TMA staging), or NULL
    int count, total, ti, tj, ks, overlap;
    bool square;      // every instance has square cells
};

// one instance of a group: level grid and coefficients, velocity and scratch
template <typename T>
struct GInst {
    int inst;
    GridDesc<T> g;
    Coeffs<T> c;
    T *vx, *vy, *sx, *sy;
    int ti, tj; // tile of this instance (the level itself for single-tile groups)
};

template <typename T>
struct Group {
    std::vector<TileLaunch<T>> launches;
    const BLevel<T> *lev = nullptr; // vx, vy, sx, sy per instance (copies)
    Sub sub;                        // the instances over (nx+1) x (ny+1), a tall map
    bool walls = false, back = false;
    T omega = T(0);
};

// the ping-pong of smooth_buffers for every instance of `gi` at once
template <typename T>
int plan_group(Owned &o, const std::vector<GInst<T>> &gi, const RasForm &f, bool walls, bool single, bool tma,
               int pair_mode, const BLevel<T> *lev, Group<T> *out, cudaStream_t s)
{
    *out = Group<T>();
    if (gi.empty() || f.sweeps == 0) return STOKES_OK;
    out->lev = lev;
    out->walls = walls;
    out->omega = (T)f.omega;
    std::vector<Rect> rects;
    for (const GInst<T> &x : gi) rects.push_back({x.inst, x.g.nx + 1, x.g.ny + 1});
    ST(make_sub(o, rects, &out->sub, s, BATCH_BY * BATCH_TALL));
    const size_t n = gi.size();
    std::vector<T *> ax(n), ay(n), bx(n), by(n);
    for (size_t q = 0; q < n; ++q) {
        ax[q] = gi[q].vx;
        ay[q] = gi[q].vy;
        bx[q] = gi[q].sx;
        by[q] = gi[q].sy;
    }
    const int n_outer = (f.sweeps + f.k - 1) / f.k;
    for (int t = 0; t < n_outer; ++t) {
        const int ks = (t == n_outer - 1) ? f.sweeps - (n_outer - 1) * f.k : f.k;
        int si = 0, sj = 0;
        if (!single && f.shift_mode == STOKES_SHIFT_SPLITMIX) {
            si = (int)(splitmix64(f.seed, 2u * (uint64_t)t) % (uint64_t)f.ti);
            sj = (int)(splitmix64(f.seed, 2u * (uint64_t)t + 1u) % (uint64_t)f.tj);
        } else if (!single && f.shift_mode == STOKES_SHIFT_LIST) {
            si = f.shifts[2 * t];
            sj = f.shifts[2 * t + 1];
            if (si < 0 || si >= f.ti || sj < 0 || sj >= f.tj) return STOKES_ERR_ARG;
        }
        std::vector<BatchTiles<T>> tab(n);
        int total = 0, shi = 1, shj = 1;
        for (size_t q = 0; q < n; ++q) {
            const GInst<T> &x = gi[q];
            BatchTiles<T> &e = tab[q];
            e.g = x.g;
            e.c = x.c;
            e.vx = ax[q];
            e.vy = ay[q];
            e.ox = bx[q];
            e.oy = by[q];
            e.tg = make_tiles(x.g.nx, x.g.ny, x.ti, x.tj, si, sj);
            e.tile_begin = total;
            e.inst = x.inst;
            total += e.tg.ntx * e.tg.nty;
            shi = std::max(shi, std::min(x.ti, x.g.nx));
            shj = std::max(shj, std::min(x.tj, x.g.ny));
            std::swap(ax[q], bx[q]);
            std::swap(ay[q], by[q]);
        }
        const int ov = single ? 0 : f.overlap;
        // a TMA-staged shape (one-column or pair layout) fits by construction
        const bool staged = tma && ras_batched_tma(shi, shj, ov, sizeof(T), pair_mode);
        if (!staged && ras_batched_smem_bytes(shi, shj, ov, sizeof(T)) > (size_t)ras_max_smem()) return STOKES_ERR_ARG;
        TileLaunch<T> L;
        ST(upload(o, tab, &L.tab, s));
        {
            std::vector<int> tm((size_t)total);
            for (size_t q = 0; q < n; ++q)
                for (int u = 0; u < tab[q].tg.ntx * tab[q].tg.nty; ++u) tm[(size_t)tab[q].tile_begin + u] = (int)q;
            ST(upload(o, tm, &L.tmap, s));
        }
        L.maps = nullptr;
        L.square = true;
        for (size_t q = 0; q < n; ++q)
            L.square = L.square && tab[q].g.ihx == tab[q].g.ihy && tab[q].g.ihx2 == tab[q].g.ihy2;
        if (staged) {
            std::vector<CUtensorMap> m(n * (ras_batched_maps_bytes() / sizeof(CUtensorMap)));
            CK(ras_batched_encode<T>(tab.data(), (int)n, shi, shj, ov, pair_mode, m.data()));
            const CUtensorMap *dm = nullptr;
            ST(upload(o, m, &dm, s));
            L.maps = dm;
        }
        L.count = (int)n;
        L.total = total;
        L.ti = shi;
        L.tj = shj;
        L.ks = ks;
        L.overlap = ov;
        out->launches.push_back(L);
    }
    out->back = (n_outer & 1) != 0;
    return STOKES_OK;
}

// live (device, may be NULL): instances whose flag is 0 are skipped
template <typename T>
int run_group(const Group<T> &G, const int *live, const RasRun &run, cudaStream_t s, long long *nk)
{
    if (G.launches.empty()) return STOKES_OK;
    if (G.walls) {
        CK(batch_copy_walls<T>(G.lev, G.sub.map, G.sub.nseg, live, s));
        ++*nk;
    }
    for (const TileLaunch<T> &L : G.launches) {
        CK(launch_ras_batched<T>(L.tab, L.tmap, L.maps, L.count, L.total, L.ti, L.tj, L.ks, L.overlap, G.omega, live,
                                 run, L.square, s));
        ++*nk;
    }
    if (G.back) {
        CK(batch_copy<T>(G.lev, G.sub.map, G.sub.nseg, G.sub.nblocks, false, live, s));
        ++*nk;
    }
    return STOKES_OK;
}

bool jacobi_like(const stokes_smooth_params &p)
{
    return p.variant == STOKES_JACOBI || p.variant == STOKES_JACOBI_FUSED || p.variant == STOKES_JACOBI_BLOCKED ||
           (p.variant == STOKES_RAS && p.overlap >= p.k - 1);
}

// RAS form of `sweeps` sweeps of smoother p on tiles (Jacobi variants: 32 x 32
// tiles, k = 4, overlap 3, no shifts)
RasForm ras_form(const stokes_smooth_params &p, int sweeps, uint64_t seed, int shift_mode)
{
    RasForm f;
    f.sweeps = sweeps;
    f.omega = p.omega;
    f.shifts = nullptr;
    if (p.variant == STOKES_RAS) {
        f.ti = p.tile_i > 0 ? p.tile_i : 32;
        f.tj = p.tile_j > 0 ? p.tile_j : 32;
        f.k = p.k;
        f.overlap = p.overlap;
        f.shift_mode = shift_mode;
        f.seed = seed;
        f.shifts = p.shifts;
    } else {
        f.ti = f.tj = 32;
        f.k = 4;
        f.overlap = 3;
        f.shift_mode = STOKES_SHIFT_NONE;
        f.seed = 0;
    }
    return f;
}

} // namespace

// ---------------------------------------------------------------------------
// the batch object
// ---------------------------------------------------------------------------
struct BHier {
    bool stale = true;
    int dtype = -1, levels_req = -1, coarsest_req = -1;
    int Lmax = 0;
    std::vector<int> L;                 // levels per instance
    std::vector<std::vector<Dims>> d;   // [level][instance]
    size_t slab_elems[B_MAX_LEVELS] = {};
    void *slab[B_MAX_LEVELS][12] = {};  // ec en ivx ivy bx by vx vy rx ry sx sy
    std::vector<int> n, ubeg;           // coarsest unknowns, first unknown
    std::vector<size_t> aoff;           // offset of each instance's inverse
    int rows = 0;
    double *Ainv = nullptr, *bvec = nullptr, *xvec = nullptr;
};

enum { H_EC, H_EN, H_IVX, H_IVY, H_BX, H_BY, H_VX, H_VY, H_RX, H_RY, H_SX, H_SY, H_NF };

struct stokes_batch {
    int count = 0, dtype = 0, device = 0;
    size_t esize = 0, total = 0;
    cudaStream_t stream = nullptr;
    std::vector<Dims> d;            // outer grids (level 0)
    std::vector<double> lx, ly;
    void *eta_c = nullptr, *eta_n = nullptr, *fx = nullptr, *fy = nullptr, *bx = nullptr, *by = nullptr;
    void *sx = nullptr, *sy = nullptr, *ivx = nullptr, *ivy = nullptr;
    void *cax = nullptr, *cay = nullptr; // flux coefficients of the outer operator apply
    bool have_eta = false, have_f = false;
    Sub all;                        // every instance over (nx+1) x (ny+1)
    Sub all_tall;                   // the same, a tall map (the right-hand side)
    double *partials = nullptr;     // 2 per block of `all`
    double *dsum = nullptr, *dpq = nullptr, *dzq = nullptr, *alpha = nullptr, *beta = nullptr;
    int *dactive = nullptr, *hactive = nullptr;
    double *hsum = nullptr;
    void *kw[8] = {};               // outer work r, z, p, q (x, y)
    int *dstatus = nullptr, *hstatus = nullptr; // bounded-wait status word
    bool use_tma = true;            // STOKES_OPT_USE_TMA
    int pair_mode = 1;              // STOKES_OPT_PAIRED
    long long wait_limit = 2000000000LL;
    BHier *mg = nullptr;
    Owned base;                     // tables tied to the batch itself
    // smoothing plan cache
    Owned sm_own;
    bool sm_valid = false;
    stokes_smooth_params sm_key{};
    std::vector<int32_t> sm_shifts;
    const void *sm_v[2] = {};
    Group<float> sm_f32;
    Group<double> sm_f64;
    // outer tables (depend on the caller's v and p)
    Owned out_own;
    bool out_valid = false;
    const void *out_key[3] = {};
    const void *outer_tab = nullptr, *rhs_tab = nullptr;
    // V-cycle plan and graph
    Owned pc_own;
    cudaStream_t gstream = nullptr;
    cudaEvent_t gev[2] = {nullptr, nullptr};
    cudaGraphExec_t gexec = nullptr;
    unsigned char gkey[sizeof(stokes_mg_params)] = {};
    long long gkernels = 0;
    // flexible CG: the graph has no casts; the finest level's right-hand side
    // (table g_l0) is written by the CG update and z read from table g_fin,
    // both in the inner precision g_inner
    bool g_direct = false;
    int g_inner = -1;
    const void *g_l0 = nullptr, *g_fin = nullptr;
    long long kernels = 0;          // kernels launched so far
};

namespace {

RasRun run_of(const stokes_batch *b)
{
    RasRun r;
    r.allow_tma = b->use_tma;
    r.pair_mode = b->pair_mode;
    r.status = b->dstatus;
    r.wait_limit = b->wait_limit;
    return r;
}

void free_hier(BHier *h)
{
    if (!h) return;
    for (int l = 0; l < B_MAX_LEVELS; ++l)
        for (int f = 0; f < H_NF; ++f)
            if (h->slab[l][f]) {
                cudaFree(h->slab[l][f]);
                h->slab[l][f] = nullptr;
            }
    void *ps[] = {h->Ainv, h->bvec, h->xvec};
    for (void *p : ps)
        if (p) cudaFree(p);
    h->Ainv = h->bvec = h->xvec = nullptr;
    h->Lmax = 0;
}

int n_unknowns(int nx, int ny) { return ny * (nx - 1) + (ny - 1) * nx; }

void *at(void *slab, size_t off, size_t es) { return slab ? (void *)((char *)slab + off * es) : nullptr; }

MgLevel level_view(const BHier *h, int l, int i, size_t es)
{
    const Dims &d = h->d[l][i];
    MgLevel v{};
    v.nx = d.nx;
    v.ny = d.ny;
    v.pitch = d.pitch;
    v.elems = d.elems;
    v.hx = d.hx;
    v.hy = d.hy;
    void **fs[H_NF] = {&v.ec, &v.en, &v.ivx, &v.ivy, &v.bx, &v.by, &v.vx, &v.vy, &v.rx, &v.ry, &v.sx, &v.sy};
    for (int f = 0; f < H_NF; ++f) *fs[f] = at(h->slab[l][f], d.off, es);
    return v;
}

template <typename To, typename Ti>
int build_hier(stokes_batch *b, BHier *h, int levels, int coarsest)
{
    const size_t es = sizeof(Ti);
    const int n = b->count;
    cudaStream_t s = b->stream;
    h->L.assign(n, 1);
    h->Lmax = 1;
    for (int i = 0; i < n; ++i) {
        int nx = b->d[i].nx, ny = b->d[i].ny, L = 1;
        while (L < levels && L < B_MAX_LEVELS && nx % 2 == 0 && ny % 2 == 0 && nx > coarsest && ny > coarsest) {
            nx /= 2;
            ny /= 2;
            ++L;
        }
        if (n_unknowns(nx, ny) > B_MAX_DENSE || nx < 2 || ny < 2) return STOKES_ERR_ARG;
        h->L[i] = L;
        h->Lmax = std::max(h->Lmax, L);
    }
    h->d.assign(h->Lmax, std::vector<Dims>(n));
    for (int l = 0; l < h->Lmax; ++l) {
        for (int i = 0; i < n; ++i)
            if (l < h->L[i]) {
                const double sc = std::ldexp(1.0, l);
                h->d[l][i] = dims_of(b->d[i].nx >> l, b->d[i].ny >> l, b->d[i].hx * sc, b->d[i].hy * sc);
            }
        h->slab_elems[l] = place(h->d[l]);
        for (int f = 0; f < H_NF; ++f) {
            CK(cudaMalloc(&h->slab[l][f], h->slab_elems[l] * es));
            CK(cudaMemsetAsync(h->slab[l][f], 0, h->slab_elems[l] * es, s));
        }
    }
    // level 0 has the outer layout: cast the viscosity slab in one go
    CK((mg_cast<To, Ti>(b->total, b->eta_c, h->slab[0][H_EC], s)));
    CK((mg_cast<To, Ti>(b->total, b->eta_n, h->slab[0][H_EN], s)));
    for (int l = 1; l < h->Lmax; ++l)
        for (int i = 0; i < n; ++i)
            if (l < h->L[i]) CK(mg_coarsen_eta<Ti>(level_view(h, l - 1, i, es), level_view(h, l, i, es), s));
    for (int l = 0; l < h->Lmax; ++l)
        for (int i = 0; i < n; ++i)
            if (l < h->L[i]) {
                const MgLevel v = level_view(h, l, i, es);
                CK(launch_inv_diag<Ti>(make_grid<Ti>(v.nx, v.ny, v.pitch, v.hx, v.hy), (const Ti *)v.ec,
                                       (const Ti *)v.en, (Ti *)v.ivx, (Ti *)v.ivy, s));
            }
    // dense inverses of -M on every coarsest level
    h->n.assign(n, 0);
    h->ubeg.assign(n, 0);
    h->aoff.assign(n, 0);
    size_t asz = 0, nmax = 0;
    h->rows = 0;
    for (int i = 0; i < n; ++i) {
        const Dims &c = h->d[h->L[i] - 1][i];
        h->n[i] = n_unknowns(c.nx, c.ny);
        h->ubeg[i] = h->rows;
        h->rows += h->n[i];
        h->aoff[i] = asz;
        asz += (size_t)h->n[i] * h->n[i];
        nmax = std::max(nmax, (size_t)h->n[i]);
    }
    CK(cudaMalloc(&h->Ainv, asz * 8));
    CK(cudaMalloc(&h->bvec, (size_t)h->rows * 8));
    CK(cudaMalloc(&h->xvec, (size_t)h->rows * 8));
    // all factorisations in chunks whose work matrices fit in 1 GB: one
    // launch per kernel and chunk, one CTA (or column block) per instance
    double *A = nullptr, *W = nullptr;
    int *dst = nullptr;
    DenseJob *djobs = nullptr;
    int st = STOKES_OK;
    const size_t budget = (size_t)1 << 30;
    const size_t per = std::max(nmax * nmax * 16, (size_t)16);
    const int chunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)n, budget / per));
    cudaError_t e = cudaMalloc(&A, (size_t)chunk * nmax * nmax * 8);
    if (e == cudaSuccess) e = cudaMalloc(&W, (size_t)chunk * nmax * nmax * 8);
    if (e == cudaSuccess) e = cudaMalloc(&dst, (size_t)n * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&djobs, (size_t)chunk * sizeof(DenseJob));
    if (e == cudaSuccess) e = cudaMemsetAsync(dst, 0, (size_t)n * sizeof(int), s);
    std::vector<DenseJob> jobs(chunk);
    for (int i0 = 0; i0 < n && e == cudaSuccess; i0 += chunk) {
        const int c = std::min(chunk, n - i0);
        for (int q = 0; q < c; ++q) {
            const int i = i0 + q;
            const MgLevel v = level_view(h, h->L[i] - 1, i, es);
            DenseJob &jb = jobs[q];
            jb.nx = v.nx;
            jb.ny = v.ny;
            jb.pitch = v.pitch;
            jb.n = h->n[i];
            jb.ihx = 1.0 / v.hx;
            jb.ihy = 1.0 / v.hy;
            jb.ec = v.ec;
            jb.en = v.en;
            jb.A = A + (size_t)q * nmax * nmax;
            jb.W = W + (size_t)q * nmax * nmax;
            jb.Ainv = h->Ainv + h->aoff[i];
            jb.status = dst + i;
        }
        e = cudaMemcpyAsync(djobs, jobs.data(), (size_t)c * sizeof(DenseJob), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = mg_dense_setup_many<Ti>(djobs, c, (int)nmax, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s); // the host table is rewritten next
    }
    std::vector<int> bad(n, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bad.data(), dst, (size_t)n * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "batch dense setup");
    cudaFree(A);
    cudaFree(W);
    cudaFree(dst);
    cudaFree(djobs);
    if (st != STOKES_OK) return st;
    for (int i = 0; i < n; ++i)
        if (bad[i]) return STOKES_ERR_DIVERGED;
    return STOKES_OK;
}

int ensure_hier(stokes_batch *b, const stokes_mg_params *p)
{
    if (!b->mg) {
        b->mg = new (std::nothrow) BHier();
        if (!b->mg) return STOKES_ERR_OOM;
    }
    BHier *h = b->mg;
    if (!h->stale && h->dtype == p->inner_dtype && h->levels_req == p->levels && h->coarsest_req == p->coarsest)
        return STOKES_OK;
    CK(cudaStreamSynchronize(b->stream));
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    b->pc_own.release();
    free_hier(h);
    h->stale = true;
    int st;
    if (b->dtype == STOKES_F64)
        st = p->inner_dtype == STOKES_F64 ? build_hier<double, double>(b, h, p->levels, p->coarsest)
                                          : build_hier<double, float>(b, h, p->levels, p->coarsest);
    else
        st = p->inner_dtype == STOKES_F64 ? build_hier<float, double>(b, h, p->levels, p->coarsest)
                                          : build_hier<float, float>(b, h, p->levels, p->coarsest);
    if (st != STOKES_OK) {
        cudaStreamSynchronize(b->stream);
        free_hier(h);
        return st;
    }
    h->stale = false;
    h->dtype = p->inner_dtype;
    h->levels_req = p->levels;
    h->coarsest_req = p->coarsest;
    return STOKES_OK;
}

int ensure_work(stokes_batch *b)
{
    if (b->kw[0]) return STOKES_OK;
    b->out_valid = false; // the outer tables point at the work slabs
    for (void *&w : b->kw) {
        CK(cudaMalloc(&w, b->total * b->esize));
        CK(cudaMemsetAsync(w, 0, b->total * b->esize, b->stream));
    }
    return STOKES_OK;
}

// ---- the preconditioner z = B r of every instance ------------------------------
template <typename To, typename Ti>
struct Precond {
    Sub l0;
    const BOuter<To> *outer = nullptr;
    const BLevel<Ti> *lev[B_MAX_LEVELS] = {}; // zero-initial velocity buffers
    // velocity buffers after the pre-smoothing (and, as the prolongation
    // source, the next coarser level's after its post-smoothing): a smoothing
    // with an odd number of passes leaves its result in the level's scratch pair
    const BLevel<Ti> *mid[B_MAX_LEVELS] = {};
    const BLevel<Ti> *fin0 = nullptr; // level 0 after its post-smoothing (z)
    Sub fine[B_MAX_LEVELS], coarse[B_MAX_LEVELS];
    Group<Ti> grp[B_MAX_LEVELS][2][2]; // [level][phase][single-tile, tiled]
    const BDense<Ti> *dense = nullptr;
    int rows = 0;
};

template <typename To>
std::vector<BOuter<To>> outer_table(const stokes_batch *b, const void *vx, const void *vy)
{
    const size_t es = sizeof(To);
    std::vector<BOuter<To>> t(b->count);
    for (int i = 0; i < b->count; ++i) {
        const Dims &d = b->d[i];
        BOuter<To> &o = t[i];
        o.g = make_grid<To>(d.nx, d.ny, d.pitch, d.hx, d.hy);
        o.ec = (const To *)at(b->eta_c, d.off, es);
        o.en = (const To *)at(b->eta_n, d.off, es);
        o.ivx = (const To *)at(b->ivx, d.off, es);
        o.ivy = (const To *)at(b->ivy, d.off, es);
        o.ax = (const To *)at(b->cax, d.off, es);
        o.ay = (const To *)at(b->cay, d.off, es);
        o.fx = (const To *)at(b->fx, d.off, es);
        o.fy = (const To *)at(b->fy, d.off, es);
        o.bx = (const To *)at(b->bx, d.off, es);
        o.by = (const To *)at(b->by, d.off, es);
        o.vx = (To *)at((void *)vx, d.off, es);
        o.vy = (To *)at((void *)vy, d.off, es);
        To **w[8] = {&o.rx, &o.ry, &o.zx, &o.zy, &o.px, &o.py, &o.qx, &o.qy};
        for (int k = 0; k < 8; ++k) *w[k] = (To *)at(b->kw[k], d.off, es);
    }
    return t;
}

template <typename To, typename Ti>
int plan_precond(stokes_batch *b, const stokes_mg_params *p, Precond<To, Ti> *P)
{
    BHier *h = b->mg;
    Owned &o = b->pc_own;
    cudaStream_t s = b->stream;
    const size_t es = sizeof(Ti);
    const int n = b->count;
    P->l0 = b->all;
    {
        const std::vector<BOuter<To>> t = outer_table<To>(b, nullptr, nullptr);
        ST(upload(o, t, &P->outer, s));
    }
    // host copies of the level tables, and where each instance's velocity
    // lives after the pre- and the post-smoothing of each level
    struct VBuf {
        Ti *vx, *vy, *sx, *sy;
    };
    std::vector<std::vector<BLevel<Ti>>> tabs(h->Lmax);
    std::vector<std::vector<VBuf>> after_pre(h->Lmax, std::vector<VBuf>(n)), after_post(h->Lmax, std::vector<VBuf>(n));
    for (int l = 0; l < h->Lmax; ++l) {
        std::vector<BLevel<Ti>> &t = tabs[l];
        t.resize(n);
        std::memset((void *)t.data(), 0, t.size() * sizeof(BLevel<Ti>));
        std::vector<Rect> rf, rc;
        for (int i = 0; i < n; ++i) {
            if (l >= h->L[i]) continue;
            const MgLevel v = level_view(h, l, i, es);
            BLevel<Ti> &e = t[i];
            e.g = make_grid<Ti>(v.nx, v.ny, v.pitch, v.hx, v.hy);
            e.ec = (Ti *)v.ec;
            e.en = (Ti *)v.en;
            e.ivx = (Ti *)v.ivx;
            e.ivy = (Ti *)v.ivy;
            e.bx = (Ti *)v.bx;
            e.by = (Ti *)v.by;
            e.vx = (Ti *)v.vx;
            e.vy = (Ti *)v.vy;
            e.rx = (Ti *)v.rx;
            e.ry = (Ti *)v.ry;
            e.sx = (Ti *)v.sx;
            e.sy = (Ti *)v.sy;
            if (l < h->L[i] - 1) {
                const MgLevel c = level_view(h, l + 1, i, es);
                e.cnx = c.nx;
                e.cny = c.ny;
                e.cp = c.pitch;
                e.cbx = (Ti *)c.bx;
                e.cby = (Ti *)c.by;
                e.cvx = (Ti *)c.vx;
                e.cvy = (Ti *)c.vy;
                rf.push_back({i, v.nx + 1, v.ny + 1});
                rc.push_back({i, c.nx + 1, c.ny + 1});
            }
        }
        ST(upload(o, t, &P->lev[l], s));
        ST(make_sub(o, rf, &P->fine[l], s));
        ST(make_sub(o, rc, &P->coarse[l], s));
        std::vector<VBuf> cur(n);
        for (int i = 0; i < n; ++i) cur[i] = {t[i].vx, t[i].vy, t[i].sx, t[i].sy};
        // smoothing groups of this level: whole-level single tiles (Jacobi-like
        // smoothers on levels up to 64^2) and tiled instances
        if (l == h->Lmax - 1) {
            after_pre[l] = cur;
            after_post[l] = cur;
            continue;
        }
        const stokes_smooth_params sm = level_smoother(p->smoother, l);
        for (int ph = 0; ph < 2; ++ph) {
            const int sweeps = mg_sweeps(ph == 0 ? p->nu_pre : p->nu_post, p->nu_growth, l, p->nu_max);
            const uint64_t seed = splitmix64(sm.seed, 2u * (uint64_t)l + (uint64_t)ph);
            std::vector<GInst<Ti>> g1, g2;
            for (int i = 0; i < n; ++i) {
                if (l >= h->L[i] - 1) continue;
                const BLevel<Ti> &e = t[i];
                GInst<Ti> x;
                x.inst = i;
                x.g = e.g;
                x.c.eta_c = e.ec;
                x.c.eta_n = e.en;
                x.c.bx = e.bx;
                x.c.by = e.by;
                x.c.inv_dx = e.ivx;
                x.c.inv_dy = e.ivy;
                x.vx = cur[i].vx;
                x.vy = cur[i].vy;
                x.sx = cur[i].sx;
                x.sy = cur[i].sy;
                const bool single = jacobi_like(sm) && sweeps > 0 && ras_whole_level_tile(e.g.nx, e.g.ny, es);
                if (single) {
                    x.ti = e.g.nx;
                    x.tj = e.g.ny;
                    g1.push_back(x);
                } else {
                    const RasForm f = ras_form(sm, sweeps, seed, STOKES_SHIFT_SPLITMIX);
                    x.ti = f.ti;
                    x.tj = f.tj;
                    g2.push_back(x);
                }
            }
            // the single-tile schedule: all sweeps in one launch, no overlap, no shift
            RasForm f1 = ras_form(sm, sweeps, seed, STOKES_SHIFT_NONE);
            f1.k = std::max(sweeps, 1);
            f1.overlap = 0;
            // zero-initialised walls of v and s at inner levels: no wall copies
            ST(plan_group<Ti>(o, g1, f1, false, true, b->use_tma, b->pair_mode, P->lev[l], &P->grp[l][ph][0], s));
            ST(plan_group<Ti>(o, g2, ras_form(sm, sweeps, seed, STOKES_SHIFT_SPLITMIX), false, false, b->use_tma,
                              b->pair_mode, P->lev[l], &P->grp[l][ph][1], s));
            // an odd number of passes leaves the result in the scratch pair:
            // no copy back, the two pairs trade roles from here on
            const std::vector<GInst<Ti>> *gs[2] = {&g1, &g2};
            for (int q = 0; q < 2; ++q) {
                Group<Ti> &G = P->grp[l][ph][q];
                if (!G.back) continue;
                G.back = false;
                for (const GInst<Ti> &x : *gs[q]) {
                    std::swap(cur[x.inst].vx, cur[x.inst].sx);
                    std::swap(cur[x.inst].vy, cur[x.inst].sy);
                }
            }
            if (ph == 0) after_pre[l] = cur;
        }
        after_post[l] = cur;
    }
    // tables of the residual, restriction and prolongation (fine velocity after
    // the pre-smoothing, coarse velocity after its post-smoothing) and of z
    for (int l = 0; l + 1 < h->Lmax; ++l) {
        std::vector<BLevel<Ti>> t = tabs[l];
        for (int i = 0; i < n; ++i) {
            if (l >= h->L[i] - 1) continue;
            t[i].vx = after_pre[l][i].vx;
            t[i].vy = after_pre[l][i].vy;
            t[i].sx = after_pre[l][i].sx;
            t[i].sy = after_pre[l][i].sy;
            t[i].cvx = after_post[l + 1][i].vx;
            t[i].cvy = after_post[l + 1][i].vy;
        }
        ST(upload(o, t, &P->mid[l], s));
    }
    {
        std::vector<BLevel<Ti>> t = tabs[0];
        for (int i = 0; i < n; ++i) {
            t[i].vx = after_post[0][i].vx;
            t[i].vy = after_post[0][i].vy;
        }
        ST(upload(o, t, &P->fin0, s));
    }
    std::vector<BDense<Ti>> dt(n);
    for (int i = 0; i < n; ++i) {
        const MgLevel c = level_view(h, h->L[i] - 1, i, es);
        BDense<Ti> &e = dt[i];
        e.nx = c.nx;
        e.ny = c.ny;
        e.pitch = c.pitch;
        e.n = h->n[i];
        e.Ainv = h->Ainv + h->aoff[i];
        e.bvec = h->bvec + h->ubeg[i];
        e.xvec = h->xvec + h->ubeg[i];
        e.bx = (const Ti *)c.bx;
        e.by = (const Ti *)c.by;
        e.vx = (Ti *)c.vx;
        e.vy = (Ti *)c.vy;
        e.unk_begin = h->ubeg[i];
    }
    ST(upload(o, dt, &P->dense, s));
    P->rows = h->rows;
    return STOKES_OK;
}

// One application of z = B r for every instance (the order of the
// single-problem V-cycle, instances in lockstep by level).
// Instances whose live flag is 0 (converged, diverged or out of cycles) are
// skipped: their z keeps its last value, which the outer iteration no
// longer uses.
template <typename To, typename Ti>
int enqueue_precond(const Precond<To, Ti> &P, int Lmax, int count, const int *live, const RasRun &run,
                    cudaStream_t s, long long *nk, bool casts)
{
    if (casts) {
        CK((batch_cast_in<To, Ti>(P.outer, P.lev[0], P.l0.map, P.l0.nseg, P.l0.nblocks, live, s)));
        ++*nk;
    }
    for (int l = 0; l < Lmax - 1; ++l) {
        CK(batch_zero_v<Ti>(P.lev[l], P.fine[l].map, P.fine[l].nseg, P.fine[l].nblocks, live, s));
        ++*nk;
    }
    for (int l = 0; l < Lmax - 1; ++l) {
        ST(run_group<Ti>(P.grp[l][0][0], live, run, s, nk));
        ST(run_group<Ti>(P.grp[l][0][1], live, run, s, nk));
        CK(batch_residual<Ti>(P.mid[l], P.fine[l].map, P.fine[l].nseg, P.fine[l].nblocks, live, s));
        CK(batch_restrict<Ti>(P.mid[l], P.coarse[l].map, P.coarse[l].nseg, P.coarse[l].nblocks, live, s));
        *nk += 2;
    }
    CK(batch_dense<Ti>(P.dense, count, P.rows, live, s));
    *nk += 3;
    for (int l = Lmax - 2; l >= 0; --l) {
        CK(batch_prolong<Ti>(P.mid[l], P.fine[l].map, P.fine[l].nseg, P.fine[l].nblocks, live, s));
        ++*nk;
        ST(run_group<Ti>(P.grp[l][1][0], live, run, s, nk));
        ST(run_group<Ti>(P.grp[l][1][1], live, run, s, nk));
    }
    if (casts) {
        CK((batch_cast_out<To, Ti>(P.outer, P.fin0, P.l0.map, P.l0.nseg, P.l0.nblocks, live, s)));
        ++*nk;
    }
    return STOKES_OK;
}

template <typename To, typename Ti>
int capture(stokes_batch *b, const stokes_mg_params *p)
{
    Precond<To, Ti> P;
    ST((plan_precond<To, Ti>(b, p, &P)));
    long long nk = 0;
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(b->gstream, cudaStreamCaptureModeThreadLocal));
    const bool direct = p->krylov != 0;
    const int st = enqueue_precond<To, Ti>(P, b->mg->Lmax, b->count, b->dactive, run_of(b), b->gstream, &nk,
                                           !direct);
    const cudaError_t e = cudaStreamEndCapture(b->gstream, &graph);
    if (st != STOKES_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    const cudaError_t ei = cudaGraphInstantiate(&b->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        b->gexec = nullptr;
        return cuda_fail(ei, "cudaGraphInstantiate");
    }
    b->gkernels = nk;
    b->g_direct = direct;
    b->g_inner = p->inner_dtype == STOKES_F64 ? STOKES_F64 : STOKES_F32;
    b->g_l0 = P.lev[0];
    b->g_fin = P.fin0;
    return STOKES_OK;
}

int ensure_graph(stokes_batch *b, const stokes_mg_params *p)
{
    if (b->gexec && std::memcmp(p, b->gkey, sizeof *p) == 0) return STOKES_OK;
    CK(cudaStreamSynchronize(b->stream));
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    b->pc_own.release();
    if (!b->gstream) {
        CK(cudaStreamCreateWithFlags(&b->gstream, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&b->gev[0], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&b->gev[1], cudaEventDisableTiming));
    }
    int st;
    const bool in64 = p->inner_dtype == STOKES_F64;
    if (b->dtype == STOKES_F64) st = in64 ? capture<double, double>(b, p) : capture<double, float>(b, p);
    else st = in64 ? capture<float, double>(b, p) : capture<float, float>(b, p);
    if (st != STOKES_OK) return st;
    std::memcpy(b->gkey, p, sizeof *p);
    return STOKES_OK;
}

int replay(stokes_batch *b)
{
    CK(cudaEventRecord(b->gev[0], b->stream));
    CK(cudaStreamWaitEvent(b->gstream, b->gev[0], 0));
    CK(cudaGraphLaunch(b->gexec, b->gstream));
    CK(cudaEventRecord(b->gev[1], b->gstream));
    CK(cudaStreamWaitEvent(b->stream, b->gev[1], 0));
    b->kernels += b->gkernels;
    return STOKES_OK;
}

// ---- outer tables: the caller's v and p ---------------------------------------
template <typename T>
int ensure_outer(stokes_batch *b, const void *vx, const void *vy, const void *p)
{
    if (b->out_valid && b->out_key[0] == vx && b->out_key[1] == vy && b->out_key[2] == p) return STOKES_OK;
    CK(cudaStreamSynchronize(b->stream));
    b->out_own.release();
    b->out_valid = false;
    const size_t es = sizeof(T);
    const std::vector<BOuter<T>> t = outer_table<T>(b, vx, vy);
    const BOuter<T> *dt = nullptr;
    ST(upload(b->out_own, t, &dt, b->stream));
    std::vector<BRhs<T>> r(b->count);
    for (int i = 0; i < b->count; ++i) {
        const Dims &d = b->d[i];
        r[i].g = t[i].g;
        r[i].fx = t[i].fx;
        r[i].fy = t[i].fy;
        r[i].p = (const T *)at((void *)p, d.off, es);
        r[i].bx = (T *)at(b->bx, d.off, es);
        r[i].by = (T *)at(b->by, d.off, es);
    }
    const BRhs<T> *dr = nullptr;
    ST(upload(b->out_own, r, &dr, b->stream));
    b->outer_tab = dt;
    b->rhs_tab = dr;
    b->out_key[0] = vx;
    b->out_key[1] = vy;
    b->out_key[2] = p;
    b->out_valid = true;
    return STOKES_OK;
}

template <typename T>
int rhs(stokes_batch *b)
{
    CK(batch_rhs<T>((const BRhs<T> *)b->rhs_tab, b->all_tall.map, b->all_tall.nseg, b->all_tall.nblocks, b->stream));
    ++b->kernels;
    return STOKES_OK;
}

// per-instance sums of the last reduction (2 doubles each), synchronising;
// reports (and clears) a bounded wait that gave up since the last check
int read_sums(stokes_batch *b, const double *dev)
{
    CK(cudaMemcpyAsync(b->hsum, dev, 2 * (size_t)b->count * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    CK(cudaMemcpyAsync(b->hstatus, b->dstatus, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    if (*b->hstatus) {
        CK(cudaMemsetAsync(b->dstatus, 0, sizeof(int), b->stream));
        CK(cudaStreamSynchronize(b->stream));
        return STOKES_ERR_TIMEOUT;
    }
    return STOKES_OK;
}

template <typename T>
int solve_impl(stokes_batch *b, void *vx, void *vy, const void *p, const stokes_mg_params *prm, double *final_e,
               int *cycles, int *status)
{
    ST(ensure_hier(b, prm));
    ST(ensure_work(b));
    ST(ensure_graph(b, prm));
    ST(ensure_outer<T>(b, vx, vy, p));
    ST(rhs<T>(b));
    const BOuter<T> *ot = (const BOuter<T> *)b->outer_tab;
    const Sub &A = b->all;
    cudaStream_t s = b->stream;
    const int n = b->count;
    CK(batch_residual_energy<T>(ot, A.map, A.nseg, A.nblocks, b->partials, b->dsum, s));
    b->kernels += 2;
    ST(read_sums(b, b->dsum));
    std::vector<double> den(n), e(n), e0(n);
    std::vector<int> it(n, 0), verdict(n, 0);
    auto check = [&](int i) {
        if (!std::isfinite(e[i]) || e[i] > 1e6 * e0[i]) return (int)STOKES_ERR_DIVERGED;
        if (e[i] <= prm->tol) return 1;
        if (it[i] >= prm->max_cycles) return (int)STOKES_ERR_NOT_CONVERGED;
        return 0;
    };
    int live = 0;
    for (int i = 0; i < n; ++i) {
        den[i] = b->hsum[2 * i + 1];
        e[i] = e0[i] = std::sqrt(b->hsum[2 * i] / den[i]);
        verdict[i] = check(i);
        b->hactive[i] = verdict[i] == 0;
        live += b->hactive[i];
    }
    // after a reduction of the new E: update verdicts and the active flags
    auto advance = [&]() {
        live = 0;
        for (int i = 0; i < n; ++i) {
            if (!b->hactive[i]) continue;
            ++it[i];
            e[i] = std::sqrt(b->hsum[2 * i] / den[i]);
            verdict[i] = check(i);
            b->hactive[i] = verdict[i] == 0;
            live += b->hactive[i];
        }
    };
    if (live > 0) CK(cudaMemcpyAsync(b->dactive, b->hactive, n * sizeof(int), cudaMemcpyHostToDevice, s));
    auto fcg_direct = [&](auto tag) -> int {
        using Ti = decltype(tag);
        const BLevel<Ti> *l0 = (const BLevel<Ti> *)b->g_l0, *fin = (const BLevel<Ti> *)b->g_fin;
        CK((batch_cast_in<T, Ti>(ot, l0, A.map, A.nseg, A.nblocks, nullptr, s)));
        ST(replay(b));
        CK((batch_direction_in<T, Ti>(ot, fin, A.map, A.nseg, A.nblocks, nullptr, s)));
        b->kernels += 2;
        for (;;) {
            CK(batch_apply_dot<T>(ot, A.map, A.nseg, A.nblocks, b->partials, b->dpq, s));
            CK(batch_scalars(n, b->dpq, nullptr, b->dactive, b->alpha, nullptr, s));
            CK((batch_update_cast<T, Ti>(ot, l0, A.map, A.nseg, A.nblocks, b->alpha, b->partials, b->dsum, s)));
            b->kernels += 5;
            ST(read_sums(b, b->dsum));
            advance();
            if (live == 0) break;
            CK(cudaMemcpyAsync(b->dactive, b->hactive, n * sizeof(int), cudaMemcpyHostToDevice, s));
            ST(replay(b));
            CK((batch_dot_zq_in<T, Ti>(ot, fin, A.map, A.nseg, A.nblocks, b->partials, b->dzq, s)));
            CK(batch_scalars(n, b->dpq, b->dzq, b->dactive, nullptr, b->beta, s));
            CK((batch_direction_in<T, Ti>(ot, fin, A.map, A.nseg, A.nblocks, b->beta, s)));
            b->kernels += 4;
        }
        return STOKES_OK;
    };
    if (prm->krylov && live > 0 && b->g_direct) {
        ST(b->g_inner == STOKES_F64 ? fcg_direct(double{}) : fcg_direct(float{}));
    } else if (prm->krylov && live > 0) {
        ST(replay(b));
        CK(batch_direction<T>(ot, A.map, A.nseg, A.nblocks, nullptr, s));
        ++b->kernels;
        for (;;) {
            CK(batch_apply_dot<T>(ot, A.map, A.nseg, A.nblocks, b->partials, b->dpq, s));
            CK(batch_scalars(n, b->dpq, nullptr, b->dactive, b->alpha, nullptr, s));
            CK(batch_update<T>(ot, A.map, A.nseg, A.nblocks, b->alpha, b->partials, b->dsum, s));
            b->kernels += 5;
            ST(read_sums(b, b->dsum));
            advance();
            if (live == 0) break;
            CK(cudaMemcpyAsync(b->dactive, b->hactive, n * sizeof(int), cudaMemcpyHostToDevice, s));
            ST(replay(b));
            CK(batch_dot_zq<T>(ot, A.map, A.nseg, A.nblocks, b->partials, b->dzq, s));
            CK(batch_scalars(n, b->dpq, b->dzq, b->dactive, nullptr, b->beta, s));
            CK(batch_direction<T>(ot, A.map, A.nseg, A.nblocks, b->beta, s));
            b->kernels += 4;
        }
    } else {
        while (live > 0) {
            ST(replay(b));
            CK(batch_add<T>(ot, A.map, A.nseg, A.nblocks, b->dactive, s));
            CK(batch_residual_energy<T>(ot, A.map, A.nseg, A.nblocks, b->partials, b->dsum, s));
            b->kernels += 3;
            ST(read_sums(b, b->dsum));
            advance();
            if (live > 0) CK(cudaMemcpyAsync(b->dactive, b->hactive, n * sizeof(int), cudaMemcpyHostToDevice, s));
        }
    }
    int worst = STOKES_OK;
    for (int i = 0; i < n; ++i) {
        const int st = verdict[i] < 0 ? verdict[i] : STOKES_OK;
        if (final_e) final_e[i] = e[i];
        if (cycles) cycles[i] = it[i];
        if (status) status[i] = st;
        if (st == STOKES_ERR_DIVERGED) worst = st;
        else if (st != STOKES_OK && worst == STOKES_OK) worst = st;
    }
    return worst;
}

// ---- smoothing --------------------------------------------------------------
int check_smooth(const stokes_batch *b, const stokes_smooth_params *p)
{
    if (!p || p->sweeps < 0 || !(p->omega > 0.0) || !std::isfinite(p->omega)) return STOKES_ERR_ARG;
    if (p->variant < STOKES_JACOBI || p->variant > STOKES_RAS) return STOKES_ERR_ARG;
    if (p->variant == STOKES_RBGS) return STOKES_ERR_ARG; // in-place colour sweeps: not batched
    if (p->variant == STOKES_RAS) {
        if (p->k < 1 || p->overlap < 0 || p->tile_i < 0 || p->tile_j < 0) return STOKES_ERR_ARG;
        if (p->shift_mode < STOKES_SHIFT_NONE || p->shift_mode > STOKES_SHIFT_LIST) return STOKES_ERR_ARG;
        if (p->shift_mode == STOKES_SHIFT_LIST && !p->shifts && p->sweeps > 0) return STOKES_ERR_ARG;
        const int ti = p->tile_i > 0 ? p->tile_i : 32, tj = p->tile_j > 0 ? p->tile_j : 32;
        if (ras_batched_smem_bytes(ti, tj, p->overlap, b->esize) > (size_t)ras_max_smem()) return STOKES_ERR_ARG;
    }
    return STOKES_OK;
}

template <typename T>
Group<T> &sm_group(stokes_batch *b);
template <>
Group<float> &sm_group<float>(stokes_batch *b) { return b->sm_f32; }
template <>
Group<double> &sm_group<double>(stokes_batch *b) { return b->sm_f64; }

template <typename T>
int smooth_impl(stokes_batch *b, void *vx, void *vy, const void *p, const stokes_smooth_params *prm)
{
    ST(ensure_outer<T>(b, vx, vy, p));
    std::vector<int32_t> shifts;
    if (prm->variant == STOKES_RAS && prm->shift_mode == STOKES_SHIFT_LIST)
        shifts.assign(prm->shifts, prm->shifts + 2 * ((prm->sweeps + prm->k - 1) / prm->k));
    stokes_smooth_params key = *prm;
    key.shifts = nullptr;
    const bool same = b->sm_valid && std::memcmp(&key, &b->sm_key, sizeof key) == 0 && shifts == b->sm_shifts &&
                      b->sm_v[0] == vx && b->sm_v[1] == vy;
    Group<T> &G = sm_group<T>(b);
    if (!same) {
        CK(cudaStreamSynchronize(b->stream));
        b->sm_own.release();
        b->sm_valid = false;
        const size_t es = sizeof(T);
        std::vector<BLevel<T>> lev(b->count);
        std::memset((void *)lev.data(), 0, lev.size() * sizeof(BLevel<T>));
        std::vector<GInst<T>> gi;
        const RasForm f = ras_form(*prm, prm->sweeps, prm->seed, prm->shift_mode);
        for (int i = 0; i < b->count; ++i) {
            const Dims &d = b->d[i];
            BLevel<T> &e = lev[i];
            e.g = make_grid<T>(d.nx, d.ny, d.pitch, d.hx, d.hy);
            e.vx = (T *)at(vx, d.off, es);
            e.vy = (T *)at(vy, d.off, es);
            e.sx = (T *)at(b->sx, d.off, es);
            e.sy = (T *)at(b->sy, d.off, es);
            GInst<T> x;
            x.inst = i;
            x.g = e.g;
            x.c.eta_c = (const T *)at(b->eta_c, d.off, es);
            x.c.eta_n = (const T *)at(b->eta_n, d.off, es);
            x.c.bx = (const T *)at(b->bx, d.off, es);
            x.c.by = (const T *)at(b->by, d.off, es);
            x.c.inv_dx = (const T *)at(b->ivx, d.off, es);
            x.c.inv_dy = (const T *)at(b->ivy, d.off, es);
            x.vx = e.vx;
            x.vy = e.vy;
            x.sx = e.sx;
            x.sy = e.sy;
            x.ti = f.ti;
            x.tj = f.tj;
            gi.push_back(x);
        }
        const BLevel<T> *dlev = nullptr;
        RasForm ff = f;
        ff.shifts = shifts.empty() ? nullptr : shifts.data();
        ST(upload(b->sm_own, lev, &dlev, b->stream));
        ST(plan_group<T>(b->sm_own, gi, ff, true, false, b->use_tma, b->pair_mode, dlev, &G, b->stream));
        b->sm_key = key;
        b->sm_shifts = shifts;
        b->sm_v[0] = vx;
        b->sm_v[1] = vy;
        b->sm_valid = true;
    }
    ST(rhs<T>(b));
    long long nk = 0;
    const int st = run_group<T>(G, nullptr, run_of(b), b->stream, &nk);
    b->kernels += nk;
    return st;
}

template <typename T>
int energy_impl(stokes_batch *b, const void *vx, const void *vy, const void *p, double *out)
{
    ST(ensure_work(b));
    ST(ensure_outer<T>(b, vx, vy, p));
    ST(rhs<T>(b));
    const Sub &A = b->all;
    CK(batch_residual_energy<T>((const BOuter<T> *)b->outer_tab, A.map, A.nseg, A.nblocks, b->partials, b->dsum,
                                b->stream));
    b->kernels += 2;
    ST(read_sums(b, b->dsum));
    std::memcpy(out, b->hsum, 2 * (size_t)b->count * sizeof(double));
    return STOKES_OK;
}

int alloc_slab(stokes_batch *b, void **p)
{
    CK(cudaMalloc(p, b->total * b->esize));
    CK(cudaMemsetAsync(*p, 0, b->total * b->esize, b->stream));
    return STOKES_OK;
}

} // namespace

// ---------------------------------------------------------------------------
extern "C" {

int stokes_batch_create(int count, const int *nx, const int *ny, const double *lx, const double *ly, int dtype,
                        void *cuda_stream, stokes_batch **out)
{
    if (!out) return STOKES_ERR_ARG;
    *out = nullptr;
    if (count < 1 || count > (1 << 20) || !nx || !ny || !lx || !ly) return STOKES_ERR_ARG;
    if (dtype != STOKES_F32 && dtype != STOKES_F64) return STOKES_ERR_ARG;
    for (int i = 0; i < count; ++i)
        if (nx[i] < 2 || ny[i] < 2 || nx[i] > (1 << 16) || ny[i] > (1 << 16) || !(lx[i] > 0.0) || !(ly[i] > 0.0))
            return STOKES_ERR_ARG;
    stokes_batch *b = new (std::nothrow) stokes_batch();
    if (!b) return STOKES_ERR_OOM;
    b->count = count;
    b->dtype = dtype;
    b->esize = dtype == STOKES_F64 ? 8 : 4;
    b->stream = (cudaStream_t)cuda_stream;
    cudaGetDevice(&b->device);
    b->d.resize(count);
    b->lx.assign(lx, lx + count);
    b->ly.assign(ly, ly + count);
    for (int i = 0; i < count; ++i) b->d[i] = dims_of(nx[i], ny[i], lx[i] / nx[i], ly[i] / ny[i]);
    b->total = place(b->d);
    int st = STOKES_OK;
    void **fields[] = {&b->eta_c, &b->eta_n, &b->fx, &b->fy, &b->bx, &b->by, &b->sx, &b->sy, &b->ivx, &b->ivy,
                       &b->cax, &b->cay};
    for (void **f : fields)
        if ((st = alloc_slab(b, f)) != STOKES_OK) break;
    if (st == STOKES_OK) {
        std::vector<Rect> r;
        for (int i = 0; i < count; ++i) r.push_back({i, b->d[i].nx + 1, b->d[i].ny + 1});
        st = make_sub(b->base, r, &b->all, b->stream);
        if (st == STOKES_OK) st = make_sub(b->base, r, &b->all_tall, b->stream, BATCH_BY * BATCH_TALL);
    }
    if (st == STOKES_OK) {
        const size_t nb = (size_t)std::max(b->all.nblocks, 1);
        cudaError_t e = cudaMalloc(&b->partials, 2 * nb * sizeof(double));
        double **ds[] = {&b->dsum, &b->dpq, &b->dzq};
        for (double **q : ds)
            if (e == cudaSuccess) e = cudaMalloc(q, 2 * (size_t)count * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&b->alpha, (size_t)count * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&b->beta, (size_t)count * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&b->dactive, (size_t)count * sizeof(int));
        if (e == cudaSuccess) e = cudaMallocHost(&b->hactive, (size_t)count * sizeof(int));
        if (e == cudaSuccess) e = cudaMallocHost(&b->hsum, 2 * (size_t)count * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&b->dstatus, sizeof(int));
        if (e == cudaSuccess) e = cudaMemsetAsync(b->dstatus, 0, sizeof(int), b->stream);
        if (e == cudaSuccess) e = cudaMallocHost(&b->hstatus, sizeof(int));
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "stokes_batch_create");
    }
    if (st != STOKES_OK) {
        stokes_batch_destroy(b);
        return st;
    }
    *out = b;
    return STOKES_OK;
}

int stokes_batch_get_layout(const stokes_batch *b, int inst, int *pitch_elems, size_t *offset_elems,
                            size_t *alloc_elems)
{
    if (!b || inst < -1 || inst >= b->count) return STOKES_ERR_ARG;
    if (inst == -1) {
        if (pitch_elems) *pitch_elems = 0;
        if (offset_elems) *offset_elems = 0;
        if (alloc_elems) *alloc_elems = b->total;
        return STOKES_OK;
    }
    if (pitch_elems) *pitch_elems = b->d[inst].pitch;
    if (offset_elems) *offset_elems = b->d[inst].off;
    if (alloc_elems) *alloc_elems = b->d[inst].elems;
    return STOKES_OK;
}

int stokes_batch_set_viscosity(stokes_batch *b, const void *eta_c, const void *eta_n)
{
    if (!b || !eta_c || !eta_n) return STOKES_ERR_ARG;
    const size_t es = b->esize;
    for (int i = 0; i < b->count; ++i) {
        const Dims &d = b->d[i];
        int st;
        if (b->dtype == STOKES_F64) {
            const GridDesc<double> g = make_grid<double>(d.nx, d.ny, d.pitch, d.hx, d.hy);
            cudaError_t e = launch_copy_eta<double>(g, (const double *)at((void *)eta_c, d.off, es),
                                                    (const double *)at((void *)eta_n, d.off, es),
                                                    (double *)at(b->eta_c, d.off, es),
                                                    (double *)at(b->eta_n, d.off, es), b->stream);
            if (e == cudaSuccess)
                e = launch_inv_diag<double>(g, (const double *)at(b->eta_c, d.off, es),
                                            (const double *)at(b->eta_n, d.off, es), (double *)at(b->ivx, d.off, es),
                                            (double *)at(b->ivy, d.off, es), b->stream);
            if (e == cudaSuccess)
                e = kry_coef<double>(KrylovView{d.nx, d.ny, d.pitch, nullptr, nullptr}, g,
                                     (const double *)at(b->eta_c, d.off, es), (double *)at(b->cax, d.off, es),
                                     (double *)at(b->cay, d.off, es), b->stream);
            st = e == cudaSuccess ? STOKES_OK : cuda_fail(e, "stokes_batch_set_viscosity");
        } else {
            const GridDesc<float> g = make_grid<float>(d.nx, d.ny, d.pitch, d.hx, d.hy);
            cudaError_t e = launch_copy_eta<float>(g, (const float *)at((void *)eta_c, d.off, es),
                                                   (const float *)at((void *)eta_n, d.off, es),
                                                   (float *)at(b->eta_c, d.off, es), (float *)at(b->eta_n, d.off, es),
                                                   b->stream);
            if (e == cudaSuccess)
                e = launch_inv_diag<float>(g, (const float *)at(b->eta_c, d.off, es),
                                           (const float *)at(b->eta_n, d.off, es), (float *)at(b->ivx, d.off, es),
                                           (float *)at(b->ivy, d.off, es), b->stream);
            if (e == cudaSuccess)
                e = kry_coef<float>(KrylovView{d.nx, d.ny, d.pitch, nullptr, nullptr}, g,
                                    (const float *)at(b->eta_c, d.off, es), (float *)at(b->cax, d.off, es),
                                    (float *)at(b->cay, d.off, es), b->stream);
            st = e == cudaSuccess ? STOKES_OK : cuda_fail(e, "stokes_batch_set_viscosity");
        }
        if (st != STOKES_OK) return st;
        b->kernels += 3;
    }
    b->have_eta = true;
    if (b->mg) b->mg->stale = true;
    return STOKES_OK;
}

int stokes_batch_set_rhs(stokes_batch *b, const void *fx, const void *fy)
{
    if (!b || !fx || !fy) return STOKES_ERR_ARG;
    CK(cudaMemcpyAsync(b->fx, fx, b->total * b->esize, cudaMemcpyDeviceToDevice, b->stream));
    CK(cudaMemcpyAsync(b->fy, fy, b->total * b->esize, cudaMemcpyDeviceToDevice, b->stream));
    b->have_f = true;
    return STOKES_OK;
}

int stokes_batch_smooth(stokes_batch *b, void *vx, void *vy, const void *p, const stokes_smooth_params *params)
{
    if (!b || !vx || !vy) return STOKES_ERR_ARG;
    ST(check_smooth(b, params));
    if (!b->have_eta || !b->have_f) return STOKES_ERR_STATE;
    if (b->dtype == STOKES_F64) return smooth_impl<double>(b, vx, vy, p, params);
    return smooth_impl<float>(b, vx, vy, p, params);
}

int stokes_batch_residual_energy(stokes_batch *b, const void *vx, const void *vy, const void *p, double *out)
{
    if (!b || !vx || !vy || !out) return STOKES_ERR_ARG;
    if (!b->have_eta || !b->have_f) return STOKES_ERR_STATE;
    if (b->dtype == STOKES_F64) return energy_impl<double>(b, vx, vy, p, out);
    return energy_impl<float>(b, vx, vy, p, out);
}

int stokes_batch_solve(stokes_batch *b, void *vx, void *vy, const void *p, const stokes_mg_params *params,
                       double *final_rel_resid, int *cycles, int *status)
{
    if (!b || !vx || !vy || !params) return STOKES_ERR_ARG;
    const stokes_mg_params &q = *params;
    if (q.levels < 1 || q.coarsest < 2 || q.nu_pre < 0 || q.nu_post < 0 || !(q.nu_growth >= 1.0) ||
        q.nu_max < 0 || q.max_cycles < 0 || !(q.tol >= 0.0) || (q.krylov != 0 && q.krylov != 1))
        return STOKES_ERR_ARG;
    if (q.inner_dtype != STOKES_F32 && q.inner_dtype != STOKES_F64) return STOKES_ERR_ARG;
    stokes_smooth_params sm = q.smoother;
    sm.sweeps = 0;
    sm.shift_mode = STOKES_SHIFT_SPLITMIX;
    sm.shifts = nullptr;
    const int es_in = q.inner_dtype == STOKES_F64 ? 8 : 4;
    if (sm.variant < STOKES_JACOBI || sm.variant > STOKES_MIXED || sm.variant == STOKES_RBGS || !(sm.omega > 0.0))
        return STOKES_ERR_ARG;
    if (sm.variant == STOKES_RAS || sm.variant == STOKES_MIXED) {
        if (sm.k < 1 || sm.overlap < 0 || sm.tile_i < 0 || sm.tile_j < 0) return STOKES_ERR_ARG;
        const int ti = sm.tile_i > 0 ? sm.tile_i : 32, tj = sm.tile_j > 0 ? sm.tile_j : 32;
        if (ras_batched_smem_bytes(ti, tj, sm.overlap, es_in) > (size_t)ras_max_smem()) return STOKES_ERR_ARG;
    }
    if (!b->have_eta || !b->have_f) return STOKES_ERR_STATE;
    if (b->dtype == STOKES_F64)
        return solve_impl<double>(b, vx, vy, p, params, final_rel_resid, cycles, status);
    return solve_impl<float>(b, vx, vy, p, params, final_rel_resid, cycles, status);
}

int stokes_batch_set_option(stokes_batch *b, int option, long long value)
{
    if (!b) return STOKES_ERR_ARG;
    switch (option) {
    case STOKES_OPT_USE_TMA:
    case STOKES_OPT_WAIT_LIMIT_CYCLES:
    case STOKES_OPT_PAIRED:
        if (option == STOKES_OPT_PAIRED && (value < 0 || value > 2)) return STOKES_ERR_ARG;
        // plans and the captured graph embed these: rebuild them
        CK(cudaStreamSynchronize(b->stream));
        if (b->gexec) {
            cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
        }
        b->pc_own.release();
        b->sm_own.release();
        b->sm_valid = false;
        if (option == STOKES_OPT_USE_TMA) b->use_tma = value != 0;
        else if (option == STOKES_OPT_PAIRED) b->pair_mode = (int)value;
        else b->wait_limit = value;
        return STOKES_OK;
    default: return STOKES_ERR_ARG;
    }
}

int stokes_batch_kernels(const stokes_batch *b, long long *kernels)
{
    if (!b || !kernels) return STOKES_ERR_ARG;
    *kernels = b->kernels;
    return STOKES_OK;
}

int stokes_batch_destroy(stokes_batch *b)
{
    if (!b) return STOKES_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    if (b->gstream) cudaStreamSynchronize(b->gstream);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->gstream) cudaStreamDestroy(b->gstream);
    for (cudaEvent_t e : b->gev)
        if (e) cudaEventDestroy(e);
    if (b->mg) {
        free_hier(b->mg);
        delete b->mg;
    }
    b->base.release();
    b->sm_own.release();
    b->out_own.release();
    b->pc_own.release();
    for (void *w : b->kw)
        if (w) cudaFree(w);
    void *fs[] = {b->eta_c, b->eta_n, b->fx, b->fy, b->bx, b->by, b->sx, b->sy, b->ivx, b->ivy, b->cax, b->cay,
                  b->partials, b->dsum, b->dpq, b->dzq, b->alpha, b->beta, b->dactive, b->dstatus};
    for (void *f : fs)
        if (f) cudaFree(f);
    if (b->hactive) cudaFreeHost(b->hactive);
    if (b->hsum) cudaFreeHost(b->hsum);
    if (b->hstatus) cudaFreeHost(b->hstatus);
    delete b;
    return STOKES_OK;
}

} // extern "C"
