// internal.h -- declarations shared by the translation units of libstokes.
// Not part of the public interface (include/stokes.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>

namespace stokes {

// Geometry and coefficients of one grid level, passed by value to kernels.
// Every field of the level is a (ny+1) x pitch array (see include/stokes.h).
template <typename T>
struct GridDesc {
    int nx, ny, pitch;
    T ihx, ihy;   // 1/hx, 1/hy
    T ihx2, ihy2; // 1/hx^2, 1/hy^2
    T two_ihx2, two_ihy2; // 2/hx^2, 2/hy^2
    double lap;   // 2/hx^2 + 2/hy^2 (pressure weight of the energy norm)
    int square;   // 1/hx = 1/hy and 1/hx^2 = 1/hy^2 in T: the square-cell form of the shear fluxes
};

template <typename T>
GridDesc<T> make_grid(int nx, int ny, int pitch, double hx, double hy)
{
    GridDesc<T> g;
    g.nx = nx;
    g.ny = ny;
    g.pitch = pitch;
    g.ihx = (T)(1.0 / hx);
    g.ihy = (T)(1.0 / hy);
    g.ihx2 = (T)(1.0 / (hx * hx));
    g.ihy2 = (T)(1.0 / (hy * hy));
    g.two_ihx2 = g.ihx2 + g.ihx2;
    g.two_ihy2 = g.ihy2 + g.ihy2;
    g.lap = 2.0 / (hx * hx) + 2.0 / (hy * hy);
    g.square = g.ihx == g.ihy && g.ihx2 == g.ihy2 ? 1 : 0;
    return g;
}

// Velocity-operator coefficients: eta_c and eta_n with the boundary nodes
// zeroed (no shear stress there), plus the right-hand side b.
template <typename T>
struct Coeffs {
    const T *eta_c;
    const T *eta_n; // boundary nodes hold 0
    const T *bx, *by;
    const T *inv_dx, *inv_dy; // 1 / diag(M) at the unknowns (zero elsewhere), or NULL
};

// ---- stencil kernels (stencil_kernels.cu) --------------------------------
template <typename T>
cudaError_t launch_copy_eta(const GridDesc<T> &g, const T *eta_c_in, const T *eta_n_in, T *eta_c, T *eta_n,
                            cudaStream_t s);
// inv_dx, inv_dy = 1 / diag(M) at the unknowns, zero elsewhere
template <typename T>
cudaError_t launch_inv_diag(const GridDesc<T> &g, const T *eta_c, const T *eta_n, T *inv_dx, T *inv_dy,
                            cudaStream_t s);
// launch_copy_eta and launch_inv_diag in one pass (the same values)
template <typename T>
cudaError_t launch_set_eta(const GridDesc<T> &g, const T *eta_c_in, const T *eta_n_in, T *eta_c, T *eta_n, T *inv_dx,
                           T *inv_dy, cudaStream_t s);
template <typename T>
cudaError_t launch_rhs(const GridDesc<T> &g, const T *fx, const T *fy, const T *p, T *bx, T *by, cudaStream_t s);
template <typename T>
cudaError_t launch_apply(const GridDesc<T> &g, const T *eta_c, const T *eta_n, const T *vx, const T *vy, const T *p,
                         T *ox, T *oy, cudaStream_t s);
// variant 0: separate vx and vy passes; 1: fused pass.  Reads (vx, vy), writes
// the unknowns and walls of (ox, oy).
template <typename T>
cudaError_t launch_jacobi(const GridDesc<T> &g, const Coeffs<T> &c, T omega, const T *vx, const T *vy, T *ox, T *oy,
                          int fused, cudaStream_t s);
// One red-black Gauss-Seidel sweep (vx red, vx black, vy red, vy black):
// reads (vx, vy), writes the unknowns of (ox, oy).
template <typename T>
cudaError_t launch_rbgs_sweep(const GridDesc<T> &g, const Coeffs<T> &c, T omega, const T *vx, const T *vy, T *ox,
                              T *oy, cudaStream_t s);
// copy the in-extent entries (unknowns and walls) of vx, vy
template <typename T>
cudaError_t launch_copy_velocity(const GridDesc<T> &g, const T *vx, const T *vy, T *ox, T *oy, cudaStream_t s);
template <typename T>
cudaError_t launch_copy_walls(const GridDesc<T> &g, const T *vx, const T *vy, T *ox, T *oy, cudaStream_t s);
// Energy sums (3 doubles) into out[0..2] on the device; `partials` holds
// energy_partials() * 3 doubles.
int energy_partials();
// b = f - G p is formed on the fly (p may be NULL); inv_dx/inv_dy may be NULL
template <typename T>
cudaError_t launch_energy(const GridDesc<T> &g, const T *eta_c, const T *eta_n, const T *inv_dx, const T *inv_dy,
                          const T *fx, const T *fy, const T *p, const T *vx, const T *vy, double *partials,
                          double *out, cudaStream_t s);

// The FP32 sums by row-marching warps (the library's viscosity copies; 1/diag
// from inv_dx / inv_dy, or formed from the viscosity when they are NULL);
// writes `*nblocks` <= energy_partials() partial triples.
cudaError_t launch_energy_rows(const GridDesc<float> &g, const float *eta_c, const float *eta_n, const float *fx,
                               const float *fy, const float *inv_dx, const float *inv_dy, const float *p,
                               const float *vx, const float *vy, double *partials, int *nblocks, cudaStream_t s);

// The same sums from the caller's raw viscosity (boundary nodes of eta_n
// zeroed on the fly, 1/diag computed in the kernel); `partials` holds
// energy_partials() * 3 doubles.
template <typename T>
cudaError_t launch_energy_raw(const GridDesc<T> &g, const T *eta_c, const T *eta_n, const T *fx, const T *fy,
                              const T *p, const T *vx, const T *vy, double *partials, double *out, cudaStream_t s);

// ---- tiled / RAS kernel (ras_kernels.cu) ---------------------------------
struct TileGrid {
    int ti, tj;   // tile size (cells)
    int si, sj;   // shift
    int ntx, nty; // tiles per direction
};
TileGrid make_tiles(int nx, int ny, int ti, int tj, int si, int sj);
// Per-launch options of the tile kernels.
struct RasRun {
    bool allow_tma;        // use the persistent TMA-staged kernel when the window fits
    int pair_mode = 1;     // FP32 packed-pair TMA kernel: 0 never, 1 windows of 49-64 columns, 2 any window <= 64
    int *status;           // device word set to 1 when a bounded wait gives up
    long long wait_limit;  // SM cycles a wait may take
};
// One RAS outer iteration: `ksweeps` local Jacobi sweeps on each tile grown by
// `overlap`, reading (vx, vy), writing the owned unknowns to (ox, oy).
template <typename T>
cudaError_t launch_ras(const GridDesc<T> &g, const Coeffs<T> &c, T omega, const TileGrid &tg, int ksweeps,
                       int overlap, const T *vx, const T *vy, T *ox, T *oy, const RasRun &run, cudaStream_t s);
// shared memory a RAS launch needs for this grid, tile and overlap
size_t ras_smem_bytes(int nx, int ny, int ti, int tj, int overlap, size_t elem);
// Whether a Jacobi-equivalent smoothing of an nx x ny level runs all its sweeps
// as one launch with the whole level as one tile (its window fits a register
// layout); the single-context and the batched V-cycle take the same decision.
bool ras_whole_level_tile(int nx, int ny, size_t elem);
// the tile kernel (stokes_tile_kernel value), CTA size and dynamic shared memory of a launch
void ras_kernel_plan(int nx, int ny, int ti, int tj, int overlap, size_t elem, bool allow_tma, int pair_mode,
                     int *kind, int *threads, size_t *smem);

// One instance's share of a batched tile launch: its grid, coefficients,
// snapshot (vx, vy) -> output (ox, oy), tiling, and the index of its first
// tile in the launch's tile list.
template <typename T>
struct BatchTiles {
    GridDesc<T> g;
    Coeffs<T> c;
    const T *vx, *vy;
    T *ox, *oy;
    TileGrid tg;
    int tile_begin;
    int inst; // index into the launch's `live` flags
};
// One RAS outer iteration (ksweeps local sweeps) for every instance of the
// device table `tab` (count entries, tiles numbered consecutively, `total`
// tiles), all with tile size (ti, tj) and `overlap`: one persistent launch.
// `tmap` (device, may be NULL): the table entry of every tile of the launch
// (else found by binary search on tile_begin).  `maps` (device, may be
// NULL): the tensor maps of every instance, filled by ras_batched_encode;
// with them the windows are staged by TMA.  `live` (device, may be NULL):
// tiles of entries whose live[inst] is 0 are skipped.  `square`: every
// instance has square cells (1/hx = 1/hy bit for bit), which lets an FP32
// launch of the pair layout use its square-cell form.
template <typename T>
cudaError_t launch_ras_batched(const BatchTiles<T> *tab, const int *tmap, const void *maps, int count, int total,
                               int ti, int tj, int ksweeps, int overlap, T omega, const int *live, const RasRun &run,
                               bool square, cudaStream_t s);
// Shared memory one batched launch needs (tile size and overlap only).
size_t ras_batched_smem_bytes(int ti, int tj, int overlap, size_t elem);
// Whether a batched launch of this shape can stage windows by TMA (in the
// one-column or, with pair_mode as STOKES_OPT_PAIRED, the pair layout), the
// bytes of one instance's tensor maps, and their encoding for the host table
// `tab` (count entries) into the host buffer `out` (count * ras_batched_maps_bytes()).
bool ras_batched_tma(int ti, int tj, int overlap, size_t elem, int pair_mode);
size_t ras_batched_maps_bytes();
template <typename T>
cudaError_t ras_batched_encode(const BatchTiles<T> *tab, int count, int ti, int tj, int overlap, int pair_mode,
                               void *out);
int ras_max_smem();

// Record a failed CUDA call for stokes_last_cuda_error; returns
// STOKES_ERR_OOM for an allocation failure, else STOKES_ERR_CUDA.
int cuda_fail(cudaError_t e, const char *where);

// SplitMix64 (Steele, Lea & Flood 2014): output c (from 0) of the generator
// seeded with `seed`.
uint64_t splitmix64(uint64_t seed, uint64_t c);

// ---- inexact Uzawa iteration (uzawa.cu) ------------------------------------
// `partials` holds uzawa_partials() doubles; results land in device doubles.
int uzawa_partials();
template <typename T> // *out = min over cells and interior nodes
cudaError_t uz_eta_min(const GridDesc<T> &g, const T *ec, const T *en, double *partials, double *out, cudaStream_t s);
template <typename T> // continuation blend from the base viscosity (boundary nodes of on stay 0)
cudaError_t uz_blend(const GridDesc<T> &g, double theta, const double *emin, const T *bc, const T *bn, T *oc, T *on,
                     cudaStream_t s);
template <typename T> // p <- p - omega_p eta_c D v, then zero mean (*sum: the sum before the shift)
cudaError_t uz_pressure_update(const GridDesc<T> &g, double omega_p, const T *ec, const T *vx, const T *vy, T *p,
                               double *partials, double *sum, cudaStream_t s);
template <typename T> // lithostatic pressure of f_y, zero mean
cudaError_t uz_lithostatic(const GridDesc<T> &g, double hy, const T *fy, T *p, double *partials, double *sum,
                           cudaStream_t s);

// Anderson acceleration over x = (vx, vy, p): up to AA_MAX stored vectors.
constexpr int AA_MAX = 16;
template <typename T>
struct AndersonSet {
    const T *x[AA_MAX], *y[AA_MAX], *p[AA_MAX];
    int n;
};
struct AndersonAlpha {
    double a[AA_MAX];
};
// aa_multidot: `uzawa_partials() * AA_MAX` partials; out[j] = <a_0, hs_j> (three fields)
template <typename T>
cudaError_t aa_diff(size_t n, const T *f, const T *x, T *r, cudaStream_t s);
template <typename T>
cudaError_t aa_multidot(size_t n, const AndersonSet<T> &a, const AndersonSet<T> &hs, double *partials, double *out,
                        cudaStream_t s);
template <typename T>
cudaError_t aa_combine(size_t n, const AndersonSet<T> &F, const AndersonAlpha &al, T *x, T *y, T *p, cudaStream_t s);

// ---- smoother schedules (smooth.cu) ---------------------------------------
// Where kernel launches go: counts (and, for a context with timing on, times)
// each launch group of `nk` kernels of class `kind` (stokes_kernel_class).
struct LaunchHook {
    virtual int run(int kind, int nk, const std::function<cudaError_t()> &launch) = 0;
    virtual ~LaunchHook() = default;
};

// One smoothing call (the fields of stokes_smooth_params, tiles resolved).
struct SmoothSpec {
    int variant, sweeps, ti, tj, k, overlap, shift_mode;
    double omega;
    uint64_t seed;
    const int32_t *shifts;
};

// Smooth M v = b in place on (vx, vy) with the coefficients `k` (b included),
// ping-ponging through the scratch pair (sx, sy).  Returns a stokes_status.
// With `swapped` non-null, a result that ends in (sx, sy) after an odd number
// of passes is left there (*swapped = true) instead of being copied back; the
// caller then treats (sx, sy) as the velocity and (vx, vy) as the scratch.
// With a second scratch pair (tx, ty) (and no `swapped`), an odd number of
// passes ends in (vx, vy) by alternating between the two scratch pairs.
template <typename T>
int smooth_buffers(const GridDesc<T> &g, const Coeffs<T> &k, T *vx, T *vy, T *sx, T *sy, const SmoothSpec &p,
                   const RasRun &run, cudaStream_t s, LaunchHook &hook, bool *swapped = nullptr, T *tx = nullptr,
                   T *ty = nullptr);
// ping-pong passes of one smoothing call (0 for RBGS, which works in place)
int smooth_passes(const SmoothSpec &p);

} // namespace stokes
