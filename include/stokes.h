/*
 * stokes.h -- C ABI of libstokes, GB300 (sm_103a) smoothers for the 2D
 * variable-viscosity incompressible Stokes velocity operator on a fully
 * staggered finite-difference grid (arXiv 2509.19061).
 *
 * Grid and layout (Sec. 2.1 and Fig. 1 of the paper).  The domain
 * [0, lx] x [0, ly] has nx x ny cells, hx = lx/nx, hy = ly/ny:
 *   vx[j][i] at (i hx, (j+1/2) hy),       0 <= j < ny,  0 <= i <= nx
 *   vy[j][i] at ((i+1/2) hx, j hy),       0 <= j <= ny, 0 <= i < nx
 *   p[j][i], eta_c[j][i] at cell centres, 0 <= j < ny,  0 <= i < nx
 *   eta_n[j][i] at nodes (i hx, j hy),    0 <= j <= ny, 0 <= i <= nx
 *   fx like vx, fy like vy (density, and so the body force, sits with vy).
 * Every field buffer the caller passes is one pitched 2D array of
 * (ny+1) rows x `pitch` elements of the context's dtype (row j starts at
 * element j*pitch), whatever the field; stokes_get_layout returns the pitch
 * and each field's own extent.  Every field buffer starts on a 16-byte
 * boundary (any cudaMalloc or torch allocation does; the smoothing, solve and
 * energy entry points return STOKES_ERR_ARG otherwise).  Entries outside a field's extent
 * are padding: their values are never used (the kernels may read the bytes,
 * which lie inside the buffer), and output buffers get zeros there.  The unknowns are
 * vx with 1 <= i <= nx-1 and vy with 1 <= j <= ny-1; the wall entries
 * vx[.][0], vx[.][nx], vy[0][.], vy[ny][.] are Dirichlet data (zero for the
 * impermeable walls of Sec. 6.1), read but never written.  The shear stress is
 * zero on boundary nodes (free slip).
 *
 * Operator (Eq. (1)-(3), Eq. (6)): M v + G p = f, with
 *   sigma'_xx = 2 eta_c dvx/dx, sigma'_yy = 2 eta_c dvy/dy at centres,
 *   sigma'_xy = eta_n (dvx/dy + dvy/dx) at interior nodes, 0 on boundary nodes,
 *   (M v)_x = d sigma'_xx/dx + d sigma'_xy/dy, (M v)_y = d sigma'_xy/dx + d sigma'_yy/dy,
 *   (G p)_x = -dp/dx, (G p)_y = -dp/dy (the -grad p of Eq. (1)-(2)).
 *
 * Ownership.  The caller owns every field buffer (device memory from any
 * allocator, dtype of the context, the pitched layout above).  The library
 * owns its copies of eta and f, the right-hand side b = f - G p, the
 * ping-pong snapshot of the smoothers, the multigrid hierarchy and the
 * reduction buffers; it allocates them in stokes_create / stokes_set_viscosity
 * and frees them in stokes_destroy.
 *
 * Streams.  Every call enqueues its kernels on the stream given to
 * stokes_create (NULL = the legacy default stream) and returns without waiting,
 * except the calls that return host scalars (stokes_residual_energy_norm,
 * stokes_vcycle, stokes_batch_solve), which synchronise that stream.
 *
 * Errors.  Every call returns STOKES_OK (0) or a negative stokes_status;
 * nothing aborts.  A context is not thread-safe: use one per host thread.
 */
#ifndef STOKES_H
#define STOKES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    STOKES_OK = 0,
    STOKES_ERR_ARG = -1,           /* invalid argument (sizes, tiles, k, NULL pointer, ...) */
    STOKES_ERR_CUDA = -2,          /* a CUDA runtime call failed; see stokes_last_cuda_error */
    STOKES_ERR_OOM = -3,           /* device allocation failed */
    STOKES_ERR_DIVERGED = -4,      /* NaN/Inf or residual growth beyond 1e6x its initial value */
    STOKES_ERR_TIMEOUT = -5,       /* a bounded device-side wait gave up */
    STOKES_ERR_NOT_CONVERGED = -6, /* the solver stopped at max_cycles above tol */
    STOKES_ERR_STATE = -7          /* call out of order (e.g. smoothing before set_viscosity) */
} stokes_status;

typedef enum { STOKES_F32 = 0, STOKES_F64 = 1 } stokes_dtype;

/* The five smoothers of Sec. 5 of the paper. */
typedef enum {
    STOKES_JACOBI = 0,         /* (ii)  damped Jacobi, separate vx and vy passes (both read the old v) */
    STOKES_JACOBI_FUSED = 1,   /* (iii) the same map, vx and vy in one pass */
    STOKES_JACOBI_BLOCKED = 2, /* (iv)  the same map, one pass over shared-memory tiles */
    STOKES_RBGS = 3,           /* (i)   red-black Gauss-Seidel: vx red, vx black, vy red, vy black */
    STOKES_RAS = 4,            /* (v)   RAS-type temporally blocked Jacobi, Sec. 4.3 / Algorithm 2 */
    STOKES_MIXED = 5           /* V-cycle smoother only (stokes_mg_params): Jacobi on the finest level,
                                  RAS (with the smoother's tiles, k, overlap) on every coarser level,
                                  the "mixed" configuration of Sec. 6.3 */
} stokes_variant;

typedef enum {
    STOKES_FIELD_VX = 0,
    STOKES_FIELD_VY = 1,
    STOKES_FIELD_P = 2,
    STOKES_FIELD_ETA_C = 3,
    STOKES_FIELD_ETA_N = 4
} stokes_field;

/* Tile shifts of the RAS outer iterations (Algorithm 2, "draw random shifts"). */
typedef enum {
    STOKES_SHIFT_NONE = 0,     /* s_i = s_j = 0 */
    STOKES_SHIFT_SPLITMIX = 1, /* outer iteration t: s_i = SplitMix64(seed) output 2t mod tile_i,
                                  s_j = output 2t+1 mod tile_j (outputs numbered from 0) */
    STOKES_SHIFT_LIST = 2      /* s_i = shifts[2t], s_j = shifts[2t+1], host array */
} stokes_shift_mode;

typedef struct stokes_ctx stokes_ctx; /* opaque, library-owned */

/* Parameters of one smoothing call.
 * variant   stokes_variant.
 * sweeps    N >= 0: number of sweeps (N_max of Algorithm 2).
 * tile_i/j  tile size in cells for STOKES_RAS (T_I, T_J) and STOKES_JACOBI_BLOCKED;
 *           0 selects the library default (32 x 32).
 * k         RAS local sweeps per outer iteration (T_inner of Algorithm 2), >= 1.
 *           ceil(N/k) outer iterations run; the last one runs N - (ceil(N/k)-1) k.
 * overlap   RAS overlap o >= 0 in cells: each tile solves for the unknowns of
 *           its cells grown by o cells, with everything beyond frozen at the
 *           snapshot of the outer iteration (Dirichlet), and keeps only the
 *           unknowns of its own cells.  o >= k-1 reproduces global Jacobi
 *           exactly; o = 0 is the paper's ring-only tile.
 * omega     damping (omega_u = 0.3 in Sec. 6.3), 0 < omega.
 * seed, shift_mode, shifts   tile shifts (stokes_shift_mode); `shifts` is a host
 *           array of 2*ceil(N/k) ints used only with STOKES_SHIFT_LIST. */
typedef struct {
    int variant;
    int sweeps;
    int tile_i, tile_j;
    int k;
    int overlap;
    double omega;
    uint64_t seed;
    int shift_mode;
    const int32_t *shifts;
} stokes_smooth_params;

/* Parameters of the multigrid solve (Sec. 3.2; configuration of Sec. 6.2).
 * levels      maximum number of levels; coarsening halves nx and ny while both are
 *             even and larger than `coarsest`.
 * coarsest    stop coarsening at this size (cells per side); the coarsest level is
 *             solved exactly with a dense FP64 inverse of -M computed on the GPU,
 *             so it must have at most 1024 unknowns.
 * nu_pre, nu_post, nu_growth, nu_max   level l runs ceil(nu_pre nu_growth^l) pre- and
 *             ceil(nu_post nu_growth^l) post-sweeps (5, 5, 2.5 in Sec. 6.2), each
 *             capped at nu_max when nu_max > 0.
 * inner_dtype stokes_dtype of the V-cycle (smoothing, restriction, prolongation);
 *             the residual and the update of v stay in the context's dtype.
 * smoother    smoother of every level (variant, tiles, k, overlap, omega, seed;
 *             `sweeps`, `shift_mode` and `shifts` are ignored: a RAS smoother on
 *             level l, phase ph (0 pre, 1 post) draws SplitMix64 shifts seeded
 *             with output 2 l + ph of SplitMix64(seed), the same in every cycle).
 * krylov      0: defect correction, v += B (f - G p - M v) per cycle; 1: flexible
 *             conjugate gradients (one-term recurrence) with B as the
 *             preconditioner, which keeps converging at high viscosity
 *             contrast where defect correction stagnates.  B is one V-cycle.
 *             2: defect correction in the context's precision whose correction
 *             is `inner_its` flexible-CG iterations run entirely in inner_dtype
 *             (operator, inner products accumulated in FP64, updates), each
 *             preconditioned by B: the outer residual is formed in the
 *             context's precision once per `inner_its` V-cycles only.
 * tol         stop when the relative velocity energy residual E_v <= tol.
 * max_cycles  at most this many V-cycles (applications of B).
 * inner_its   flexible-CG iterations per outer step when krylov = 2 (>= 1);
 *             ignored otherwise.  Not supported by stokes_batch_solve. */
typedef struct {
    int levels;
    int coarsest;
    int nu_pre, nu_post;
    double nu_growth;
    int nu_max;
    int inner_dtype;
    stokes_smooth_params smoother;
    int krylov;
    double tol;
    int max_cycles;
    int inner_its;
} stokes_mg_params;

/* Create a context for an nx x ny grid on [0, lx] x [0, ly] computing in `dtype`
 * on `cuda_stream` (a cudaStream_t, NULL for the legacy default stream) of the
 * current device.  2 <= nx, ny <= 262144 (larger sides are rejected with
 * STOKES_ERR_ARG); lx, ly > 0.  *out is set on success, NULL
 * otherwise.  Allocates the library's per-grid buffers.  (Sec. 2.1.) */
int stokes_create(int nx, int ny, double lx, double ly, int dtype, void *cuda_stream, stokes_ctx **out);

/* Layout of the field buffers: every buffer is (ny+1) x *pitch_elems elements
 * (*alloc_elems in total, may be NULL); *rows x *cols is the extent of `field`
 * (stokes_field) inside it.  Any output pointer may be NULL. */
int stokes_get_layout(const stokes_ctx *ctx, int field, int *rows, int *cols, int *pitch_elems,
                      size_t *alloc_elems);

/* Set the viscosity at cell centres (eta_c, "eta_P") and nodes (eta_n,
 * "eta_B"), Fig. 1.  Device pointers in the context's layout and dtype, read
 * once and copied; every viscosity must be positive and finite (not checked
 * on the device).  Invalidates the multigrid hierarchy, which the next
 * stokes_vcycle rebuilds. */
int stokes_set_viscosity(stokes_ctx *ctx, const void *eta_c, const void *eta_n);

/* Set the body force f of Eq. (6) (fx like vx, fy like vy; f_y = -rho g_y for
 * Eq. (2) with gravity g_y).  Device pointers, copied at the unknowns (the
 * wall and padding entries are not read). */
int stokes_set_rhs(stokes_ctx *ctx, const void *fx, const void *fy);

/* out = M v + G p at every unknown (Eq. (6) left-hand side), zero on walls and
 * padding.  p may be NULL (p = 0).  out_x/out_y must not alias vx/vy/p. */
int stokes_apply_operator(stokes_ctx *ctx, const void *vx, const void *vy, const void *p, void *out_x, void *out_y);

/* Smooth M v = f - G p in place on (vx, vy) with the smoother of `params`
 * (Sec. 5).  p may be NULL (p = 0).  Requires stokes_set_viscosity and
 * stokes_set_rhs.  Asynchronous.  The passes ping-pong between (vx, vy) and
 * context-owned scratch fields; the first call whose pass count is odd and at
 * least 3 (RAS: ceil(sweeps / k) outer iterations; Jacobi variants: one pass
 * per sweep) allocates a second scratch pair (two fields) so that the result
 * ends in (vx, vy) without a copy: make that call once before capturing
 * stokes_smooth into a CUDA graph.  Returns STOKES_ERR_OOM if that allocation
 * fails. */
int stokes_smooth(stokes_ctx *ctx, void *vx, void *vy, const void *p, const stokes_smooth_params *params);

/* Energy residual sums of Sec. 6.4, accumulated in FP64:
 *   out[0] = sum over velocity unknowns of r_v^2 / (-diag M),  r_v = f - G p - M v
 *   out[1] = sum over cells of r_p^2 eta_c / (2/hx^2 + 2/hy^2), r_p = -D v
 *   out[2] = sum over velocity unknowns of f^2 / (-diag M)
 * The relative energy residual is sqrt((out[0] + out[1]) / out[2]).  p may be
 * NULL.  `out` is host memory; the call synchronises the context's stream.
 * The summation order is fixed, so repeated calls give identical bits.
 * STOKES_ERR_ARG if vx, vy or p does not start on a 16-byte boundary. */
int stokes_residual_energy_norm(stokes_ctx *ctx, const void *vx, const void *vy, const void *p, double out[3]);

/* Solve M v = f - G p with a geometric-multigrid V-cycle B (Sec. 3.2) as the
 * preconditioner of an outer iteration in the context's dtype: the residual
 * r = f - G p - M v, the energy residual E_v = sqrt(sum r^2/(-diag M) /
 * sum f^2/(-diag M)) and the update of v stay in the context's dtype, while
 * B (smoothing, restriction, prolongation) runs in params->inner_dtype from a
 * zero guess; the outer iteration is defect correction (v += B r) or flexible
 * CG (params->krylov).  Stops when E_v <= tol.  Improves (vx, vy) in place.
 * *final_rel_resid receives the last E_v and *cycles the number of V-cycles
 * (either may be NULL).  Returns STOKES_ERR_NOT_CONVERGED when max_cycles
 * is reached above tol, STOKES_ERR_DIVERGED on NaN/Inf or growth of E_v beyond
 * 1e6 times its first value.  The hierarchy is built on the first call after
 * stokes_set_viscosity (or after a change of levels, coarsest or inner_dtype).
 * The V-cycle is captured once as a CUDA graph (on context-owned work
 * buffers) and replayed on a context-owned stream ordered after the context's
 * stream.  Synchronises. */
int stokes_vcycle(stokes_ctx *ctx, void *vx, void *vy, const void *p, const stokes_mg_params *params,
                  double *final_rel_resid, int *cycles);

/* Parameters of the inexact Uzawa iteration (Sec. 3.1-3.2; solver
 * configuration of Sec. 6.2).
 * mg              the velocity step of every Uzawa cycle: mg.max_cycles (>= 1)
 *                 applications of the V-cycle, as flexible-CG iterations
 *                 (mg.krylov = 1, which stays stable where the V-cycle is not a
 *                 convergent splitting at high viscosity contrast) or as
 *                 defect-correction cycles (mg.krylov = 0, the paper's "one
 *                 multigrid iteration per Uzawa cycle" taken literally);
 *                 mg.tol is ignored.
 * omega_p         pressure relaxation (0.6 in Sec. 6.3): p <- p - omega_p eta_c D v,
 *                 with the cell viscosity as the approximate inverse Schur
 *                 complement and D the divergence; p is then shifted to zero mean.
 * cycles          maximum number of Uzawa cycles.
 * theta_interval, theta_stages   viscosity continuation (Sec. 6.2): cycle n uses
 *                 eta_theta = (1 - theta) eta_min + theta eta with
 *                 theta = min(n / theta_interval, theta_stages - 1) / (theta_stages - 1)
 *                 (25 and 5 in the paper); theta_interval = 0 turns it off.
 *                 eta_min is the smallest viscosity over the cells and the
 *                 interior nodes.  The context's viscosity is restored on return.
 * tol             stop once the relative energy residual (velocity and pressure
 *                 parts of Sec. 6.4, the caller's viscosity) is <= tol; 0 runs
 *                 every cycle.
 * lithostatic_init  1: start from the lithostatic pressure of f (p[0][i] = 0,
 *                 p[j][i] = p[j-1][i] - hy fy[j][i], zero mean), overwriting p;
 *                 0: start from the caller's p.
 * anderson_depth  Anderson acceleration of the Uzawa map over x = [v, p]
 *                 (Algorithm 1) with depth m = anderson_depth (0 <= m < 16; 0 off):
 *                 x_{k+1} = sum_i alpha_i F(x_i) over the last min(m, k) + 1
 *                 iterates, alpha minimising || sum_i alpha_i (F(x_i) - x_i) ||_2
 *                 (2-norm over every entry of vx, vy, p) subject to sum alpha = 1,
 *                 solved on the host from FP64 inner products with a relative
 *                 diagonal shift of 1e-14; the history restarts at every
 *                 continuation stage.  Needs 6 (m + 1) + 3 extra device fields. */
typedef struct {
    stokes_mg_params mg;
    double omega_p;
    int cycles;
    int theta_interval, theta_stages;
    double tol;
    int lithostatic_init;
    int anderson_depth;
} stokes_uzawa_params;

/* Solve the Stokes system M v + G p = f, D v = 0 (Eq. (6) and Eq. (4)) by the
 * inexact Uzawa iteration of `params`, improving (vx, vy, p) in place (device
 * buffers in the context's layout; p must hold an initial pressure unless
 * lithostatic_init).  history (host, may be NULL) receives the relative energy
 * residual after every cycle (params->cycles entries at most); *cycles the
 * number of cycles run and *final_rel_resid the last residual (either may be
 * NULL).  Returns STOKES_ERR_NOT_CONVERGED when tol > 0 was not reached,
 * STOKES_ERR_DIVERGED on NaN/Inf.  Synchronises after every cycle. */
int stokes_uzawa(stokes_ctx *ctx, void *vx, void *vy, void *p, const stokes_uzawa_params *params, double *history,
                 int *cycles, double *final_rel_resid);

/* Context options (stokes_set_option). */
typedef enum {
    STOKES_OPT_USE_TMA = 0,          /* 1 (default): the tile smoothers stage windows with TMA bulk
                                        tensor copies in a persistent kernel when the window fits;
                                        0: they read windows straight from global memory.  The
                                        results are identical either way. */
    STOKES_OPT_WAIT_LIMIT_CYCLES = 1, /* SM clock cycles a device-side wait for a staged window may
                                        take before the kernel gives up, records STOKES_ERR_TIMEOUT
                                        and exits (default 2e9, about one second; 0 = one try;
                                        negative = give up at once, which tests use to exercise the
                                        timeout path). */
    STOKES_OPT_PAIRED = 2            /* 1 (default): FP32 tile windows of 49 to 64 columns run the
                                        packed-pair kernel (two columns per thread, paired FP32
                                        instructions); 2: every FP32 window of at most 64 columns
                                        does; 0: never (one column per thread).  Needs
                                        STOKES_OPT_USE_TMA; the results are identical either way
                                        (up to the sign of exact zeros).  Other values:
                                        STOKES_ERR_ARG. */
} stokes_option;

int stokes_set_option(stokes_ctx *ctx, int option, long long value);

/* Synchronise the context's stream and report (then clear) any error a kernel
 * recorded on the device since the last check: STOKES_ERR_TIMEOUT if a
 * bounded wait gave up (the smoothing result is then unspecified).
 * stokes_residual_energy_norm and stokes_vcycle perform the same check. */
int stokes_synchronize(stokes_ctx *ctx);

/* Kernel classes counted and timed by the profiling hooks below. */
typedef enum {
    STOKES_K_RAS = 0,    /* RAS / blocked-Jacobi tile kernel (one launch per outer iteration or sweep) */
    STOKES_K_JACOBI = 1, /* global Jacobi pass kernels */
    STOKES_K_RBGS = 2,   /* red-black Gauss-Seidel colour kernels */
    STOKES_K_RHS = 3,    /* b = f - G p */
    STOKES_K_ENERGY = 4, /* energy-norm reduction kernels */
    STOKES_K_COPY = 5,   /* velocity / wall / viscosity copies and casts */
    STOKES_K_APPLY = 6,  /* operator apply */
    STOKES_K_MG = 7,     /* multigrid transfer, coarse-level and correction kernels */
    STOKES_K_COUNT = 8
} stokes_kernel_class;

/* Profiling hooks (tracing, not needed for computing).  The context always
 * counts the kernels it launches per class.  With timing enabled it also
 * brackets every launch group with a pair of CUDA events on the context's
 * stream.  stokes_profile_reset zeroes counts and times and sets the timing
 * flag (0/1).  stokes_profile_read synchronises the stream and returns, for
 * class `kind`, the number of kernel launches, the number of timed launch
 * groups and their summed device time in milliseconds (any output may be
 * NULL). */
int stokes_profile_reset(stokes_ctx *ctx, int enable_timing);
int stokes_profile_read(stokes_ctx *ctx, int kind, long long *kernels, long long *groups, double *total_ms);

/* Which tile kernel a RAS / blocked-Jacobi launch of this grid, tile and
 * overlap uses (Sec. 4.3: the window is the tile grown by overlap + 1), with
 * the given STOKES_OPT_USE_TMA (0/1) and STOKES_OPT_PAIRED (0/1/2) values: *kernel gets a
 * stokes_tile_kernel value, *threads the CTA size, *smem_bytes the dynamic
 * shared memory (outputs may be NULL).  Diagnostic only; reads the current
 * device's shared-memory limit.  STOKES_ERR_ARG on sizes < 1, overlap < 0, a
 * bad dtype or pair mode; STOKES_ERR_CUDA without a device. */
typedef enum {
    STOKES_TILE_TMA = 0,    /* persistent, TMA-staged window, one column per thread */
    STOKES_TILE_GLOBAL = 1, /* one CTA per tile, window read from global memory */
    STOKES_TILE_SHARED = 2, /* general kernel, every field of the window in shared memory */
    STOKES_TILE_PAIR = 3    /* persistent, TMA-staged, two columns per thread, paired FP32 instructions */
} stokes_tile_kernel;

int stokes_tile_kernel_plan(int nx, int ny, int ti, int tj, int overlap, int dtype, int use_tma, int pair_mode,
                            int *kernel, int *threads, size_t *smem_bytes);

/* Energy residual sums without allocating.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc, for instance
 * code that runs inside a framework's device-memory budget that forbids side
 * allocations, that hands every byte of the GPU to its own pools, or that
 * must not risk the device-wide synchronisation cudaMalloc and cudaFree can
 * cause.  Such callers cannot create a stokes_ctx (which allocates), so this
 * call takes everything as arguments and allocates nothing.
 *
 * It computes the three sums of stokes_residual_energy_norm for the grid
 * nx x ny on [0, lx] x [0, ly] in `dtype`: every field pointer is a device
 * buffer of (ny+1) rows x `pitch` elements in the layout described at the top
 * of this file (eta_n is the caller's own array, its boundary nodes are
 * ignored); p may be NULL (p = 0).  out_dev is a device pointer to 3 doubles
 * that receives the sums.  The work is enqueued on `cuda_stream` (NULL = the
 * legacy default stream) and the call returns without waiting.
 *
 * Scratch: the per-block partial sums live in a file-scope device array of
 * 608 x 3 doubles (14,592 bytes) that every GPU loading the library holds
 * until the process exits.  Each call overwrites all of it before reading it,
 * so nothing carries over between calls, but every call shares the one array:
 * calls whose work overlaps on the GPU (on different streams, or from
 * different host threads) race and return wrong sums.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  The
 * address is looked up again if the device's context was replaced since (after
 * cudaDeviceReset), so that call, too, must come before any stream capture.
 *
 * Limits: 2 <= nx, ny <= 46340, pitch >= nx + 1 and (ny + 1) * pitch < 2^31;
 * anything else returns STOKES_ERR_ARG, as do NULL inputs or a bad dtype.
 * The reduction writes one triple of partial sums per block: if the library's
 * energy reduction ran more than the array's 608 blocks, the call would
 * return STOKES_ERR_ARG (the library runs exactly 608).  CUDA failures return
 * STOKES_ERR_CUDA. */
int stokes_energy_norm_noalloc(int nx, int ny, double lx, double ly, int dtype, int pitch, const void *eta_c,
                               const void *eta_n, const void *fx, const void *fy, const void *p, const void *vx,
                               const void *vy, double *out_dev, void *cuda_stream);

/* ---- Batches: many independent problems of different sizes ---------------
 * A batch holds `count` instances, instance i an nx[i] x ny[i] grid on
 * [0, lx[i]] x [0, ly[i]], all in one dtype, and advances them together: each
 * step of a smoothing call, of the V-cycle and of the outer iteration is one
 * kernel launch over every instance taking part in it, and the V-cycle of the
 * whole batch is one CUDA graph.  Each instance follows exactly the schedule
 * of a context of its own with the same parameters, so its smoothing and
 * V-cycle results match that context's bit for bit (the outer iteration's
 * FP64 sums are accumulated in another fixed order, so a solve agrees to
 * rounding).
 *
 * Layout: every field of a batch is one device "slab" holding the instances
 * back to back; instance i occupies (ny[i]+1) rows x pitch_i elements starting
 * at element offset_i of the slab, in the single-context layout described at
 * the top of this file (stokes_batch_get_layout).  The caller owns the slabs
 * it passes (vx, vy, p, and the eta and f slabs it copies in).
 *
 * Smoothers: the Jacobi variants and RAS (STOKES_RBGS is not batched and
 * returns STOKES_ERR_ARG).  Every instance uses the same parameters, seed
 * and shifts. */
typedef struct stokes_batch stokes_batch; /* opaque, library-owned */

/* Create a batch of `count` >= 1 instances (host arrays nx, ny, lx, ly of
 * `count` entries; 2 <= nx, ny <= 65536; lx, ly > 0) computing in `dtype` on
 * `cuda_stream`.  Allocates the library's slabs. */
int stokes_batch_create(int count, const int *nx, const int *ny, const double *lx, const double *ly, int dtype,
                        void *cuda_stream, stokes_batch **out);

/* Instance `inst`: row pitch, offset of its first element in a slab, and its
 * extent ((ny+1) x pitch).  inst = -1: *alloc_elems receives the size of a
 * whole slab (elements), the others 0.  Outputs may be NULL. */
int stokes_batch_get_layout(const stokes_batch *b, int inst, int *pitch_elems, size_t *offset_elems,
                            size_t *alloc_elems);

/* Viscosity and body force of every instance from device slabs (copied);
 * the same rules as stokes_set_viscosity / stokes_set_rhs. */
int stokes_batch_set_viscosity(stokes_batch *b, const void *eta_c, const void *eta_n);
int stokes_batch_set_rhs(stokes_batch *b, const void *fx, const void *fy);

/* stokes_smooth for every instance: smooth M v = f - G p in place on the vx,
 * vy slabs (p slab may be NULL).  Asynchronous. */
int stokes_batch_smooth(stokes_batch *b, void *vx, void *vy, const void *p, const stokes_smooth_params *params);

/* Velocity energy sums of Sec. 6.4 for every instance, into the host array
 * out[2 * count]: out[2i] = sum r_v^2 / (-diag M), out[2i+1] = sum f^2 /
 * (-diag M), accumulated in FP64 in a fixed order.  Synchronises. */
int stokes_batch_residual_energy(stokes_batch *b, const void *vx, const void *vy, const void *p, double *out);

/* stokes_vcycle for every instance at once (the same parameters; the
 * coarsest level of every instance must have at most 1024 unknowns).  An
 * instance stops updating when it reaches tol, hits max_cycles or diverges.
 * Host arrays of `count` entries (each may be NULL) receive each instance's
 * final E_v, its number of V-cycles and its status (STOKES_OK,
 * STOKES_ERR_NOT_CONVERGED or STOKES_ERR_DIVERGED).  Returns STOKES_OK when
 * every instance converged, else STOKES_ERR_DIVERGED if any diverged, else
 * STOKES_ERR_NOT_CONVERGED.  The batched V-cycle is captured once as a CUDA
 * graph and replayed on a batch-owned stream.  Synchronises. */
int stokes_batch_solve(stokes_batch *b, void *vx, void *vy, const void *p, const stokes_mg_params *params,
                       double *final_rel_resid, int *cycles, int *status);

/* Batch options: the stokes_option values of stokes_set_option, with the
 * same meaning (STOKES_OPT_USE_TMA: 0 reads the windows of the batched tile
 * kernel straight from global memory, same results).  A bounded wait that
 * gives up is reported by the next stokes_batch_residual_energy or
 * stokes_batch_solve as STOKES_ERR_TIMEOUT. */
int stokes_batch_set_option(stokes_batch *b, int option, long long value);

/* Number of kernels the batch has launched so far (graph replays count
 * every kernel node). */
int stokes_batch_kernels(const stokes_batch *b, long long *kernels);

/* Release every library-owned buffer of the batch.  NULL is accepted. */
int stokes_batch_destroy(stokes_batch *b);

/* ---- Slab decomposition: RAS as a domain decomposition ---------------------
 * RAS-Jacobi (Sec. 4.3, Algorithm 2) is a domain decomposition: each tile
 * solves its local problem on an overlapping subdomain and writes only the
 * unknowns it owns.  A slab set splits the grid into `nslabs` horizontal
 * slabs, the layout of a multi-GPU run with one slab per GPU: slab s owns the
 * cell rows [r0, r1) of a balanced split and keeps its own copy of the
 * viscosity, the right-hand side and the velocity on the rows [R0, R1) =
 * [r0 - H, r1 + H) clipped to the grid, H = tile_j + overlap + 1.  Each outer
 * iteration runs the tile kernel on every slab's storage (the global shifted
 * tiling of Algorithm 2, so every tile that meets a slab's own rows is
 * computed there exactly as on the whole grid) and then copies to every slab
 * the rows it stores but does not own from the neighbour that owns them
 * (one device-to-device copy per field and side).  The result equals
 * stokes_smooth's with the same parameters, bit for bit.  All slabs live on
 * the device and stream of the set; every slab must own at least H + 1 rows.
 * Layouts are those of a single context (stokes_get_layout of a context of
 * the same nx, ny, dtype). */
typedef struct stokes_slabs stokes_slabs; /* opaque, library-owned */

/* Own rows [out[0], out[1]) and stored rows [out[2], out[3]) of slab `slab`
 * of an ny-row grid split into nslabs slabs, for tiles of tile_j rows and
 * `overlap`; a host computation (no device).  STOKES_ERR_ARG if a slab would
 * own fewer than tile_j + overlap + 2 rows. */
int stokes_slab_plan(int ny, int nslabs, int tile_j, int overlap, int slab, int out[4]);

/* Create a set of nslabs (1 <= nslabs <= ny/2) slabs of an nx x ny grid on
 * [0, lx] x [0, ly] in `dtype` on `cuda_stream`; the same limits as
 * stokes_create.  Allocates the global copies; the slab storage is allocated
 * by the first smoothing (and again when tile_j + overlap changes). */
int stokes_slabs_create(int nx, int ny, double lx, double ly, int dtype, int nslabs, void *cuda_stream,
                        stokes_slabs **out);

/* Viscosity and body force of the whole grid (device buffers in the
 * single-context layout, copied), as stokes_set_viscosity / stokes_set_rhs. */
int stokes_slabs_set_viscosity(stokes_slabs *s, const void *eta_c, const void *eta_n);
int stokes_slabs_set_rhs(stokes_slabs *s, const void *fx, const void *fy);

/* RAS-Jacobi smoothing of the whole grid's (vx, vy) in place (p may be NULL)
 * through the slabs: `params` as for stokes_smooth with variant STOKES_RAS
 * (anything else is STOKES_ERR_ARG).  Scatters (vx, vy) and p into the
 * slabs, runs the outer iterations with their halo exchanges, gathers the
 * own rows back and synchronises the stream (STOKES_ERR_TIMEOUT if a bounded
 * wait of the tile kernel gave up).  STOKES_ERR_STATE before the viscosity
 * and the right-hand side are set. */
int stokes_slabs_smooth(stokes_slabs *s, void *vx, void *vy, const void *p, const stokes_smooth_params *params);

/* Halo copies made so far and their bytes. */
int stokes_slabs_exchanges(const stokes_slabs *s, long long *copies, long long *bytes);

/* Release the set.  NULL returns STOKES_ERR_ARG. */
int stokes_slabs_destroy(stokes_slabs *s);

/* ---- 3D: the staggered operator in three dimensions -------------------------
 * The paper develops the method in 2D and names the 3D extension (space-time
 * "4D" blocking) as future work (Sec. 9).  A 3D context carries the same
 * operator, readings and smoothers over to an nx x ny x nz grid on
 * [0, lx] x [0, ly] x [0, lz]:
 *   vx[k][j][i] at (i hx, (j+1/2) hy, (k+1/2) hz),  k < nz, j < ny, i <= nx
 *   vy[k][j][i] at ((i+1/2) hx, j hy, (k+1/2) hz),  k < nz, j <= ny, i < nx
 *   vz[k][j][i] at ((i+1/2) hx, (j+1/2) hy, k hz),  k <= nz, j < ny, i < nx
 *   p, eta_c at cell centres (k < nz, j < ny, i < nx)
 *   eta_xy at x-y edges (i hx, j hy, (k+1/2) hz), the viscosity of sigma'_xy
 *   eta_xz at x-z edges (i hx, (j+1/2) hy, k hz), of sigma'_xz
 *   eta_yz at y-z edges ((i+1/2) hx, j hy, k hz), of sigma'_yz
 * sigma'_ii = 2 eta_c dv_i/dx_i at the cells, sigma'_ij = eta_ij (dv_i/dx_j +
 * dv_j/dx_i) at the edges, zero on an edge in a wall it is tangential to (free
 * slip); the unknowns are the interior faces of each component.  Every field
 * buffer is one array of (nz+1) planes x (ny+1) rows x pitch elements of the
 * context's dtype, entry (k, j, i) at (k (ny+1) + j) pitch + i, starting on a
 * 16-byte boundary (stokes3d_get_layout gives pitch and size).  Ownership,
 * streams and errors as for the 2D context. */
typedef struct stokes3d_ctx stokes3d_ctx; /* opaque, library-owned */

/* Smoothing parameters in 3D: variant STOKES_JACOBI_FUSED or STOKES_RAS;
 * RAS tiles of tile_i x tile_j x tile_k cells (all >= 1) cut at s + m T in
 * each direction, `k` local sweeps on the tile grown by `overlap`; shifts as
 * in 2D with three values per outer iteration (SplitMix64 draws 3t, 3t+1,
 * 3t+2 of `seed` taken mod the tile sizes, or the list shifts[3t .. 3t+2]). */
typedef struct {
    int variant;
    int sweeps;
    int tile_i, tile_j, tile_k;
    int k;
    int overlap;
    double omega;
    uint64_t seed;
    int shift_mode;
    const int32_t *shifts;
} stokes3d_smooth_params;

/* Create a 3D context: 2 <= nx, ny, nz <= 4096, lengths > 0, dtype
 * STOKES_F32 or STOKES_F64, work on `cuda_stream`.  Allocates its buffers. */
int stokes3d_create(int nx, int ny, int nz, double lx, double ly, double lz, int dtype, void *cuda_stream,
                    stokes3d_ctx **out);

/* Row pitch (elements), rows per plane (ny + 1) and elements of one field buffer. */
int stokes3d_get_layout(const stokes3d_ctx *ctx, int *pitch_elems, int *plane_rows, size_t *alloc_elems);

/* Viscosity at cells and edges (device buffers, copied; the edges in walls
 * they are tangential to are ignored). */
int stokes3d_set_viscosity(stokes3d_ctx *ctx, const void *eta_c, const void *eta_xy, const void *eta_xz,
                           const void *eta_yz);

/* Body force (fx like vx, fy like vy, fz like vz; copied). */
int stokes3d_set_rhs(stokes3d_ctx *ctx, const void *fx, const void *fy, const void *fz);

/* out = M v + G p at the unknowns (p may be NULL), zero elsewhere in each
 * field's extent.  STOKES_ERR_STATE before the viscosity is set. */
int stokes3d_apply_operator(stokes3d_ctx *ctx, const void *vx, const void *vy, const void *vz, const void *p,
                            void *out_x, void *out_y, void *out_z);

/* Smooth M v = f - G p in place on (vx, vy, vz) (p may be NULL).  Fused
 * Jacobi, or RAS-Jacobi on 3D tiles (Algorithm 2 on boxes of tile_i x tile_j
 * x tile_k cells).  A window (the tile grown by overlap + 1 cells on every
 * side) 16 to 32 cells wide in x with at most 8 levels in z and 16 rows in y
 * (FP32; also 12 levels with at most 12 rows) or 8 levels and 8 rows (FP64)
 * runs with the velocity in registers and the y neighbours in shared memory;
 * any other window must fit shared memory whole (10 words per window cell):
 * STOKES_ERR_ARG when it does not.  Both give the same values bit for bit. */
int stokes3d_smooth(stokes3d_ctx *ctx, void *vx, void *vy, void *vz, const void *p,
                    const stokes3d_smooth_params *params);

/* The three energy sums of stokes_residual_energy_norm in 3D: sum r_v^2 /
 * (-diag M), sum (D v)^2 eta_c / (2/hx^2 + 2/hy^2 + 2/hz^2), sum f^2 /
 * (-diag M), accumulated in FP64 in a fixed order; synchronises. */
int stokes3d_residual_energy_norm(stokes3d_ctx *ctx, const void *vx, const void *vy, const void *vz, const void *p,
                                  double out[3]);

/* Kernels launched by the context so far. */
int stokes3d_kernels(const stokes3d_ctx *ctx, long long *kernels);

/* Release the context.  NULL is accepted. */
int stokes3d_destroy(stokes3d_ctx *ctx);

/* Release every library-owned buffer of the context.  NULL is accepted. */
int stokes_destroy(stokes_ctx *ctx);

/* Static text for a stokes_status value. */
const char *stokes_strerror(int status);

/* Text of the last CUDA error this thread's calls met ("" if none). */
const char *stokes_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* STOKES_H */
