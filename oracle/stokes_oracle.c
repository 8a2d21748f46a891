/*
 * stokes_oracle.c -- plain, slow, FP64 CPU statement of the staggered-grid
 * variable-viscosity Stokes velocity operator and of every smoother, norm and
 * multigrid step that the CUDA library computes.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path loads this file: only
 * the tests, the smoke check and the CPU-baseline leg of the benchmark may.  It
 * shares no code, header, table or helper with the CUDA library.
 *
 * Compile with -O2 -ffp-contract=off so that every product and sum is rounded
 * exactly where it is written.
 *
 * Sources (arXiv 2509.19061):
 *   Eq. (1)-(4)   Cauchy form of the 2D Stokes equations; sigma' = eta (dv_i/dx_j + dv_j/dx_i)
 *   Sec. 2.1      fully staggered grid: vx, vy on faces, p at centres, eta at
 *                 nodes (eta_B) and centres (eta_P), rho with vy (Fig. 1 caption)
 *   Eq. (6)       M v + G p = f  (the velocity subsystem)
 *   Sec. 5        the five smoothers (RBGS, Jacobi, fused, blocked fused, RAS)
 *   Sec. 4.3 / Algorithm 2   RAS-type temporal blocking
 *   Sec. 6.3      under-relaxation omega_u
 *   Sec. 6.4      energy residual norm
 *   Sec. 3.2 / 6.2  geometric multigrid V-cycle used for the velocity solve
 *
 * Natural (unpadded, row-major, y-major) layouts used by every function here:
 *   vx, fx, bx : ny     x (nx+1)   vx[j][i] at (i*hx, (j+1/2)*hy)
 *   vy, fy, by : (ny+1) x nx       vy[j][i] at ((i+1/2)*hx, j*hy)
 *   p, eta_c   : ny     x nx       cell centres ((i+1/2)*hx, (j+1/2)*hy)
 *   eta_n      : (ny+1) x (nx+1)   nodes (i*hx, j*hy)
 * Unknowns: vx with 1 <= i <= nx-1, vy with 1 <= j <= ny-1.  The wall entries
 * vx[.][0], vx[.][nx], vy[0][.], vy[ny][.] are Dirichlet data (zero for the
 * no-penetration walls of Sec. 6.1) and are never written.
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *  - the shear stress is zero on boundary nodes (free slip, Sec. 6.1);
 *  - Jacobi: v <- v + omega (b - M v) / diag(M), all from the old v; plain,
 *    fused and blocked fused Jacobi are this one map (Sec. 5 (ii)-(iv));
 *  - RBGS colour = parity of (i+j) in each array's own index, red = even,
 *    order vx-red, vx-black, vy-red, vy-black, same damping omega;
 *  - RAS: tiles start at s + m*T (clipped), a tile owns the unknowns of its
 *    cells (a cell owns its low-x vx face and its low-y vy face), local problem
 *    = unknowns of the tile grown by `overlap` cells, everything else frozen at
 *    the snapshot taken at the start of the outer iteration; the last outer
 *    iteration runs the remaining N - (N_outer-1) k sweeps.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* grid description                                                         */
/* ------------------------------------------------------------------------ */
typedef struct {
    int nx, ny;
    double hx, hy;
    const double *eta_c; /* ny x nx */
    const double *eta_n; /* (ny+1) x (nx+1) */
} grid_t;

static grid_t mkgrid(int nx, int ny, double hx, double hy, const double *eta_c, const double *eta_n)
{
    grid_t g;
    g.nx = nx; g.ny = ny; g.hx = hx; g.hy = hy; g.eta_c = eta_c; g.eta_n = eta_n;
    return g;
}

/* element access in the natural layouts */
#define VX(a, j, i) (a)[(size_t)(j) * (size_t)(g->nx + 1) + (size_t)(i)]
#define VY(a, j, i) (a)[(size_t)(j) * (size_t)(g->nx) + (size_t)(i)]
#define CC(a, j, i) (a)[(size_t)(j) * (size_t)(g->nx) + (size_t)(i)]
#define ND(a, j, i) (a)[(size_t)(j) * (size_t)(g->nx + 1) + (size_t)(i)]

static size_t nvx(const grid_t *g) { return (size_t)g->ny * (size_t)(g->nx + 1); }
static size_t nvy(const grid_t *g) { return (size_t)(g->ny + 1) * (size_t)g->nx; }

static int is_vx_unknown(const grid_t *g, int j, int i) { return j >= 0 && j < g->ny && i >= 1 && i <= g->nx - 1; }
static int is_vy_unknown(const grid_t *g, int j, int i) { return i >= 0 && i < g->nx && j >= 1 && j <= g->ny - 1; }

/* ------------------------------------------------------------------------ */
/* deviatoric stresses, Eq. (3): sigma'_ij = eta (dv_i/dx_j + dv_j/dx_i)    */
/* ------------------------------------------------------------------------ */
/* sigma'_xx at cell centre (i, j): 2 eta_c dvx/dx */
static double sxx(const grid_t *g, const double *vx, int j, int i)
{
    return 2.0 * CC(g->eta_c, j, i) * (VX(vx, j, i + 1) - VX(vx, j, i)) / g->hx;
}

/* sigma'_yy at cell centre (i, j): 2 eta_c dvy/dy */
static double syy(const grid_t *g, const double *vy, int j, int i)
{
    return 2.0 * CC(g->eta_c, j, i) * (VY(vy, j + 1, i) - VY(vy, j, i)) / g->hy;
}

/* sigma'_xy at node (i, j): eta_n (dvx/dy + dvy/dx); zero on boundary nodes (free slip) */
static double sxy(const grid_t *g, const double *vx, const double *vy, int j, int i)
{
    if (i <= 0 || i >= g->nx || j <= 0 || j >= g->ny) return 0.0;
    double dvx_dy = (VX(vx, j, i) - VX(vx, j - 1, i)) / g->hy;
    double dvy_dx = (VY(vy, j, i) - VY(vy, j, i - 1)) / g->hx;
    return ND(g->eta_n, j, i) * (dvx_dy + dvy_dx);
}

/* ------------------------------------------------------------------------ */
/* momentum operator M, Eq. (1)-(2) left-hand side without the pressure     */
/* ------------------------------------------------------------------------ */
/* (M v)_x at vx unknown (i, j): d sigma'_xx/dx + d sigma'_xy/dy */
static double mx_at(const grid_t *g, const double *vx, const double *vy, int j, int i)
{
    double dsxx_dx = (sxx(g, vx, j, i) - sxx(g, vx, j, i - 1)) / g->hx;
    double dsxy_dy = (sxy(g, vx, vy, j + 1, i) - sxy(g, vx, vy, j, i)) / g->hy;
    return dsxx_dx + dsxy_dy;
}

/* (M v)_y at vy unknown (i, j): d sigma'_yx/dx + d sigma'_yy/dy */
static double my_at(const grid_t *g, const double *vx, const double *vy, int j, int i)
{
    double dsyx_dx = (sxy(g, vx, vy, j, i + 1) - sxy(g, vx, vy, j, i)) / g->hx;
    double dsyy_dy = (syy(g, vy, j, i) - syy(g, vy, j - 1, i)) / g->hy;
    return dsyx_dx + dsyy_dy;
}

/* diagonal entries of M: the coefficient of vx[j][i] in (M v)_x[j][i] (and
 * likewise for vy).  Boundary nodes carry no shear stress, so their eta_n
 * does not enter. */
static double eta_n_interior(const grid_t *g, int j, int i)
{
    if (i <= 0 || i >= g->nx || j <= 0 || j >= g->ny) return 0.0;
    return ND(g->eta_n, j, i);
}

static double dmx_at(const grid_t *g, int j, int i)
{
    double hx2 = g->hx * g->hx, hy2 = g->hy * g->hy;
    return -2.0 * (CC(g->eta_c, j, i) + CC(g->eta_c, j, i - 1)) / hx2
           - (eta_n_interior(g, j + 1, i) + eta_n_interior(g, j, i)) / hy2;
}

static double dmy_at(const grid_t *g, int j, int i)
{
    double hx2 = g->hx * g->hx, hy2 = g->hy * g->hy;
    return -2.0 * (CC(g->eta_c, j, i) + CC(g->eta_c, j - 1, i)) / hy2
           - (eta_n_interior(g, j, i + 1) + eta_n_interior(g, j, i)) / hx2;
}

/* ------------------------------------------------------------------------ */
/* exported: operator, gradient, divergence, diagonal, right-hand side      */
/* ------------------------------------------------------------------------ */

/* out = M v at every unknown; wall entries of out are set to zero. */
void ora_apply_M(int nx, int ny, double hx, double hy, const double *eta_c, const double *eta_n,
                 const double *vx, const double *vy, double *out_x, double *out_y)
{
    grid_t G = mkgrid(nx, ny, hx, hy, eta_c, eta_n), *g = &G;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i <= nx; ++i)
            VX(out_x, j, i) = is_vx_unknown(g, j, i) ? mx_at(g, vx, vy, j, i) : 0.0;
    for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i)
            VY(out_y, j, i) = is_vy_unknown(g, j, i) ? my_at(g, vx, vy, j, i) : 0.0;
}

/* G p with the sign of Eq. (1): the pressure term is -dp/dx, so (G p)_x = -dp/dx. */
void ora_apply_G(int nx, int ny, double hx, double hy, const double *p, double *gx, double *gy)
{
    grid_t G = mkgrid(nx, ny, hx, hy, NULL, NULL), *g = &G;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i <= nx; ++i)
            VX(gx, j, i) = is_vx_unknown(g, j, i) ? -(CC(p, j, i) - CC(p, j, i - 1)) / hx : 0.0;
    for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i)
            VY(gy, j, i) = is_vy_unknown(g, j, i) ? -(CC(p, j, i) - CC(p, j - 1, i)) / hy : 0.0;
}

/* D v = dvx/dx + dvy/dy at cell centres, Eq. (4). */
void ora_apply_D(int nx, int ny, double hx, double hy, const double *vx, const double *vy, double *dv)
{
    grid_t G = mkgrid(nx, ny, hx, hy, NULL, NULL), *g = &G;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
            CC(dv, j, i) = (VX(vx, j, i + 1) - VX(vx, j, i)) / hx + (VY(vy, j + 1, i) - VY(vy, j, i)) / hy;
}

/* diag(M) at every unknown (zero at walls). */
void ora_diag_M(int nx, int ny, double hx, double hy, const double *eta_c, const double *eta_n,
                double *dx, double *dy)
{
    grid_t G = mkgrid(nx, ny, hx, hy, eta_c, eta_n), *g = &G;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i <= nx; ++i)
            VX(dx, j, i) = is_vx_unknown(g, j, i) ? dmx_at(g, j, i) : 0.0;
    for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i)
            VY(dy, j, i) = is_vy_unknown(g, j, i) ? dmy_at(g, j, i) : 0.0;
}

/* b = f - G p (Eq. (7)'s right-hand side for fixed p); p may be NULL (p = 0).
 * Wall entries of b are zero. */
void ora_rhs(int nx, int ny, double hx, double hy, const double *fx, const double *fy, const double *p,
             double *bx, double *by)
{
    grid_t G = mkgrid(nx, ny, hx, hy, NULL, NULL), *g = &G;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i <= nx; ++i) {
            if (!is_vx_unknown(g, j, i)) { VX(bx, j, i) = 0.0; continue; }
            double gp = p ? -(CC(p, j, i) - CC(p, j, i - 1)) / hx : 0.0;
            VX(bx, j, i) = VX(fx, j, i) - gp;
        }
    for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) {
            if (!is_vy_unknown(g, j, i)) { VY(by, j, i) = 0.0; continue; }
            double gp = p ? -(CC(p, j, i) - CC(p, j - 1, i)) / hy : 0.0;
            VY(by, j, i) = VY(fy, j, i) - gp;
        }
}

/* ------------------------------------------------------------------------ */
/* damped point-Jacobi update (Sec. 5 (ii)-(iv), omega_u of Sec. 6.3)       */
/* ------------------------------------------------------------------------ */
static double jacobi_x(const grid_t *g, const double *vx, const double *vy, const double *bx, double omega,
                       int j, int i)
{
    return VX(vx, j, i) + omega * (VX(bx, j, i) - mx_at(g, vx, vy, j, i)) / dmx_at(g, j, i);
}

static double jacobi_y(const grid_t *g, const double *vx, const double *vy, const double *by, double omega,
                       int j, int i)
{
    return VY(vy, j, i) + omega * (VY(by, j, i) - my_at(g, vx, vy, j, i)) / dmy_at(g, j, i);
}

/* `sweeps` global Jacobi sweeps, in place.  Every update of a sweep is taken
 * from the values of the previous sweep. */
void ora_jacobi(int nx, int ny, double hx, double hy, const double *eta_c, const double *eta_n,
                const double *bx, const double *by, double omega, int sweeps, double *vx, double *vy)
{
    grid_t G = mkgrid(nx, ny, hx, hy, eta_c, eta_n), *g = &G;
    double *nxv = malloc(nvx(g) * sizeof(double));
    double *nyv = malloc(nvy(g) * sizeof(double));
    for (int s = 0; s < sweeps; ++s) {
        memcpy(nxv, vx, nvx(g) * sizeof(double));
        memcpy(nyv, vy, nvy(g) * sizeof(double));
        for (int j = 0; j < ny; ++j)
            for (int i = 1; i <= nx - 1; ++i) VX(nxv, j, i) = jacobi_x(g, vx, vy, bx, omega, j, i);
        for (int j = 1; j <= ny - 1; ++j)
            for (int i = 0; i < nx; ++i) VY(nyv, j, i) = jacobi_y(g, vx, vy, by, omega, j, i);
        memcpy(vx, nxv, nvx(g) * sizeof(double));
        memcpy(vy, nyv, nvy(g) * sizeof(double));
    }
    free(nxv);
    free(nyv);
}

/* ------------------------------------------------------------------------ */
/* Red-Black Gauss-Seidel (Sec. 5 (i))                                      */
/* ------------------------------------------------------------------------ */
/* One half-sweep updates every unknown of one component and one colour from
 * the current values (same-colour unknowns of one component are not coupled). */
void ora_rbgs(int nx, int ny, double hx, double hy, const double *eta_c, const double *eta_n,
              const double *bx, const double *by, double omega, int sweeps, double *vx, double *vy)
{
    grid_t G = mkgrid(nx, ny, hx, hy, eta_c, eta_n), *g = &G;
    double *nxv = malloc(nvx(g) * sizeof(double));
    double *nyv = malloc(nvy(g) * sizeof(double));
    for (int s = 0; s < sweeps; ++s) {
        for (int colour = 0; colour < 2; ++colour) {
            memcpy(nxv, vx, nvx(g) * sizeof(double));
            for (int j = 0; j < ny; ++j)
                for (int i = 1; i <= nx - 1; ++i)
                    if (((i + j) & 1) == colour) VX(nxv, j, i) = jacobi_x(g, vx, vy, bx, omega, j, i);
            memcpy(vx, nxv, nvx(g) * sizeof(double));
        }
        for (int colour = 0; colour < 2; ++colour) {
            memcpy(nyv, vy, nvy(g) * sizeof(double));
            for (int j = 1; j <= ny - 1; ++j)
                for (int i = 0; i < nx; ++i)
                    if (((i + j) & 1) == colour) VY(nyv, j, i) = jacobi_y(g, vx, vy, by, omega, j, i);
            memcpy(vy, nyv, nvy(g) * sizeof(double));
        }
    }
    free(nxv);
    free(nyv);
}

/* ------------------------------------------------------------------------ */
/* counter-based SplitMix64 (Steele, Lea & Flood, OOPSLA 2014)              */
/* ------------------------------------------------------------------------ */
/* The c-th output (c = 0, 1, ...) of a SplitMix64 generator whose state
 * starts at `seed`: the state advances by the golden gamma before each
 * output, and the output is the state passed through the mix64 finaliser. */
uint64_t ora_splitmix64(uint64_t seed, uint64_t c)
{
    uint64_t z = seed + (c + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* ------------------------------------------------------------------------ */
/* RAS-type temporal blocking with Jacobi as the local solver (Alg. 2)      */
/* ------------------------------------------------------------------------ */
/* Tile shifts of outer iteration t (0-based).
 * mode 0: no shift; mode 1: SplitMix64 draws 2t and 2t+1 of `seed` taken mod
 * the tile size; mode 2: explicit list shifts[2t], shifts[2t+1]. */
static void ras_shift(int mode, uint64_t seed, const int *shifts, int t, int ti, int tj, int *si, int *sj)
{
    if (mode == 1) {
        *si = (int)(ora_splitmix64(seed, 2u * (uint64_t)t) % (uint64_t)ti);
        *sj = (int)(ora_splitmix64(seed, 2u * (uint64_t)t + 1u) % (uint64_t)tj);
    } else if (mode == 2) {
        *si = shifts[2 * t];
        *sj = shifts[2 * t + 1];
    } else {
        *si = 0;
        *sj = 0;
    }
}

/* Cut [0, n) at s + m*T (m integer).  Writes the cut points (including 0 and
 * n) to cuts and returns the number of intervals. */
static int tile_cuts(int n, int T, int s, int *cuts)
{
    int m = 0;
    cuts[m++] = 0;
    for (int c = s; c < n; c += T)
        if (c > 0) cuts[m++] = c;
    cuts[m++] = n;
    return m - 1;
}

/* One RAS outer iteration with `ksweeps` local sweeps: reads the snapshot
 * (sx, sy) and writes the owned unknowns of every tile into (ox, oy).
 * `work` arrays are full-size scratch copies of the snapshot that are
 * restored after each tile. */
static int ras_outer(const grid_t *g, const double *bx, const double *by, double omega, int ti, int tj,
                     int ksweeps, int overlap, int si, int sj, uint64_t order_seed, const double *sx,
                     const double *sy, double *ox, double *oy, int *count_x, int *count_y)
{
    int nx = g->nx, ny = g->ny;
    int *cx = malloc((size_t)(nx / ti + 3) * sizeof(int));
    int *cy = malloc((size_t)(ny / tj + 3) * sizeof(int));
    int ntx = tile_cuts(nx, ti, si, cx);
    int nty = tile_cuts(ny, tj, sj, cy);
    int ntiles = ntx * nty;
    int *order = malloc((size_t)ntiles * sizeof(int));
    for (int t = 0; t < ntiles; ++t) order[t] = t;
    if (order_seed) /* Fisher-Yates shuffle of the tile processing order */
        for (int t = ntiles - 1; t > 0; --t) {
            int r = (int)(ora_splitmix64(order_seed, (uint64_t)t) % (uint64_t)(t + 1));
            int tmp = order[t]; order[t] = order[r]; order[r] = tmp;
        }

    /* The tiles are independent (each reads the snapshot and writes only the
     * unknowns it owns), so an OpenMP build runs them in parallel, each
     * thread with its own work copies; the plain build runs them in order. */
#ifdef _OPENMP
#pragma omp parallel
#endif
    {
        double *wx = malloc(nvx(g) * sizeof(double)), *wy = malloc(nvy(g) * sizeof(double));
        double *tx = malloc(nvx(g) * sizeof(double)), *ty = malloc(nvy(g) * sizeof(double));
        memcpy(wx, sx, nvx(g) * sizeof(double));
        memcpy(wy, sy, nvy(g) * sizeof(double));
        memcpy(tx, sx, nvx(g) * sizeof(double));
        memcpy(ty, sy, nvy(g) * sizeof(double));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int q = 0; q < ntiles; ++q) {
            int tid = order[q];
            int bxi = tid % ntx, byj = tid / ntx;
            int x0 = cx[bxi], x1 = cx[bxi + 1], y0 = cy[byj], y1 = cy[byj + 1];
            /* local problem: cells of the tile grown by `overlap`, clipped */
            int lx0 = x0 - overlap < 0 ? 0 : x0 - overlap;
            int lx1 = x1 + overlap > nx ? nx : x1 + overlap;
            int ly0 = y0 - overlap < 0 ? 0 : y0 - overlap;
            int ly1 = y1 + overlap > ny ? ny : y1 + overlap;
            /* k local Jacobi sweeps; w holds the local iterate, everything
             * outside the local problem stays at the snapshot (Dirichlet) */
            for (int s = 0; s < ksweeps; ++s) {
                for (int j = ly0; j < ly1; ++j)
                    for (int i = lx0; i < lx1; ++i) {
                        if (is_vx_unknown(g, j, i)) VX(tx, j, i) = jacobi_x(g, wx, wy, bx, omega, j, i);
                        if (is_vy_unknown(g, j, i)) VY(ty, j, i) = jacobi_y(g, wx, wy, by, omega, j, i);
                    }
                for (int j = ly0; j < ly1; ++j)
                    for (int i = lx0; i < lx1; ++i) {
                        if (is_vx_unknown(g, j, i)) VX(wx, j, i) = VX(tx, j, i);
                        if (is_vy_unknown(g, j, i)) VY(wy, j, i) = VY(ty, j, i);
                    }
            }
            /* keep only the unknowns owned by the tile's own cells */
            for (int j = y0; j < y1; ++j)
                for (int i = x0; i < x1; ++i) {
                    if (is_vx_unknown(g, j, i)) {
                        VX(ox, j, i) = VX(wx, j, i);
                        if (count_x) VX(count_x, j, i) += 1;
                    }
                    if (is_vy_unknown(g, j, i)) {
                        VY(oy, j, i) = VY(wy, j, i);
                        if (count_y) VY(count_y, j, i) += 1;
                    }
                }
            /* restore the snapshot in the local region */
            for (int j = ly0; j < ly1; ++j)
                for (int i = lx0; i < lx1; ++i) {
                    if (is_vx_unknown(g, j, i)) VX(wx, j, i) = VX(tx, j, i) = VX(sx, j, i);
                    if (is_vy_unknown(g, j, i)) VY(wy, j, i) = VY(ty, j, i) = VY(sy, j, i);
                }
        }
        free(wx); free(wy); free(tx); free(ty);
    }
    free(order); free(cx); free(cy);
    return 0;
}

/* RAS-Jacobi smoother: `sweeps` = N_max of Alg. 2, `k` = T_inner.
 * Runs ceil(N/k) outer iterations; the last one runs N - (N_outer-1) k local
 * sweeps.  `order_seed` != 0 shuffles the order in which tiles are processed
 * (the result must not depend on it).  `owner_count` (optional, natural vx
 * layout followed by natural vy layout) receives, for the LAST outer
 * iteration, how many tiles wrote each unknown.  Returns 0, or -1 on bad
 * arguments. */
int ora_ras(int nx, int ny, double hx, double hy, const double *eta_c, const double *eta_n,
            const double *bx, const double *by, double omega, int sweeps, int ti, int tj, int k,
            int overlap, int shift_mode, uint64_t seed, const int *shifts, uint64_t order_seed,
            double *vx, double *vy, int *owner_count)
{
    if (nx < 1 || ny < 1 || ti < 1 || tj < 1 || k < 1 || overlap < 0 || sweeps < 0) return -1;
    grid_t G = mkgrid(nx, ny, hx, hy, eta_c, eta_n), *g = &G;
    int n_outer = (sweeps + k - 1) / k;
    double *sx = malloc(nvx(g) * sizeof(double)), *sy = malloc(nvy(g) * sizeof(double));
    for (int t = 0; t < n_outer; ++t) {
        int kk = (t == n_outer - 1) ? sweeps - (n_outer - 1) * k : k;
        int si, sj;
        ras_shift(shift_mode, seed, shifts, t, ti, tj, &si, &sj);
        memcpy(sx, vx, nvx(g) * sizeof(double));
        memcpy(sy, vy, nvy(g) * sizeof(double));
        int *cxc = NULL, *cyc = NULL;
        if (owner_count && t == n_outer - 1) {
            memset(owner_count, 0, (nvx(g) + nvy(g)) * sizeof(int));
            cxc = owner_count;
            cyc = owner_count + nvx(g);
        }
        ras_outer(g, bx, by, omega, ti, tj, kk, overlap, si, sj, order_seed, sx, sy, vx, vy, cxc, cyc);
    }
    free(sx);
    free(sy);
    return 0;
}

/* The (s_i, s_j) shift that ora_ras draws for outer iteration t. */
void ora_ras_shift(int shift_mode, uint64_t seed, int t, int ti, int tj, int *out)
{
    ras_shift(shift_mode, seed, NULL, t, ti, tj, &out[0], &out[1]);
}

/* ------------------------------------------------------------------------ */
/* energy residual norm (Sec. 6.4)                                          */
/* ------------------------------------------------------------------------ */
/* out[0] = sum over velocity unknowns of r_v^2 / (-diag M), r_v = f - G p - M v
 * out[1] = sum over cells of r_p^2 * eta_c / (2/hx^2 + 2/hy^2), r_p = -D v
 * out[2] = sum over velocity unknowns of f^2 / (-diag M)
 * The relative energy residual is sqrt((out[0] + out[1]) / out[2]). */
void ora_energy(int nx, int ny, double hx, double hy, const double *eta_c, const double *eta_n,
                const double *fx, const double *fy, const double *p, const double *vx, const double *vy,
                double *out)
{
    grid_t G = mkgrid(nx, ny, hx, hy, eta_c, eta_n), *g = &G;
    double *bx = malloc(nvx(g) * sizeof(double)), *by = malloc(nvy(g) * sizeof(double));
    ora_rhs(nx, ny, hx, hy, fx, fy, p, bx, by);
    double rv = 0.0, rp = 0.0, ff = 0.0;
    for (int j = 0; j < ny; ++j)
        for (int i = 1; i <= nx - 1; ++i) {
            double w = -dmx_at(g, j, i);
            double r = VX(bx, j, i) - mx_at(g, vx, vy, j, i);
            rv += r * r / w;
            ff += VX(fx, j, i) * VX(fx, j, i) / w;
        }
    for (int j = 1; j <= ny - 1; ++j)
        for (int i = 0; i < nx; ++i) {
            double w = -dmy_at(g, j, i);
            double r = VY(by, j, i) - my_at(g, vx, vy, j, i);
            rv += r * r / w;
            ff += VY(fy, j, i) * VY(fy, j, i) / w;
        }
    double lap = 2.0 / (hx * hx) + 2.0 / (hy * hy);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double r = -((VX(vx, j, i + 1) - VX(vx, j, i)) / hx + (VY(vy, j + 1, i) - VY(vy, j, i)) / hy);
            rp += r * r * CC(g->eta_c, j, i) / lap;
        }
    out[0] = rv;
    out[1] = rp;
    out[2] = ff;
    free(bx);
    free(by);
}

/* ------------------------------------------------------------------------ */
/* geometric multigrid V-cycle for M v = b (Sec. 3.2, configuration Sec. 6.2) */
/* ------------------------------------------------------------------------ */
/* The paper fixes only the level count, the sweep counts and their growth per
 * level; the transfer operators below are this implementation's reading:
 *  - coarsening halves nx and ny while both are even and larger than
 *    `coarsest`, up to `max_levels` levels;
 *  - coarse eta_c = mean of its four children; coarse eta_n at an interior
 *    node = full-weighting mean of the 3 x 3 fine nodes around the coincident
 *    fine node (weights 4 centre, 2 edges, 1 corners, over 16), boundary
 *    nodes 0 (injecting eta_n makes the coarse operator too soft next to
 *    stiff inclusions and the cycle diverges at high viscosity contrast);
 *    the coarse operator is the same stencil on the coarse grid;
 *  - prolongation P: bilinear interpolation in the staggered coordinates,
 *    mirror ghosts (free slip) for the tangential direction, zero walls;
 *  - restriction R = P^T / 4 (the adjoint of P, rows summing to one inside);
 *  - the coarsest level is solved exactly (dense Cholesky of -M);
 *  - level l runs ceil(nu_pre g^l) pre- and ceil(nu_post g^l) post-sweeps
 *    (Sec. 6.2), each capped at nu_max when nu_max > 0;
 *  - a RAS smoother on level l, phase ph (0 pre, 1 post) draws its tile
 *    shifts from SplitMix64 seeded with splitmix64(seed, 2 l + ph): the same
 *    in every cycle, so one V-cycle is one fixed linear map. */

typedef struct {
    int nx, ny;
    double hx, hy;
    double *eta_c, *eta_n;
} level_t;

static int mg_build(int nx, int ny, double hx, double hy, const double *eta_c, const double *eta_n,
                    int max_levels, int coarsest, level_t *lv)
{
    int L = 0;
    lv[0].nx = nx; lv[0].ny = ny; lv[0].hx = hx; lv[0].hy = hy;
    lv[0].eta_c = malloc((size_t)nx * ny * sizeof(double));
    lv[0].eta_n = malloc((size_t)(nx + 1) * (ny + 1) * sizeof(double));
    memcpy(lv[0].eta_c, eta_c, (size_t)nx * ny * sizeof(double));
    memcpy(lv[0].eta_n, eta_n, (size_t)(nx + 1) * (ny + 1) * sizeof(double));
    L = 1;
    while (L < max_levels) {
        level_t *f = &lv[L - 1];
        if (f->nx % 2 || f->ny % 2 || f->nx <= coarsest || f->ny <= coarsest) break;
        level_t *c = &lv[L];
        c->nx = f->nx / 2; c->ny = f->ny / 2; c->hx = 2.0 * f->hx; c->hy = 2.0 * f->hy;
        c->eta_c = malloc((size_t)c->nx * c->ny * sizeof(double));
        c->eta_n = malloc((size_t)(c->nx + 1) * (c->ny + 1) * sizeof(double));
        for (int J = 0; J < c->ny; ++J)
            for (int I = 0; I < c->nx; ++I) {
                const double *e = f->eta_c;
                int fn = f->nx;
                double s = e[(2 * J) * fn + 2 * I] + e[(2 * J) * fn + 2 * I + 1] + e[(2 * J + 1) * fn + 2 * I]
                           + e[(2 * J + 1) * fn + 2 * I + 1];
                c->eta_c[J * c->nx + I] = 0.25 * s;
            }
        for (int J = 0; J <= c->ny; ++J)
            for (int I = 0; I <= c->nx; ++I) {
                double v = 0.0;
                if (I >= 1 && I <= c->nx - 1 && J >= 1 && J <= c->ny - 1) {
                    const double *e = f->eta_n;
                    int fn = f->nx + 1, j = 2 * J, i = 2 * I;
                    double centre = e[j * fn + i];
                    double edges = e[(j - 1) * fn + i] + e[(j + 1) * fn + i] + e[j * fn + i - 1] + e[j * fn + i + 1];
                    double corners = e[(j - 1) * fn + i - 1] + e[(j - 1) * fn + i + 1] + e[(j + 1) * fn + i - 1]
                                     + e[(j + 1) * fn + i + 1];
                    v = (4.0 * centre + 2.0 * edges + corners) / 16.0;
                }
                c->eta_n[J * (c->nx + 1) + I] = v;
            }
        ++L;
    }
    return L;
}

static void mg_free(level_t *lv, int L)
{
    for (int l = 0; l < L; ++l) {
        free(lv[l].eta_c);
        free(lv[l].eta_n);
    }
}

/* number of levels the hierarchy has */
int ora_mg_levels(int nx, int ny, int max_levels, int coarsest)
{
    int L = 1;
    while (L < max_levels && nx % 2 == 0 && ny % 2 == 0 && nx > coarsest && ny > coarsest) {
        nx /= 2;
        ny /= 2;
        ++L;
    }
    return L;
}

/* sweeps on level l: ceil(nu0 * growth^l), capped at nu_max when nu_max > 0 */
int ora_mg_sweeps(int nu0, double growth, int l, int nu_max)
{
    double f = (double)nu0;
    for (int q = 0; q < l; ++q) f *= growth;
    int nu = (int)ceil(f);
    return (nu_max > 0 && nu > nu_max) ? nu_max : nu;
}

/* 1D interpolation weights of the prolongation.
 * Cell-centred direction: fine index a lies at coarse position (a - 1/2)/2;
 * weights 3/4 (nearest coarse) and 1/4 (next), mirrored at the walls.
 * Node-centred direction: even a = coarse a/2, odd a = half of each neighbour. */
static int w_cell(int a, int nc, int *idx, double *w)
{
    int A = a >> 1;
    int B = (a & 1) ? A + 1 : A - 1;
    if (B < 0) B = 0;
    if (B > nc - 1) B = nc - 1;
    idx[0] = A; w[0] = 0.75;
    idx[1] = B; w[1] = 0.25;
    return 2;
}

static int w_node(int a, int *idx, double *w)
{
    if ((a & 1) == 0) {
        idx[0] = a >> 1; w[0] = 1.0;
        return 1;
    }
    idx[0] = a >> 1; w[0] = 0.5;
    idx[1] = (a >> 1) + 1; w[1] = 0.5;
    return 2;
}

/* fine += P coarse (unknowns only) */
static void mg_prolong_add(const level_t *F, const level_t *C, const double *cx, const double *cy, double *fx,
                           double *fy)
{
    int iy[2], ix[2];
    double wy[2], wx[2];
    for (int j = 0; j < F->ny; ++j)
        for (int i = 1; i <= F->nx - 1; ++i) {
            int ny_ = w_cell(j, C->ny, iy, wy), nx_ = w_node(i, ix, wx);
            double s = 0.0;
            for (int a = 0; a < ny_; ++a)
                for (int b = 0; b < nx_; ++b) s += wy[a] * wx[b] * cx[iy[a] * (C->nx + 1) + ix[b]];
            fx[j * (F->nx + 1) + i] += s;
        }
    for (int j = 1; j <= F->ny - 1; ++j)
        for (int i = 0; i < F->nx; ++i) {
            int ny_ = w_node(j, iy, wy), nx_ = w_cell(i, C->nx, ix, wx);
            double s = 0.0;
            for (int a = 0; a < ny_; ++a)
                for (int b = 0; b < nx_; ++b) s += wy[a] * wx[b] * cy[iy[a] * C->nx + ix[b]];
            fy[j * F->nx + i] += s;
        }
}

/* coarse = P^T fine / 4 at coarse unknowns (coarse walls stay zero) */
static void mg_restrict(const level_t *F, const level_t *C, const double *fx, const double *fy, double *cx,
                        double *cy)
{
    int iy[2], ix[2];
    double wy[2], wx[2];
    memset(cx, 0, (size_t)C->ny * (C->nx + 1) * sizeof(double));
    memset(cy, 0, (size_t)(C->ny + 1) * C->nx * sizeof(double));
    for (int j = 0; j < F->ny; ++j)
        for (int i = 1; i <= F->nx - 1; ++i) {
            int ny_ = w_cell(j, C->ny, iy, wy), nx_ = w_node(i, ix, wx);
            for (int a = 0; a < ny_; ++a)
                for (int b = 0; b < nx_; ++b)
                    if (ix[b] >= 1 && ix[b] <= C->nx - 1)
                        cx[iy[a] * (C->nx + 1) + ix[b]] += 0.25 * (wy[a] * wx[b]) * fx[j * (F->nx + 1) + i];
        }
    for (int j = 1; j <= F->ny - 1; ++j)
        for (int i = 0; i < F->nx; ++i) {
            int ny_ = w_node(j, iy, wy), nx_ = w_cell(i, C->nx, ix, wx);
            for (int a = 0; a < ny_; ++a)
                for (int b = 0; b < nx_; ++b)
                    if (iy[a] >= 1 && iy[a] <= C->ny - 1)
                        cy[iy[a] * C->nx + ix[b]] += 0.25 * (wy[a] * wx[b]) * fy[j * F->nx + i];
        }
}

/* exported for tests: one prolongation (fine += P coarse) and one restriction */
void ora_mg_prolong_add(int nxf, int nyf, const double *cx, const double *cy, double *fx, double *fy)
{
    level_t F = {nxf, nyf, 1.0, 1.0, NULL, NULL}, C = {nxf / 2, nyf / 2, 2.0, 2.0, NULL, NULL};
    mg_prolong_add(&F, &C, cx, cy, fx, fy);
}

void ora_mg_restrict(int nxf, int nyf, const double *fx, const double *fy, double *cx, double *cy)
{
    level_t F = {nxf, nyf, 1.0, 1.0, NULL, NULL}, C = {nxf / 2, nyf / 2, 2.0, 2.0, NULL, NULL};
    mg_restrict(&F, &C, fx, fy, cx, cy);
}

/* unknown numbering for the dense coarsest solve: vx unknowns row-major,
 * then vy unknowns row-major */
static int n_unknowns(int nx, int ny) { return ny * (nx - 1) + (ny - 1) * nx; }

/* Assemble A = -M column by column (unit-vector applies) and factor A = L L^T
 * in place (lower triangle).  Returns 0, or -1 if A is not positive definite. */
static int dense_factor(const level_t *lv, double *A, int n)
{
    int nx = lv->nx, ny = lv->ny;
    double *ux = calloc((size_t)ny * (nx + 1), sizeof(double)), *uy = calloc((size_t)(ny + 1) * nx, sizeof(double));
    double *mx = malloc((size_t)ny * (nx + 1) * sizeof(double)), *my = malloc((size_t)(ny + 1) * nx * sizeof(double));
    int col = 0;
    for (int comp = 0; comp < 2; ++comp) {
        int jlo = comp ? 1 : 0, jhi = comp ? ny - 1 : ny - 1;
        int ilo = comp ? 0 : 1, ihi = comp ? nx - 1 : nx - 1;
        for (int j = jlo; j <= jhi; ++j)
            for (int i = ilo; i <= ihi; ++i) {
                double *u = comp ? &uy[j * nx + i] : &ux[j * (nx + 1) + i];
                *u = 1.0;
                ora_apply_M(nx, ny, lv->hx, lv->hy, lv->eta_c, lv->eta_n, ux, uy, mx, my);
                *u = 0.0;
                int row = 0;
                for (int jj = 0; jj < ny; ++jj)
                    for (int ii = 1; ii <= nx - 1; ++ii) A[(size_t)row++ * n + col] = -mx[jj * (nx + 1) + ii];
                for (int jj = 1; jj <= ny - 1; ++jj)
                    for (int ii = 0; ii < nx; ++ii) A[(size_t)row++ * n + col] = -my[jj * nx + ii];
                ++col;
            }
    }
    free(ux); free(uy); free(mx); free(my);
    /* Cholesky-Banachiewicz */
    for (int r = 0; r < n; ++r) {
        for (int c = 0; c <= r; ++c) {
            double s = A[(size_t)r * n + c];
            for (int q = 0; q < c; ++q) s -= A[(size_t)r * n + q] * A[(size_t)c * n + q];
            if (r == c) {
                if (!(s > 0.0)) return -1;
                A[(size_t)r * n + r] = sqrt(s);
            } else {
                A[(size_t)r * n + c] = s / A[(size_t)c * n + c];
            }
        }
    }
    return 0;
}

/* solve M e = r on the coarsest level: e = (-M)^{-1} (-r) */
static int dense_solve(const level_t *lv, const double *rx, const double *ry, double *ex, double *ey)
{
    int nx = lv->nx, ny = lv->ny, n = n_unknowns(nx, ny);
    double *A = malloc((size_t)n * n * sizeof(double)), *y = malloc((size_t)n * sizeof(double));
    if (dense_factor(lv, A, n)) { free(A); free(y); return -1; }
    int row = 0;
    for (int j = 0; j < ny; ++j)
        for (int i = 1; i <= nx - 1; ++i) y[row++] = -rx[j * (nx + 1) + i];
    for (int j = 1; j <= ny - 1; ++j)
        for (int i = 0; i < nx; ++i) y[row++] = -ry[j * nx + i];
    for (int r = 0; r < n; ++r) { /* L z = y */
        double s = y[r];
        for (int q = 0; q < r; ++q) s -= A[(size_t)r * n + q] * y[q];
        y[r] = s / A[(size_t)r * n + r];
    }
    for (int r = n - 1; r >= 0; --r) { /* L^T e = z */
        double s = y[r];
        for (int q = r + 1; q < n; ++q) s -= A[(size_t)q * n + r] * y[q];
        y[r] = s / A[(size_t)r * n + r];
    }
    memset(ex, 0, (size_t)ny * (nx + 1) * sizeof(double));
    memset(ey, 0, (size_t)(ny + 1) * nx * sizeof(double));
    row = 0;
    for (int j = 0; j < ny; ++j)
        for (int i = 1; i <= nx - 1; ++i) ex[j * (nx + 1) + i] = y[row++];
    for (int j = 1; j <= ny - 1; ++j)
        for (int i = 0; i < nx; ++i) ey[j * nx + i] = y[row++];
    free(A); free(y);
    return 0;
}

/* exported for tests: exact solve of M v = b on a small grid */
int ora_dense_solve(int nx, int ny, double hx, double hy, const double *eta_c, const double *eta_n,
                    const double *bx, const double *by, double *vx, double *vy)
{
    level_t lv = {nx, ny, hx, hy, (double *)eta_c, (double *)eta_n};
    return dense_solve(&lv, bx, by, vx, vy);
}

/* smoother codes shared with the C interface's enumeration */
/* ORA_MIXED (V-cycle only): the "mixed" smoother of Sec. 6.3, Jacobi on the
 * finest level and RAS on every coarser level. */
enum { ORA_JACOBI = 0, ORA_JACOBI_FUSED = 1, ORA_JACOBI_BLOCKED = 2, ORA_RBGS = 3, ORA_RAS = 4, ORA_MIXED = 5 };

typedef struct {
    int variant, ti, tj, k, overlap;
    double omega;
    uint64_t seed;
    int nu_max;
} smoother_t;

static void run_smoother(const level_t *lv, int level, const smoother_t *sm, const double *bx, const double *by,
                         int sweeps, uint64_t call_index, double *vx, double *vy)
{
    if (sweeps <= 0) return;
    int variant = sm->variant;
    if (variant == ORA_MIXED) variant = level == 0 ? ORA_JACOBI : ORA_RAS;
    if (variant == ORA_RBGS)
        ora_rbgs(lv->nx, lv->ny, lv->hx, lv->hy, lv->eta_c, lv->eta_n, bx, by, sm->omega, sweeps, vx, vy);
    else if (variant == ORA_RAS)
        ora_ras(lv->nx, lv->ny, lv->hx, lv->hy, lv->eta_c, lv->eta_n, bx, by, sm->omega, sweeps, sm->ti, sm->tj,
                sm->k, sm->overlap, 1, ora_splitmix64(sm->seed, call_index), NULL, 0, vx, vy, NULL);
    else
        ora_jacobi(lv->nx, lv->ny, lv->hx, lv->hy, lv->eta_c, lv->eta_n, bx, by, sm->omega, sweeps, vx, vy);
}

/* r = b - M v at unknowns, zero at walls */
static void residual(const level_t *lv, const double *bx, const double *by, const double *vx, const double *vy,
                     double *rx, double *ry)
{
    int nx = lv->nx, ny = lv->ny;
    ora_apply_M(nx, ny, lv->hx, lv->hy, lv->eta_c, lv->eta_n, vx, vy, rx, ry);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i <= nx; ++i) {
            size_t q = (size_t)j * (nx + 1) + i;
            rx[q] = (i >= 1 && i <= nx - 1) ? bx[q] - rx[q] : 0.0;
        }
    for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t q = (size_t)j * nx + i;
            ry[q] = (j >= 1 && j <= ny - 1) ? by[q] - ry[q] : 0.0;
        }
}

static int vcycle_rec(level_t *lv, int L, int l, const smoother_t *sm, int nu_pre, int nu_post, double growth,
                      const double *bx, const double *by, double *vx, double *vy)
{
    level_t *F = &lv[l];
    if (l == L - 1) {
        double *ex = malloc((size_t)F->ny * (F->nx + 1) * sizeof(double));
        double *ey = malloc((size_t)(F->ny + 1) * F->nx * sizeof(double));
        double *rx = malloc((size_t)F->ny * (F->nx + 1) * sizeof(double));
        double *ry = malloc((size_t)(F->ny + 1) * F->nx * sizeof(double));
        residual(F, bx, by, vx, vy, rx, ry);
        int st = dense_solve(F, rx, ry, ex, ey);
        for (size_t q = 0; q < (size_t)F->ny * (F->nx + 1); ++q) vx[q] += ex[q];
        for (size_t q = 0; q < (size_t)(F->ny + 1) * F->nx; ++q) vy[q] += ey[q];
        free(ex); free(ey); free(rx); free(ry);
        return st;
    }
    uint64_t base = (uint64_t)l * 2u;
    run_smoother(F, l, sm, bx, by, ora_mg_sweeps(nu_pre, growth, l, sm->nu_max), base, vx, vy);
    level_t *C = &lv[l + 1];
    size_t fnx = (size_t)F->ny * (F->nx + 1), fny = (size_t)(F->ny + 1) * F->nx;
    size_t cnx = (size_t)C->ny * (C->nx + 1), cny = (size_t)(C->ny + 1) * C->nx;
    double *rx = malloc(fnx * sizeof(double)), *ry = malloc(fny * sizeof(double));
    double *cbx = malloc(cnx * sizeof(double)), *cby = malloc(cny * sizeof(double));
    double *cvx = calloc(cnx, sizeof(double)), *cvy = calloc(cny, sizeof(double));
    residual(F, bx, by, vx, vy, rx, ry);
    mg_restrict(F, C, rx, ry, cbx, cby);
    int st = vcycle_rec(lv, L, l + 1, sm, nu_pre, nu_post, growth, cbx, cby, cvx, cvy);
    mg_prolong_add(F, C, cvx, cvy, vx, vy);
    run_smoother(F, l, sm, bx, by, ora_mg_sweeps(nu_post, growth, l, sm->nu_max), base + 1u, vx, vy);
    free(rx); free(ry); free(cbx); free(cby); free(cvx); free(cvy);
    return st;
}

/* One V-cycle for M v = b, improving (vx, vy) in place (the shift seeds are
 * described at the top of this section).  Returns 0, or -1 if the coarsest
 * matrix is not positive definite / the arguments are bad. */
int ora_vcycle(int nx, int ny, double hx, double hy, const double *eta_c, const double *eta_n, const double *bx,
               const double *by, int max_levels, int coarsest, int nu_pre, int nu_post, double growth, int nu_max,
               int variant, double omega, int ti, int tj, int k, int overlap, uint64_t seed, double *vx, double *vy)
{
    if (max_levels < 1 || max_levels > 32) return -1;
    level_t lv[32];
    int L = mg_build(nx, ny, hx, hy, eta_c, eta_n, max_levels, coarsest, lv);
    smoother_t sm = {variant, ti, tj, k, overlap, omega, seed, nu_max};
    int st = vcycle_rec(lv, L, 0, &sm, nu_pre, nu_post, growth, bx, by, vx, vy);
    mg_free(lv, L);
    return st;
}

/* relative velocity energy residual E_v = sqrt(sum r_v^2/(-d) / sum f^2/(-d)) */
static double energy_v(const level_t *lv, const double *fx, const double *fy, const double *rx, const double *ry)
{
    grid_t G = mkgrid(lv->nx, lv->ny, lv->hx, lv->hy, lv->eta_c, lv->eta_n), *g = &G;
    double num = 0.0, den = 0.0;
    for (int j = 0; j < g->ny; ++j)
        for (int i = 1; i <= g->nx - 1; ++i) {
            double w = -dmx_at(g, j, i);
            num += VX(rx, j, i) * VX(rx, j, i) / w;
            den += VX(fx, j, i) * VX(fx, j, i) / w;
        }
    for (int j = 1; j <= g->ny - 1; ++j)
        for (int i = 0; i < g->nx; ++i) {
            double w = -dmy_at(g, j, i);
            num += VY(ry, j, i) * VY(ry, j, i) / w;
            den += VY(fy, j, i) * VY(fy, j, i) / w;
        }
    return sqrt(num / den);
}

/* Defect-correction solve of M v = f - G p: repeat { r = b - M v; stop when
 * E_v <= tol; e = Vcycle(r, 0); v += e }.  history (optional, max_cycles+1
 * entries) receives E_v before each cycle.  Returns the number of cycles run,
 * or -1 on failure; *final_e receives the last E_v. */
int ora_mg_solve(int nx, int ny, double hx, double hy, const double *eta_c, const double *eta_n, const double *fx,
                 const double *fy, const double *p, int max_levels, int coarsest, int nu_pre, int nu_post,
                 double growth, int nu_max, int variant, double omega, int ti, int tj, int k, int overlap,
                 uint64_t seed, double tol, int max_cycles, double *vx, double *vy, double *final_e,
                 double *history)
{
    if (max_levels < 1 || max_levels > 32) return -1;
    level_t lv[32];
    int L = mg_build(nx, ny, hx, hy, eta_c, eta_n, max_levels, coarsest, lv);
    smoother_t sm = {variant, ti, tj, k, overlap, omega, seed, nu_max};
    size_t snx = (size_t)ny * (nx + 1), sny = (size_t)(ny + 1) * nx;
    double *bx = malloc(snx * sizeof(double)), *by = malloc(sny * sizeof(double));
    double *rx = malloc(snx * sizeof(double)), *ry = malloc(sny * sizeof(double));
    double *ex = malloc(snx * sizeof(double)), *ey = malloc(sny * sizeof(double));
    ora_rhs(nx, ny, hx, hy, fx, fy, p, bx, by);
    int c = 0, st = 0;
    double e = 0.0;
    for (;;) {
        residual(&lv[0], bx, by, vx, vy, rx, ry);
        e = energy_v(&lv[0], fx, fy, rx, ry);
        if (history) history[c] = e;
        if (e <= tol || c >= max_cycles) break;
        memset(ex, 0, snx * sizeof(double));
        memset(ey, 0, sny * sizeof(double));
        if (vcycle_rec(lv, L, 0, &sm, nu_pre, nu_post, growth, rx, ry, ex, ey)) { st = -1; break; }
        for (size_t q = 0; q < snx; ++q) vx[q] += ex[q];
        for (size_t q = 0; q < sny; ++q) vy[q] += ey[q];
        ++c;
    }
    if (final_e) *final_e = e;
    free(bx); free(by); free(rx); free(ry); free(ex); free(ey);
    mg_free(lv, L);
    return st ? -1 : c;
}

/* One RAS outer iteration restricted to a list of tiles: tiles (bx, by) =
 * (tiles[2q], tiles[2q+1]) of the tiling with shift (si, sj) run `ksweeps`
 * local sweeps from the snapshot (vx, vy) and write their owned unknowns to
 * (ox, oy); every other entry of (ox, oy) is left as it is.  Used to check
 * sampled tiles of full-size runs.  Returns 0, or -1 on bad arguments. */
int ora_ras_tiles(int nx, int ny, double hx, double hy, const double *eta_c, const double *eta_n,
                  const double *bx, const double *by, double omega, int ti, int tj, int ksweeps, int overlap,
                  int si, int sj, const int *tiles, int ntiles, const double *vx, const double *vy, double *ox,
                  double *oy)
{
    if (nx < 1 || ny < 1 || ti < 1 || tj < 1 || ksweeps < 0 || overlap < 0) return -1;
    grid_t G = mkgrid(nx, ny, hx, hy, eta_c, eta_n), *g = &G;
    int *cx = malloc((size_t)(nx / ti + 3) * sizeof(int));
    int *cy = malloc((size_t)(ny / tj + 3) * sizeof(int));
    int ntx = tile_cuts(nx, ti, si, cx), nty = tile_cuts(ny, tj, sj, cy);
    double *wx = malloc(nvx(g) * sizeof(double)), *wy = malloc(nvy(g) * sizeof(double));
    double *tx = malloc(nvx(g) * sizeof(double)), *ty = malloc(nvy(g) * sizeof(double));
    memcpy(wx, vx, nvx(g) * sizeof(double));
    memcpy(wy, vy, nvy(g) * sizeof(double));
    memcpy(tx, vx, nvx(g) * sizeof(double));
    memcpy(ty, vy, nvy(g) * sizeof(double));
    int st = 0;
    for (int q = 0; q < ntiles; ++q) {
        int bxi = tiles[2 * q], byj = tiles[2 * q + 1];
        if (bxi < 0 || bxi >= ntx || byj < 0 || byj >= nty) { st = -1; break; }
        int x0 = cx[bxi], x1 = cx[bxi + 1], y0 = cy[byj], y1 = cy[byj + 1];
        int lx0 = x0 - overlap < 0 ? 0 : x0 - overlap, lx1 = x1 + overlap > nx ? nx : x1 + overlap;
        int ly0 = y0 - overlap < 0 ? 0 : y0 - overlap, ly1 = y1 + overlap > ny ? ny : y1 + overlap;
        for (int s = 0; s < ksweeps; ++s) {
            for (int j = ly0; j < ly1; ++j)
                for (int i = lx0; i < lx1; ++i) {
                    if (is_vx_unknown(g, j, i)) VX(tx, j, i) = jacobi_x(g, wx, wy, bx, omega, j, i);
                    if (is_vy_unknown(g, j, i)) VY(ty, j, i) = jacobi_y(g, wx, wy, by, omega, j, i);
                }
            for (int j = ly0; j < ly1; ++j)
                for (int i = lx0; i < lx1; ++i) {
                    if (is_vx_unknown(g, j, i)) VX(wx, j, i) = VX(tx, j, i);
                    if (is_vy_unknown(g, j, i)) VY(wy, j, i) = VY(ty, j, i);
                }
        }
        for (int j = y0; j < y1; ++j)
            for (int i = x0; i < x1; ++i) {
                if (is_vx_unknown(g, j, i)) VX(ox, j, i) = VX(wx, j, i);
                if (is_vy_unknown(g, j, i)) VY(oy, j, i) = VY(wy, j, i);
            }
        for (int j = ly0; j < ly1; ++j)
            for (int i = lx0; i < lx1; ++i) {
                if (is_vx_unknown(g, j, i)) VX(wx, j, i) = VX(tx, j, i) = VX(vx, j, i);
                if (is_vy_unknown(g, j, i)) VY(wy, j, i) = VY(ty, j, i) = VY(vy, j, i);
            }
    }
    free(wx); free(wy); free(tx); free(ty); free(cx); free(cy);
    return st;
}

/* Number of tiles per direction of the tiling of [0, n) cut at s + m T. */
int ora_tile_count(int n, int T, int s)
{
    int *c = malloc((size_t)(n / T + 3) * sizeof(int));
    int m = tile_cuts(n, T, s, c);
    free(c);
    return m;
}

/* Flexible conjugate gradients (one-term recurrence) for M v = f - G p with
 * one V-cycle as the preconditioner B ~ M^{-1} (M is negative definite, so
 * every quotient below is well defined):
 *   r = b - M v, z = B r, p = z;
 *   repeat { q = M p; a = <p, r> / <p, q>; v += a p; r -= a q;
 *            stop when E_v(r) <= tol; z = B r; beta = -<z, q> / <p, q>;
 *            p = z + beta p }
 * Inner products run over the velocity unknowns.  The velocity solve of
 * Sec. 3.2 needs only an approximate M^{-1}; this Krylov acceleration of the
 * multigrid cycle is what drives E_v to 1e-8 at high viscosity contrast.
 * history (optional, max_its+1 entries) receives E_v before each iteration.
 * Returns the number of iterations, or -1 on failure. */
static double dot_unk(const level_t *lv, const double *ax, const double *ay, const double *bx, const double *by)
{
    int nx = lv->nx, ny = lv->ny;
    double s = 0.0;
    for (int j = 0; j < ny; ++j)
        for (int i = 1; i <= nx - 1; ++i) s += ax[j * (nx + 1) + i] * bx[j * (nx + 1) + i];
    for (int j = 1; j <= ny - 1; ++j)
        for (int i = 0; i < nx; ++i) s += ay[j * nx + i] * by[j * nx + i];
    return s;
}

int ora_mg_fcg(int nx, int ny, double hx, double hy, const double *eta_c, const double *eta_n, const double *fx,
               const double *fy, const double *p, int max_levels, int coarsest, int nu_pre, int nu_post,
               double growth, int nu_max, int variant, double omega, int ti, int tj, int k, int overlap,
               uint64_t seed, double tol, int max_its, double *vx, double *vy, double *final_e, double *history)
{
    if (max_levels < 1 || max_levels > 32) return -1;
    level_t lv[32];
    int L = mg_build(nx, ny, hx, hy, eta_c, eta_n, max_levels, coarsest, lv);
    smoother_t sm = {variant, ti, tj, k, overlap, omega, seed, nu_max};
    size_t snx = (size_t)ny * (nx + 1), sny = (size_t)(ny + 1) * nx;
    double *bx = malloc(snx * 8), *by = malloc(sny * 8), *rx = malloc(snx * 8), *ry = malloc(sny * 8);
    double *zx = malloc(snx * 8), *zy = malloc(sny * 8), *px = malloc(snx * 8), *py = malloc(sny * 8);
    double *qx = malloc(snx * 8), *qy = malloc(sny * 8);
    ora_rhs(nx, ny, hx, hy, fx, fy, p, bx, by);
    residual(&lv[0], bx, by, vx, vy, rx, ry);
    int it = 0, st = 0;
    double e = energy_v(&lv[0], fx, fy, rx, ry);
    if (history) history[0] = e;
    if (e > tol && max_its > 0) {
        memset(zx, 0, snx * 8);
        memset(zy, 0, sny * 8);
        st = vcycle_rec(lv, L, 0, &sm, nu_pre, nu_post, growth, rx, ry, zx, zy);
        memcpy(px, zx, snx * 8);
        memcpy(py, zy, sny * 8);
        while (!st) {
            ora_apply_M(nx, ny, hx, hy, eta_c, eta_n, px, py, qx, qy);
            double pq = dot_unk(&lv[0], px, py, qx, qy);
            double a = dot_unk(&lv[0], px, py, rx, ry) / pq;
            for (size_t q = 0; q < snx; ++q) { vx[q] += a * px[q]; rx[q] -= a * qx[q]; }
            for (size_t q = 0; q < sny; ++q) { vy[q] += a * py[q]; ry[q] -= a * qy[q]; }
            ++it;
            e = energy_v(&lv[0], fx, fy, rx, ry);
            if (history) history[it] = e;
            if (e <= tol || it >= max_its) break;
            memset(zx, 0, snx * 8);
            memset(zy, 0, sny * 8);
            st = vcycle_rec(lv, L, 0, &sm, nu_pre, nu_post, growth, rx, ry, zx, zy);
            double beta = -dot_unk(&lv[0], zx, zy, qx, qy) / pq;
            for (size_t q = 0; q < snx; ++q) px[q] = zx[q] + beta * px[q];
            for (size_t q = 0; q < sny; ++q) py[q] = zy[q] + beta * py[q];
        }
    }
    if (final_e) *final_e = e;
    free(bx); free(by); free(rx); free(ry); free(zx); free(zy); free(px); free(py); free(qx); free(qy);
    mg_free(lv, L);
    return st ? -1 : it;
}
