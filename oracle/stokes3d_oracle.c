/*
 * stokes3d_oracle.c -- plain, slow, FP64 CPU statement of the 3D staggered-grid
 * variable-viscosity Stokes velocity operator, damped Jacobi, RAS-Jacobi on 3D
 * tiles and the energy residual norm: the 3D extension the paper names as
 * future work (Sec. 9), written with the same readings as the 2D oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path loads this file: only
 * the tests, the smoke check and the CPU-baseline leg of the benchmark may.  It
 * shares no code, header, table or helper with the CUDA library.
 *
 * Grid (the 3D counterpart of Sec. 2.1): nx x ny x nz cells, h = (hx, hy, hz).
 * Natural layouts (z-major, then y, then x), every index range inclusive of
 * the walls:
 *   vx : nz x ny x (nx+1)       at (i hx, (j+1/2) hy, (k+1/2) hz)
 *   vy : nz x (ny+1) x nx       at ((i+1/2) hx, j hy, (k+1/2) hz)
 *   vz : (nz+1) x ny x nx       at ((i+1/2) hx, (j+1/2) hy, k hz)
 *   p, eta_c : nz x ny x nx     at cell centres
 *   eta_xy : nz x (ny+1) x (nx+1)   at x-y edges (i hx, j hy, (k+1/2) hz), sigma'_xy
 *   eta_xz : (nz+1) x ny x (nx+1)   at x-z edges (i hx, (j+1/2) hy, k hz), sigma'_xz
 *   eta_yz : (nz+1) x (ny+1) x nx   at y-z edges ((i+1/2) hx, j hy, k hz), sigma'_yz
 * Unknowns: vx with 1 <= i <= nx-1, vy with 1 <= j <= ny-1, vz with
 * 1 <= k <= nz-1; the wall entries are Dirichlet data, never written.
 *
 * Readings (each listed in the design notes):
 *  - Eq. (3) in 3D: sigma'_ii = 2 eta dv_i/dx_i at cells, sigma'_ij = eta
 *    (dv_i/dx_j + dv_j/dx_i) at the edges where both derivatives are centred;
 *  - free slip on every wall: a shear stress is zero on an edge that lies in a
 *    wall it is tangential to (sigma'_xy on x = 0, Lx and y = 0, Ly, ...);
 *  - Jacobi and RAS exactly as in 2D; a RAS tile is a box of T_I x T_J x T_K
 *    cells cut at s + m T in each direction, the shifts of outer iteration t
 *    are SplitMix64 draws 3t, 3t+1, 3t+2 of the seed taken mod T_I, T_J, T_K,
 *    a tile owns the unknowns of its cells (a cell owns its low faces);
 *  - energy norm: the 2D sums of Sec. 6.4 over the three components, the
 *    pressure weight eta_c / (2/hx^2 + 2/hy^2 + 2/hz^2).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int nx, ny, nz;
    double hx, hy, hz;
    const double *ec, *exy, *exz, *eyz;
} g3_t;

#define X3(a, k, j, i) (a)[((size_t)(k) * (size_t)g->ny + (size_t)(j)) * (size_t)(g->nx + 1) + (size_t)(i)]
#define Y3(a, k, j, i) (a)[((size_t)(k) * (size_t)(g->ny + 1) + (size_t)(j)) * (size_t)g->nx + (size_t)(i)]
#define Z3(a, k, j, i) (a)[((size_t)(k) * (size_t)g->ny + (size_t)(j)) * (size_t)g->nx + (size_t)(i)]
#define C3(a, k, j, i) (a)[((size_t)(k) * (size_t)g->ny + (size_t)(j)) * (size_t)g->nx + (size_t)(i)]
#define EXY(k, j, i) g->exy[((size_t)(k) * (size_t)(g->ny + 1) + (size_t)(j)) * (size_t)(g->nx + 1) + (size_t)(i)]
#define EXZ(k, j, i) g->exz[((size_t)(k) * (size_t)g->ny + (size_t)(j)) * (size_t)(g->nx + 1) + (size_t)(i)]
#define EYZ(k, j, i) g->eyz[((size_t)(k) * (size_t)(g->ny + 1) + (size_t)(j)) * (size_t)g->nx + (size_t)(i)]

static g3_t mk3(int nx, int ny, int nz, double hx, double hy, double hz, const double *ec, const double *exy,
                const double *exz, const double *eyz)
{
    g3_t g;
    g.nx = nx; g.ny = ny; g.nz = nz;
    g.hx = hx; g.hy = hy; g.hz = hz;
    g.ec = ec; g.exy = exy; g.exz = exz; g.eyz = eyz;
    return g;
}

static size_t n_vx(const g3_t *g) { return (size_t)g->nz * g->ny * (g->nx + 1); }
static size_t n_vy(const g3_t *g) { return (size_t)g->nz * (g->ny + 1) * g->nx; }
static size_t n_vz(const g3_t *g) { return (size_t)(g->nz + 1) * g->ny * g->nx; }

static int ux3(const g3_t *g, int k, int j, int i)
{
    return k >= 0 && k < g->nz && j >= 0 && j < g->ny && i >= 1 && i <= g->nx - 1;
}
static int uy3(const g3_t *g, int k, int j, int i)
{
    return k >= 0 && k < g->nz && i >= 0 && i < g->nx && j >= 1 && j <= g->ny - 1;
}
static int uz3(const g3_t *g, int k, int j, int i)
{
    return j >= 0 && j < g->ny && i >= 0 && i < g->nx && k >= 1 && k <= g->nz - 1;
}

/* ---- deviatoric stresses --------------------------------------------------- */
static double s_xx(const g3_t *g, const double *vx, int k, int j, int i)
{
    return 2.0 * C3(g->ec, k, j, i) * (X3(vx, k, j, i + 1) - X3(vx, k, j, i)) / g->hx;
}
static double s_yy(const g3_t *g, const double *vy, int k, int j, int i)
{
    return 2.0 * C3(g->ec, k, j, i) * (Y3(vy, k, j + 1, i) - Y3(vy, k, j, i)) / g->hy;
}
static double s_zz(const g3_t *g, const double *vz, int k, int j, int i)
{
    return 2.0 * C3(g->ec, k, j, i) * (Z3(vz, k + 1, j, i) - Z3(vz, k, j, i)) / g->hz;
}
/* x-y edge (i, j) of cell layer k; zero on the x and y walls */
static double s_xy(const g3_t *g, const double *vx, const double *vy, int k, int j, int i)
{
    if (i <= 0 || i >= g->nx || j <= 0 || j >= g->ny) return 0.0;
    double a = (X3(vx, k, j, i) - X3(vx, k, j - 1, i)) / g->hy;
    double b = (Y3(vy, k, j, i) - Y3(vy, k, j, i - 1)) / g->hx;
    return EXY(k, j, i) * (a + b);
}
/* x-z edge (i, k) of cell row j; zero on the x and z walls */
static double s_xz(const g3_t *g, const double *vx, const double *vz, int k, int j, int i)
{
    if (i <= 0 || i >= g->nx || k <= 0 || k >= g->nz) return 0.0;
    double a = (X3(vx, k, j, i) - X3(vx, k - 1, j, i)) / g->hz;
    double b = (Z3(vz, k, j, i) - Z3(vz, k, j, i - 1)) / g->hx;
    return EXZ(k, j, i) * (a + b);
}
/* y-z edge (j, k) of cell column i; zero on the y and z walls */
static double s_yz(const g3_t *g, const double *vy, const double *vz, int k, int j, int i)
{
    if (j <= 0 || j >= g->ny || k <= 0 || k >= g->nz) return 0.0;
    double a = (Y3(vy, k, j, i) - Y3(vy, k - 1, j, i)) / g->hz;
    double b = (Z3(vz, k, j, i) - Z3(vz, k, j - 1, i)) / g->hy;
    return EYZ(k, j, i) * (a + b);
}

/* ---- momentum operator M ---------------------------------------------------- */
static double mx3(const g3_t *g, const double *vx, const double *vy, const double *vz, int k, int j, int i)
{
    return (s_xx(g, vx, k, j, i) - s_xx(g, vx, k, j, i - 1)) / g->hx
           + (s_xy(g, vx, vy, k, j + 1, i) - s_xy(g, vx, vy, k, j, i)) / g->hy
           + (s_xz(g, vx, vz, k + 1, j, i) - s_xz(g, vx, vz, k, j, i)) / g->hz;
}
static double my3(const g3_t *g, const double *vx, const double *vy, const double *vz, int k, int j, int i)
{
    return (s_xy(g, vx, vy, k, j, i + 1) - s_xy(g, vx, vy, k, j, i)) / g->hx
           + (s_yy(g, vy, k, j, i) - s_yy(g, vy, k, j - 1, i)) / g->hy
           + (s_yz(g, vy, vz, k + 1, j, i) - s_yz(g, vy, vz, k, j, i)) / g->hz;
}
static double mz3(const g3_t *g, const double *vx, const double *vy, const double *vz, int k, int j, int i)
{
    return (s_xz(g, vx, vz, k, j, i + 1) - s_xz(g, vx, vz, k, j, i)) / g->hx
           + (s_yz(g, vy, vz, k, j + 1, i) - s_yz(g, vy, vz, k, j, i)) / g->hy
           + (s_zz(g, vz, k, j, i) - s_zz(g, vz, k - 1, j, i)) / g->hz;
}

/* edge viscosities that enter the operator (zero on the walls they are tangential to) */
static double exy_in(const g3_t *g, int k, int j, int i)
{
    return (i <= 0 || i >= g->nx || j <= 0 || j >= g->ny) ? 0.0 : EXY(k, j, i);
}
static double exz_in(const g3_t *g, int k, int j, int i)
{
    return (i <= 0 || i >= g->nx || k <= 0 || k >= g->nz) ? 0.0 : EXZ(k, j, i);
}
static double eyz_in(const g3_t *g, int k, int j, int i)
{
    return (j <= 0 || j >= g->ny || k <= 0 || k >= g->nz) ? 0.0 : EYZ(k, j, i);
}

/* diag(M): the coefficient of an unknown in its own row */
static double dx3(const g3_t *g, int k, int j, int i)
{
    return -2.0 * (C3(g->ec, k, j, i) + C3(g->ec, k, j, i - 1)) / (g->hx * g->hx)
           - (exy_in(g, k, j + 1, i) + exy_in(g, k, j, i)) / (g->hy * g->hy)
           - (exz_in(g, k + 1, j, i) + exz_in(g, k, j, i)) / (g->hz * g->hz);
}
static double dy3(const g3_t *g, int k, int j, int i)
{
    return -(exy_in(g, k, j, i + 1) + exy_in(g, k, j, i)) / (g->hx * g->hx)
           - 2.0 * (C3(g->ec, k, j, i) + C3(g->ec, k, j - 1, i)) / (g->hy * g->hy)
           - (eyz_in(g, k + 1, j, i) + eyz_in(g, k, j, i)) / (g->hz * g->hz);
}
static double dz3(const g3_t *g, int k, int j, int i)
{
    return -(exz_in(g, k, j, i + 1) + exz_in(g, k, j, i)) / (g->hx * g->hx)
           - (eyz_in(g, k, j + 1, i) + eyz_in(g, k, j, i)) / (g->hy * g->hy)
           - 2.0 * (C3(g->ec, k, j, i) + C3(g->ec, k - 1, j, i)) / (g->hz * g->hz);
}

#define HEAD3 int nx, int ny, int nz, double hx, double hy, double hz, const double *ec, const double *exy, \
              const double *exz, const double *eyz
#define MK3 g3_t G = mk3(nx, ny, nz, hx, hy, hz, ec, exy, exz, eyz), *g = &G

/* out = M v at the unknowns, zero elsewhere */
void o3_apply_M(HEAD3, const double *vx, const double *vy, const double *vz, double *ox, double *oy, double *oz)
{
    MK3;
    memset(ox, 0, n_vx(g) * sizeof(double));
    memset(oy, 0, n_vy(g) * sizeof(double));
    memset(oz, 0, n_vz(g) * sizeof(double));
    for (int k = 0; k <= nz; ++k)
        for (int j = 0; j <= ny; ++j)
            for (int i = 0; i <= nx; ++i) {
                if (ux3(g, k, j, i)) X3(ox, k, j, i) = mx3(g, vx, vy, vz, k, j, i);
                if (uy3(g, k, j, i)) Y3(oy, k, j, i) = my3(g, vx, vy, vz, k, j, i);
                if (uz3(g, k, j, i)) Z3(oz, k, j, i) = mz3(g, vx, vy, vz, k, j, i);
            }
}

/* diag(M) at the unknowns, zero elsewhere */
void o3_diag_M(HEAD3, double *ox, double *oy, double *oz)
{
    MK3;
    memset(ox, 0, n_vx(g) * sizeof(double));
    memset(oy, 0, n_vy(g) * sizeof(double));
    memset(oz, 0, n_vz(g) * sizeof(double));
    for (int k = 0; k <= nz; ++k)
        for (int j = 0; j <= ny; ++j)
            for (int i = 0; i <= nx; ++i) {
                if (ux3(g, k, j, i)) X3(ox, k, j, i) = dx3(g, k, j, i);
                if (uy3(g, k, j, i)) Y3(oy, k, j, i) = dy3(g, k, j, i);
                if (uz3(g, k, j, i)) Z3(oz, k, j, i) = dz3(g, k, j, i);
            }
}

/* out = D v = dvx/dx + dvy/dy + dvz/dz at the cells */
void o3_apply_D(int nx, int ny, int nz, double hx, double hy, double hz, const double *vx, const double *vy,
                const double *vz, double *out)
{
    g3_t G = mk3(nx, ny, nz, hx, hy, hz, NULL, NULL, NULL, NULL), *g = &G;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                C3(out, k, j, i) = (X3(vx, k, j, i + 1) - X3(vx, k, j, i)) / hx
                                   + (Y3(vy, k, j + 1, i) - Y3(vy, k, j, i)) / hy
                                   + (Z3(vz, k + 1, j, i) - Z3(vz, k, j, i)) / hz;
}

/* b = f - G p with (G p) = -grad p at the unknowns (p may be NULL), zero elsewhere */
void o3_rhs(int nx, int ny, int nz, double hx, double hy, double hz, const double *fx, const double *fy,
            const double *fz, const double *p, double *bx, double *by, double *bz)
{
    g3_t G = mk3(nx, ny, nz, hx, hy, hz, NULL, NULL, NULL, NULL), *g = &G;
    memset(bx, 0, n_vx(g) * sizeof(double));
    memset(by, 0, n_vy(g) * sizeof(double));
    memset(bz, 0, n_vz(g) * sizeof(double));
    for (int k = 0; k <= nz; ++k)
        for (int j = 0; j <= ny; ++j)
            for (int i = 0; i <= nx; ++i) {
                if (ux3(g, k, j, i))
                    X3(bx, k, j, i) = X3(fx, k, j, i) + (p ? (C3(p, k, j, i) - C3(p, k, j, i - 1)) / hx : 0.0);
                if (uy3(g, k, j, i))
                    Y3(by, k, j, i) = Y3(fy, k, j, i) + (p ? (C3(p, k, j, i) - C3(p, k, j - 1, i)) / hy : 0.0);
                if (uz3(g, k, j, i))
                    Z3(bz, k, j, i) = Z3(fz, k, j, i) + (p ? (C3(p, k, j, i) - C3(p, k - 1, j, i)) / hz : 0.0);
            }
}

/* one damped Jacobi update of an unknown, all from the old v */
static double jx3(const g3_t *g, const double *vx, const double *vy, const double *vz, const double *bx,
                  double omega, int k, int j, int i)
{
    return X3(vx, k, j, i) + omega * (X3(bx, k, j, i) - mx3(g, vx, vy, vz, k, j, i)) / dx3(g, k, j, i);
}
static double jy3(const g3_t *g, const double *vx, const double *vy, const double *vz, const double *by,
                  double omega, int k, int j, int i)
{
    return Y3(vy, k, j, i) + omega * (Y3(by, k, j, i) - my3(g, vx, vy, vz, k, j, i)) / dy3(g, k, j, i);
}
static double jz3(const g3_t *g, const double *vx, const double *vy, const double *vz, const double *bz,
                  double omega, int k, int j, int i)
{
    return Z3(vz, k, j, i) + omega * (Z3(bz, k, j, i) - mz3(g, vx, vy, vz, k, j, i)) / dz3(g, k, j, i);
}

/* `sweeps` damped Jacobi sweeps in place */
void o3_jacobi(HEAD3, const double *bx, const double *by, const double *bz, double omega, int sweeps, double *vx,
               double *vy, double *vz)
{
    MK3;
    double *tx = malloc(n_vx(g) * sizeof(double)), *ty = malloc(n_vy(g) * sizeof(double));
    double *tz = malloc(n_vz(g) * sizeof(double));
    for (int s = 0; s < sweeps; ++s) {
        memcpy(tx, vx, n_vx(g) * sizeof(double));
        memcpy(ty, vy, n_vy(g) * sizeof(double));
        memcpy(tz, vz, n_vz(g) * sizeof(double));
        for (int k = 0; k <= nz; ++k)
            for (int j = 0; j <= ny; ++j)
                for (int i = 0; i <= nx; ++i) {
                    if (ux3(g, k, j, i)) X3(tx, k, j, i) = jx3(g, vx, vy, vz, bx, omega, k, j, i);
                    if (uy3(g, k, j, i)) Y3(ty, k, j, i) = jy3(g, vx, vy, vz, by, omega, k, j, i);
                    if (uz3(g, k, j, i)) Z3(tz, k, j, i) = jz3(g, vx, vy, vz, bz, omega, k, j, i);
                }
        memcpy(vx, tx, n_vx(g) * sizeof(double));
        memcpy(vy, ty, n_vy(g) * sizeof(double));
        memcpy(vz, tz, n_vz(g) * sizeof(double));
    }
    free(tx); free(ty); free(tz);
}

/* SplitMix64 (Steele, Lea & Flood 2014): output c (from 0) of the generator seeded with `seed` */
static uint64_t sm64(uint64_t seed, uint64_t c)
{
    uint64_t z = seed + (c + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* cut [0, n) at s + m T; returns the number of intervals, cut points in cuts */
static int cuts3(int n, int T, int s, int *cuts)
{
    int m = 0;
    cuts[m++] = 0;
    for (int c = s; c < n; c += T)
        if (c > 0) cuts[m++] = c;
    cuts[m++] = n;
    return m - 1;
}

/* The shift (si, sj, sk) RAS draws for outer iteration t. mode 0: none;
 * 1: SplitMix64 draws 3t, 3t+1, 3t+2; 2: the list shifts[3t .. 3t+2]. */
void o3_ras_shift(int mode, uint64_t seed, const int *shifts, int t, int ti, int tj, int tk, int *out)
{
    if (mode == 1) {
        out[0] = (int)(sm64(seed, 3u * (uint64_t)t) % (uint64_t)ti);
        out[1] = (int)(sm64(seed, 3u * (uint64_t)t + 1u) % (uint64_t)tj);
        out[2] = (int)(sm64(seed, 3u * (uint64_t)t + 2u) % (uint64_t)tk);
    } else if (mode == 2) {
        out[0] = shifts[3 * t];
        out[1] = shifts[3 * t + 1];
        out[2] = shifts[3 * t + 2];
    } else {
        out[0] = out[1] = out[2] = 0;
    }
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* RAS-Jacobi on 3D tiles (Algorithm 2 in 3D): ceil(sweeps/k) outer
 * iterations; in each, every tile runs kk local Jacobi sweeps on its cells
 * grown by `overlap` (clipped), everything else frozen at the snapshot, and
 * writes the unknowns of its own cells.  order_seed != 0 shuffles the order
 * the tiles run in (the result must not depend on it).  counts (optional:
 * vx, vy, vz natural layouts back to back) receives, for the last outer
 * iteration, how many tiles wrote each unknown.  Returns 0, -1 on bad input. */
int o3_ras(HEAD3, const double *bx, const double *by, const double *bz, double omega, int sweeps, int ti, int tj,
           int tk, int k, int overlap, int shift_mode, uint64_t seed, const int *shifts, uint64_t order_seed,
           double *vx, double *vy, double *vz, int *counts)
{
    if (nx < 1 || ny < 1 || nz < 1 || ti < 1 || tj < 1 || tk < 1 || k < 1 || overlap < 0 || sweeps < 0) return -1;
    MK3;
    const size_t nX = n_vx(g), nY = n_vy(g), nZ = n_vz(g);
    double *sx = malloc(nX * sizeof(double)), *sy = malloc(nY * sizeof(double)), *sz = malloc(nZ * sizeof(double));
    double *wx = malloc(nX * sizeof(double)), *wy = malloc(nY * sizeof(double)), *wz = malloc(nZ * sizeof(double));
    double *tx = malloc(nX * sizeof(double)), *ty = malloc(nY * sizeof(double)), *tz = malloc(nZ * sizeof(double));
    int *cx = malloc((size_t)(nx / ti + 3) * sizeof(int)), *cy = malloc((size_t)(ny / tj + 3) * sizeof(int));
    int *cz = malloc((size_t)(nz / tk + 3) * sizeof(int));
    const int n_outer = (sweeps + k - 1) / k;
    for (int t = 0; t < n_outer; ++t) {
        const int kk = (t == n_outer - 1) ? sweeps - (n_outer - 1) * k : k;
        int sh[3];
        o3_ras_shift(shift_mode, seed, shifts, t, ti, tj, tk, sh);
        const int ntx = cuts3(nx, ti, sh[0], cx), nty = cuts3(ny, tj, sh[1], cy), ntz = cuts3(nz, tk, sh[2], cz);
        const int ntiles = ntx * nty * ntz;
        int *order = malloc((size_t)ntiles * sizeof(int));
        for (int q = 0; q < ntiles; ++q) order[q] = q;
        if (order_seed)
            for (int q = ntiles - 1; q > 0; --q) {
                int r = (int)(sm64(order_seed, (uint64_t)q) % (uint64_t)(q + 1));
                int tmp = order[q]; order[q] = order[r]; order[r] = tmp;
            }
        memcpy(sx, vx, nX * sizeof(double));
        memcpy(sy, vy, nY * sizeof(double));
        memcpy(sz, vz, nZ * sizeof(double));
        memcpy(wx, vx, nX * sizeof(double));
        memcpy(wy, vy, nY * sizeof(double));
        memcpy(wz, vz, nZ * sizeof(double));
        memcpy(tx, vx, nX * sizeof(double));
        memcpy(ty, vy, nY * sizeof(double));
        memcpy(tz, vz, nZ * sizeof(double));
        if (counts && t == n_outer - 1) memset(counts, 0, (nX + nY + nZ) * sizeof(int));
        for (int q = 0; q < ntiles; ++q) {
            const int id = order[q];
            const int a = id % ntx, b = (id / ntx) % nty, c = id / (ntx * nty);
            const int x0 = cx[a], x1 = cx[a + 1], y0 = cy[b], y1 = cy[b + 1], z0 = cz[c], z1 = cz[c + 1];
            const int lx0 = clampi(x0 - overlap, 0, nx), lx1 = clampi(x1 + overlap, 0, nx);
            const int ly0 = clampi(y0 - overlap, 0, ny), ly1 = clampi(y1 + overlap, 0, ny);
            const int lz0 = clampi(z0 - overlap, 0, nz), lz1 = clampi(z1 + overlap, 0, nz);
            for (int s = 0; s < kk; ++s) {
                for (int kz = lz0; kz < lz1; ++kz)
                    for (int j = ly0; j < ly1; ++j)
                        for (int i = lx0; i < lx1; ++i) {
                            if (ux3(g, kz, j, i)) X3(tx, kz, j, i) = jx3(g, wx, wy, wz, bx, omega, kz, j, i);
                            if (uy3(g, kz, j, i)) Y3(ty, kz, j, i) = jy3(g, wx, wy, wz, by, omega, kz, j, i);
                            if (uz3(g, kz, j, i)) Z3(tz, kz, j, i) = jz3(g, wx, wy, wz, bz, omega, kz, j, i);
                        }
                for (int kz = lz0; kz < lz1; ++kz)
                    for (int j = ly0; j < ly1; ++j)
                        for (int i = lx0; i < lx1; ++i) {
                            if (ux3(g, kz, j, i)) X3(wx, kz, j, i) = X3(tx, kz, j, i);
                            if (uy3(g, kz, j, i)) Y3(wy, kz, j, i) = Y3(ty, kz, j, i);
                            if (uz3(g, kz, j, i)) Z3(wz, kz, j, i) = Z3(tz, kz, j, i);
                        }
            }
            for (int kz = z0; kz < z1; ++kz)
                for (int j = y0; j < y1; ++j)
                    for (int i = x0; i < x1; ++i) {
                        if (ux3(g, kz, j, i)) {
                            X3(vx, kz, j, i) = X3(wx, kz, j, i);
                            if (counts && t == n_outer - 1) X3(counts, kz, j, i) += 1;
                        }
                        if (uy3(g, kz, j, i)) {
                            Y3(vy, kz, j, i) = Y3(wy, kz, j, i);
                            if (counts && t == n_outer - 1) Y3((counts + nX), kz, j, i) += 1;
                        }
                        if (uz3(g, kz, j, i)) {
                            Z3(vz, kz, j, i) = Z3(wz, kz, j, i);
                            if (counts && t == n_outer - 1) Z3((counts + nX + nY), kz, j, i) += 1;
                        }
                    }
            /* restore the snapshot in the local region */
            for (int kz = lz0; kz < lz1; ++kz)
                for (int j = ly0; j < ly1; ++j)
                    for (int i = lx0; i < lx1; ++i) {
                        if (ux3(g, kz, j, i)) X3(wx, kz, j, i) = X3(tx, kz, j, i) = X3(sx, kz, j, i);
                        if (uy3(g, kz, j, i)) Y3(wy, kz, j, i) = Y3(ty, kz, j, i) = Y3(sy, kz, j, i);
                        if (uz3(g, kz, j, i)) Z3(wz, kz, j, i) = Z3(tz, kz, j, i) = Z3(sz, kz, j, i);
                    }
        }
        free(order);
    }
    free(sx); free(sy); free(sz); free(wx); free(wy); free(wz); free(tx); free(ty); free(tz);
    free(cx); free(cy); free(cz);
    return 0;
}

/* Energy sums (Sec. 6.4 over three components): out[0] = sum r_v^2/(-diag M),
 * out[1] = sum (D v)^2 eta_c / (2/hx^2 + 2/hy^2 + 2/hz^2), out[2] = sum f^2/(-diag M);
 * r_v = f - G p - M v (p may be NULL). */
void o3_energy(HEAD3, const double *fx, const double *fy, const double *fz, const double *p, const double *vx,
               const double *vy, const double *vz, double *out)
{
    MK3;
    double *bx = malloc(n_vx(g) * sizeof(double)), *by = malloc(n_vy(g) * sizeof(double));
    double *bz = malloc(n_vz(g) * sizeof(double));
    o3_rhs(nx, ny, nz, hx, hy, hz, fx, fy, fz, p, bx, by, bz);
    double rv = 0.0, rp = 0.0, ff = 0.0;
    for (int k = 0; k <= nz; ++k)
        for (int j = 0; j <= ny; ++j)
            for (int i = 0; i <= nx; ++i) {
                if (ux3(g, k, j, i)) {
                    double w = -dx3(g, k, j, i), r = X3(bx, k, j, i) - mx3(g, vx, vy, vz, k, j, i);
                    rv += r * r / w;
                    ff += X3(fx, k, j, i) * X3(fx, k, j, i) / w;
                }
                if (uy3(g, k, j, i)) {
                    double w = -dy3(g, k, j, i), r = Y3(by, k, j, i) - my3(g, vx, vy, vz, k, j, i);
                    rv += r * r / w;
                    ff += Y3(fy, k, j, i) * Y3(fy, k, j, i) / w;
                }
                if (uz3(g, k, j, i)) {
                    double w = -dz3(g, k, j, i), r = Z3(bz, k, j, i) - mz3(g, vx, vy, vz, k, j, i);
                    rv += r * r / w;
                    ff += Z3(fz, k, j, i) * Z3(fz, k, j, i) / w;
                }
            }
    const double lap = 2.0 / (hx * hx) + 2.0 / (hy * hy) + 2.0 / (hz * hz);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double d = (X3(vx, k, j, i + 1) - X3(vx, k, j, i)) / hx + (Y3(vy, k, j + 1, i) - Y3(vy, k, j, i)) / hy
                           + (Z3(vz, k + 1, j, i) - Z3(vz, k, j, i)) / hz;
                rp += d * d * C3(g->ec, k, j, i) / lap;
            }
    out[0] = rv;
    out[1] = rp;
    out[2] = ff;
    free(bx); free(by); free(bz);
}
