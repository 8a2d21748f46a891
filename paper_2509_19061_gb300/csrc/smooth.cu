// smooth.cu -- schedules of the five smoothers of Sec. 5 over the kernels:
// sweep loops, RAS outer iterations with their tile shifts (Algorithm 2),
// and the ping-pong between the caller's velocity and a scratch pair.
#include "../../include/stokes.h"
#include "internal.h"

namespace stokes {

// number of ping-pong passes of a smoothing (one per sweep; one per outer
// iteration of RAS)
int smooth_passes(const SmoothSpec &p)
{
    if (p.sweeps <= 0) return 0;
    if (p.variant == STOKES_RAS) return (p.sweeps + p.k - 1) / p.k;
    return p.sweeps;
}

template <typename T>
int smooth_buffers(const GridDesc<T> &g, const Coeffs<T> &k, T *vx, T *vy, T *sx, T *sy, const SmoothSpec &p,
                   const RasRun &run, cudaStream_t s, LaunchHook &hook, bool *swapped, T *tx, T *ty)
{
    if (swapped) *swapped = false;
    const T omega = (T)p.omega;
    int st = STOKES_OK;
#define LAUNCH(kind, nk, expr)                                                                                     \
    do {                                                                                                           \
        st = hook.run((kind), (nk), [&]() { return (expr); });                                                     \
        if (st != STOKES_OK) return st;                                                                            \
    } while (0)
    if (p.sweeps == 0) return STOKES_OK;
    // ping-pong between (vx, vy) and the scratch pair; the scratch walls take
    // the Dirichlet values of (vx, vy).  With a second scratch pair (tx, ty)
    // and an odd number n >= 3 of passes, pass 1 goes from (vx, vy) to (sx, sy),
    // passes 2 .. n-1 alternate between the two scratch pairs and pass n
    // writes (vx, vy): the result lands in place without a copy back.
    const int n_pass = smooth_passes(p);
    const bool three = tx && ty && !swapped && n_pass >= 3 && (n_pass & 1);
    T *ax = vx, *ay = vy, *bx = sx, *by = sy;
    LAUNCH(STOKES_K_COPY, 1, launch_copy_walls<T>(g, vx, vy, sx, sy, s));
    if (three) LAUNCH(STOKES_K_COPY, 1, launch_copy_walls<T>(g, vx, vy, tx, ty, s));
    int passes = 0;
    // after pass `passes` (1-based) wrote (bx, by): the source and target of the next
    auto advance = [&]() {
        T *nx_ = bx, *ny_ = by;
        if (!three) {
            bx = ax;
            by = ay;
        } else if (passes == n_pass - 1) {
            bx = vx;
            by = vy;
        } else {
            bx = (nx_ == sx) ? tx : sx;
            by = (ny_ == sy) ? ty : sy;
        }
        ax = nx_;
        ay = ny_;
    };
    if (p.variant == STOKES_RAS) {
        const int n_outer = (p.sweeps + p.k - 1) / p.k;
        for (int t = 0; t < n_outer; ++t) {
            const int ks = (t == n_outer - 1) ? p.sweeps - (n_outer - 1) * p.k : p.k;
            int si = 0, sj = 0;
            if (p.shift_mode == STOKES_SHIFT_SPLITMIX) {
                si = (int)(splitmix64(p.seed, 2u * (uint64_t)t) % (uint64_t)p.ti);
                sj = (int)(splitmix64(p.seed, 2u * (uint64_t)t + 1u) % (uint64_t)p.tj);
            } else if (p.shift_mode == STOKES_SHIFT_LIST) {
                si = p.shifts[2 * t];
                sj = p.shifts[2 * t + 1];
                if (si < 0 || si >= p.ti || sj < 0 || sj >= p.tj) return STOKES_ERR_ARG;
            }
            const TileGrid tg = make_tiles(g.nx, g.ny, p.ti, p.tj, si, sj);
            LAUNCH(STOKES_K_RAS, 1, launch_ras<T>(g, k, omega, tg, ks, p.overlap, ax, ay, bx, by, run, s));
            ++passes;
            advance();
        }
    } else {
        for (int it = 0; it < p.sweeps; ++it) {
            if (p.variant == STOKES_RBGS) {
                LAUNCH(STOKES_K_RBGS, 1, launch_rbgs_sweep<T>(g, k, omega, ax, ay, bx, by, s));
            } else if (p.variant == STOKES_JACOBI_BLOCKED) {
                const TileGrid tg = make_tiles(g.nx, g.ny, p.ti, p.tj, 0, 0);
                LAUNCH(STOKES_K_RAS, 1, launch_ras<T>(g, k, omega, tg, 1, 0, ax, ay, bx, by, run, s));
            } else {
                const int fused = p.variant == STOKES_JACOBI_FUSED;
                LAUNCH(STOKES_K_JACOBI, fused ? 1 : 2, launch_jacobi<T>(g, k, omega, ax, ay, bx, by, fused, s));
            }
            ++passes;
            advance();
        }
    }
    if ((passes & 1) && !three) {
        if (swapped)
            *swapped = true; // the result stays in (sx, sy); the caller swaps its pointers
        else
            LAUNCH(STOKES_K_COPY, 1, launch_copy_velocity<T>(g, ax, ay, vx, vy, s));
    }
#undef LAUNCH
    return STOKES_OK;
}

template int smooth_buffers<float>(const GridDesc<float> &, const Coeffs<float> &, float *, float *, float *,
                                   float *, const SmoothSpec &, const RasRun &, cudaStream_t, LaunchHook &, bool *,
                                   float *, float *);
template int smooth_buffers<double>(const GridDesc<double> &, const Coeffs<double> &, double *, double *, double *,
                                    double *, const SmoothSpec &, const RasRun &, cudaStream_t, LaunchHook &, bool *,
                                    double *, double *);

} // namespace stokes
