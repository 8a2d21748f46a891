// mg_point.cuh -- per-point arithmetic of the multigrid transfer operators,
// shared by the single-instance and the batched kernels.  Prolongation P:
// bilinear in the staggered coordinates, mirror ghosts for the tangential
// direction, zero walls; restriction R = P^T / 4 (gather form).
#pragma once
#include "internal.h"
#include "stencil.cuh"

namespace stokes {

// Weights of one fine index a in the cell-centred direction: fine point at
// coarse position (a - 1/2)/2, nearest coarse 3/4, next 1/4, mirrored at the
// walls (nc coarse cells).
__device__ __forceinline__ void w_cell(int a, int nc, int &A, int &B)
{
    A = a >> 1;
    B = (a & 1) ? A + 1 : A - 1;
    B = B < 0 ? 0 : (B > nc - 1 ? nc - 1 : B);
}

// fine += P coarse at fine point (j, i) (both components)
template <typename T>
__device__ __forceinline__ void prolong_point(int nfx, int nfy, int fp, int ncx, int ncy, int cp,
                                              const T *__restrict__ cx, const T *__restrict__ cy,
                                              T *__restrict__ fx, T *__restrict__ fy, int j, int i)
{
    const size_t q = (size_t)j * fp + i;
    const T c34 = T(0.75), c14 = T(0.25), c12 = T(0.5);
    if (j < nfy && i >= 1 && i <= nfx - 1) { // vx: cell-centred in y, node-centred in x
        int A, B;
        w_cell(j, ncy, A, B);
        T s = T(0);
        const int ys[2] = {A, B};
        const T wy[2] = {c34, c14};
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const T *row = cx + (size_t)ys[a] * cp;
            if ((i & 1) == 0) {
                s = r_add(s, r_mul(r_mul(wy[a], T(1)), row[i >> 1]));
            } else {
                s = r_add(s, r_mul(r_mul(wy[a], c12), row[i >> 1]));
                s = r_add(s, r_mul(r_mul(wy[a], c12), row[(i >> 1) + 1]));
            }
        }
        fx[q] = r_add(fx[q], s);
    }
    if (i < nfx && j >= 1 && j <= nfy - 1) { // vy: node-centred in y, cell-centred in x
        int A, B;
        w_cell(i, ncx, A, B);
        T s = T(0);
        const int nrow = (j & 1) ? 2 : 1;
        const int ys[2] = {j >> 1, (j >> 1) + 1};
        const T wy[2] = {(j & 1) ? c12 : T(1), c12};
        for (int a = 0; a < nrow; ++a) {
            const T *row = cy + (size_t)ys[a] * cp;
            s = r_add(s, r_mul(r_mul(wy[a], c34), row[A]));
            s = r_add(s, r_mul(r_mul(wy[a], c14), row[B]));
        }
        fy[q] = r_add(fy[q], s);
    }
}

// coarse b = P^T r / 4 at coarse point (J, I) (both components; zero off the
// coarse unknowns)
template <typename T>
__device__ __forceinline__ void restrict_point(int nfx, int nfy, int fp, int ncx, int ncy, int cp,
                                               const T *__restrict__ rx, const T *__restrict__ ry,
                                               T *__restrict__ bx, T *__restrict__ by, int J, int I)
{
    const size_t cq = (size_t)J * cp + I;
    const T c34 = T(0.75), c14 = T(0.25), c12 = T(0.5);
    if (J < ncy) { // vx
        T s = T(0);
        if (I >= 1 && I <= ncx - 1) {
            // fine rows (cell-centred in y) and their weights toward coarse row J
            int rows[4];
            T wr[4];
            int nr = 0;
            if (J >= 1) { rows[nr] = 2 * J - 1; wr[nr++] = c14; }
            rows[nr] = 2 * J; wr[nr++] = J == 0 ? T(1) : c34;
            rows[nr] = 2 * J + 1; wr[nr++] = J == ncy - 1 ? T(1) : c34;
            if (J + 1 <= ncy - 1) { rows[nr] = 2 * J + 2; wr[nr++] = c14; }
            for (int a = 0; a < nr; ++a) {
                const T *row = rx + (size_t)rows[a] * fp;
                s = r_add(s, r_mul(r_mul(wr[a], c12), row[2 * I - 1]));
                s = r_add(s, r_mul(wr[a], row[2 * I]));
                s = r_add(s, r_mul(r_mul(wr[a], c12), row[2 * I + 1]));
            }
            s = r_mul(c14, s);
        }
        bx[cq] = s;
    }
    if (I < ncx) { // vy
        T s = T(0);
        if (J >= 1 && J <= ncy - 1) {
            int cols[4];
            T wc[4];
            int nc = 0;
            if (I >= 1) { cols[nc] = 2 * I - 1; wc[nc++] = c14; }
            cols[nc] = 2 * I; wc[nc++] = I == 0 ? T(1) : c34;
            cols[nc] = 2 * I + 1; wc[nc++] = I == ncx - 1 ? T(1) : c34;
            if (I + 1 <= ncx - 1) { cols[nc] = 2 * I + 2; wc[nc++] = c14; }
            const int rows[3] = {2 * J - 1, 2 * J, 2 * J + 1};
            const T wr[3] = {c12, T(1), c12};
            for (int a = 0; a < 3; ++a) {
                const T *row = ry + (size_t)rows[a] * fp;
                for (int b = 0; b < nc; ++b) s = r_add(s, r_mul(r_mul(wr[a], wc[b]), row[cols[b]]));
            }
            s = r_mul(c14, s);
        }
        by[cq] = s;
    }
}

} // namespace stokes
