/*
 * Oracle native routines -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously-correct FP64 CPU code used to check the CUDA path.
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load this library.  It shares no code with the CUDA library.
 *
 *   or_chol_band        banded Cholesky Q = L L^T in natural order (Sec. 2:
 *                       log det Q = 2 sum_j log l_jj), no reordering.
 *   or_logdet_from_chol 2 * sum log L_jj.
 *   or_lsolve_band      forward substitution with a banded lower factor.
 *   or_takahashi_diag   selected inverse Z = Q^{-1} inside the band of L
 *                       (Takahashi-Fagan-Chin recurrences), for exact
 *                       tr(Q^{-1} E) gradients.
 *   or_ldlt_band_z      complex-symmetric banded LDL^T (no pivoting) of
 *                       Q - sigma I, for the shifted systems of the rational
 *                       approximation (Sec. 2.1, Eq. "eq_rat_app").
 *   or_fwd_quadform_z   v^T (L D L^T)^{-1} v = sum_j y_j^2 / D_j, y = L^{-1} v
 *                       (bilinear form, no conjugation, as in COCG).
 *   or_colour_greedy    greedy distance-d colouring of the graph of Q in
 *                       natural vertex order, smallest free colour (Sec. 2.1,
 *                       probing vectors from a neighbour colouring of the
 *                       graph of Q^d).
 *
 * Band storage: lower band, column-major: entry (i, j), j <= i <= j+b, is at
 * A[j*(b+1) + (i-j)].
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define BAND(A, b, i, j) (A)[(int64_t)(j) * ((b) + 1) + ((i) - (j))]

static int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

/* In-place banded Cholesky (right-looking).  Returns 0 on success, or
 * j+1 when the pivot of column j is not positive (Q not SPD). */
int or_chol_band(int64_t n, int64_t b, double *A) {
    for (int64_t j = 0; j < n; ++j) {
        double d = BAND(A, b, j, j);
        if (!(d > 0.0)) return (int)(j + 1 > 0x7fffffff ? 0x7fffffff : j + 1);
        double l = sqrt(d);
        BAND(A, b, j, j) = l;
        int64_t last = imin64(j + b, n - 1);
        for (int64_t i = j + 1; i <= last; ++i) BAND(A, b, i, j) /= l;
        /* trailing update of columns k = j+1..last, rows i = k..last */
        for (int64_t k = j + 1; k <= last; ++k) {
            double lkj = BAND(A, b, k, j);
            if (lkj == 0.0) continue;
            for (int64_t i = k; i <= last; ++i)
                BAND(A, b, i, k) -= BAND(A, b, i, j) * lkj;
        }
    }
    return 0;
}

double or_logdet_from_chol(int64_t n, int64_t b, const double *L) {
    double s = 0.0;
    for (int64_t j = 0; j < n; ++j) s += log(BAND(L, b, j, j));
    return 2.0 * s;
}

/* Y <- L^{-1} Y for nrhs column-major right-hand sides of length n. */
void or_lsolve_band(int64_t n, int64_t b, const double *L, int64_t nrhs, double *Y) {
    for (int64_t r = 0; r < nrhs; ++r) {
        double *y = Y + r * n;
        for (int64_t j = 0; j < n; ++j) {
            double yj = y[j] / BAND(L, b, j, j);
            y[j] = yj;
            if (yj == 0.0) continue;
            int64_t last = imin64(j + b, n - 1);
            for (int64_t i = j + 1; i <= last; ++i) y[i] -= BAND(L, b, i, j) * yj;
        }
    }
}

/* Selected inverse: Z (same band storage) holds (Q^{-1})_{ij} for j <= i <= j+b.
 * From L^T Z = L^{-1}:  for i >= j,
 *   Z_ij = ( [i==j]/L_jj - sum_{k=j+1}^{j+b} L_kj Z_ki ) / L_jj,
 * evaluated for j = n-1 .. 0 and, within a column, i = last .. j.  */
void or_takahashi_diag(int64_t n, int64_t b, const double *L, double *Z) {
    memset(Z, 0, sizeof(double) * (size_t)((b + 1) * n));
    for (int64_t j = n - 1; j >= 0; --j) {
        double ljj = BAND(L, b, j, j);
        int64_t last = imin64(j + b, n - 1);
        for (int64_t i = last; i >= j; --i) {
            double s = 0.0;
            for (int64_t k = j + 1; k <= last; ++k) {
                /* Z_ki, symmetric: stored at (max(k,i), min(k,i)) */
                double zki = (k >= i) ? BAND(Z, b, k, i) : BAND(Z, b, i, k);
                s += BAND(L, b, k, j) * zki;
            }
            double rhs = (i == j ? 1.0 / ljj : 0.0) - s;
            BAND(Z, b, i, j) = rhs / ljj;
        }
    }
}

/* In-place complex-symmetric LDL^T without pivoting: on exit the diagonal
 * slot holds D_j and the strictly-lower band holds the unit-L multipliers.
 * Returns 0, or j+1 when D_j == 0. */
int or_ldlt_band_z(int64_t n, int64_t b, double complex *A) {
    for (int64_t j = 0; j < n; ++j) {
        double complex d = BAND(A, b, j, j);
        if (d == 0.0) return (int)(j + 1 > 0x7fffffff ? 0x7fffffff : j + 1);
        int64_t last = imin64(j + b, n - 1);
        /* trailing update uses the unscaled column a_ij: A_ik -= a_ij a_kj / d */
        for (int64_t k = j + 1; k <= last; ++k) {
            double complex akj = BAND(A, b, k, j);
            if (akj == 0.0) continue;
            double complex f = akj / d;
            for (int64_t i = k; i <= last; ++i)
                BAND(A, b, i, k) -= BAND(A, b, i, j) * f;
        }
        for (int64_t i = j + 1; i <= last; ++i) BAND(A, b, i, j) /= d;
    }
    return 0;
}

/* For each real right-hand side v (column-major, nrhs of them), return
 * q = v^T (L D L^T)^{-1} v = sum_j y_j^2 / D_j with y = L^{-1} v (unit L).
 * work: complex buffer of length n. */
void or_fwd_quadform_z(int64_t n, int64_t b, const double complex *F, int64_t nrhs,
                       const double *V, double complex *out, double complex *work) {
    for (int64_t r = 0; r < nrhs; ++r) {
        const double *v = V + r * n;
        for (int64_t j = 0; j < n; ++j) work[j] = v[j];
        double complex q = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double complex yj = work[j];
            if (yj != 0.0) {
                int64_t last = imin64(j + b, n - 1);
                for (int64_t i = j + 1; i <= last; ++i) work[i] -= BAND(F, b, i, j) * yj;
                q += yj * yj / BAND(F, b, j, j);
            }
        }
        out[r] = q;
    }
}

/* Greedy distance-d colouring in natural order.  The graph is the pattern of
 * the CSR matrix (diagonal entries ignored; pattern assumed symmetric).
 * Vertex i gets the smallest colour not used by any already-coloured vertex
 * at graph distance 1..d from i (breadth-first search limited to depth d).
 * Returns the number of colours, or -1 on allocation failure. */
int or_colour_greedy(int64_t n, const int64_t *rowptr, const int32_t *col, int d,
                     int32_t *colour) {
    int64_t *stamp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int32_t *depth = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t used_cap = 64;
    int64_t *used = (int64_t *)malloc(sizeof(int64_t) * (size_t)used_cap);
    if (!stamp || !queue || !depth || !used) {
        free(stamp); free(queue); free(depth); free(used);
        return -1;
    }
    for (int64_t i = 0; i < n; ++i) { stamp[i] = -1; colour[i] = -1; }
    for (int64_t i = 0; i < used_cap; ++i) used[i] = -1;
    int ncol = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t head = 0, tail = 0;
        queue[tail++] = i;
        stamp[i] = i;
        depth[i] = 0;
        while (head < tail) {
            int64_t u = queue[head++];
            if (depth[u] == d) continue;
            for (int64_t e = rowptr[u]; e < rowptr[u + 1]; ++e) {
                int64_t w = col[e];
                if (stamp[w] == i) continue;
                stamp[w] = i;
                depth[w] = depth[u] + 1;
                queue[tail++] = w;
                int32_t cw = colour[w];
                if (cw >= 0) {
                    if (cw >= used_cap) {
                        int64_t nc = used_cap;
                        while (nc <= cw) nc *= 2;
                        int64_t *nu = (int64_t *)realloc(used, sizeof(int64_t) * (size_t)nc);
                        if (!nu) { free(stamp); free(queue); free(depth); free(used); return -1; }
                        for (int64_t t = used_cap; t < nc; ++t) nu[t] = -1;
                        used = nu;
                        used_cap = nc;
                    }
                    used[cw] = i;
                }
            }
        }
        int32_t c = 0;
        while (c < used_cap && used[c] == i) ++c;
        colour[i] = c;
        if (c + 1 > ncol) ncol = c + 1;
    }
    free(stamp); free(queue); free(depth); free(used);
    return ncol;
}
