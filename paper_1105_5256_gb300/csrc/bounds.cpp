// Spectral interval of a general CSR matrix (the rational log of Sec. 2.1 needs an
// interval [m, M] enclosing the spectrum; grid kinds get exact bounds elsewhere).
//
//   M: Gershgorin, max_i sum_j |Q_ij|, a guaranteed upper bound;
//   m: half the smallest Ritz value theta of a Lanczos run (no reorthogonalisation, a
//      fixed +-1 start vector).  Ritz values lie inside the spectrum, so theta
//      over-estimates lambda_min until it converges, which takes about sqrt(cond)
//      steps (thousands for a second-order SPDE precision on a fine mesh).  The run
//      therefore continues until theta has stagnated: at a check after k >= 60 steps,
//      theta moved by less than 1e-3 relative since the check at or before k/2 (the
//      smallest Ritz value never increases with k, so a stalled value over the second
//      half of the run has converged, apart from a start vector blind to lambda_min's
//      eigenvector).  Past lambda_min's convergence finite-precision Lanczos only adds
//      copies of it, so steps beyond n are harmless.  Checks are spaced geometrically
//      (5 %).  A host-work budget of about 4e9 flop caps the steps (at least 300);
//      a run that ends unconverged reports failure instead of a guess.
// The extreme eigenvalue of the Lanczos tridiagonal comes from Sturm-sequence bisection.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "internal.h"

namespace ld {

// number of eigenvalues of the symmetric tridiagonal (a, b) below x (Sturm sequence)
static int sturm_count(const std::vector<double> &a, const std::vector<double> &b, double x) {
    int count = 0;
    double q = 1.0;
    for (size_t i = 0; i < a.size(); ++i) {
        const double bb = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
        q = (a[i] - x) - (i > 0 ? bb / q : 0.0);
        if (q == 0.0) q = -1e-300;
        if (q < 0.0) ++count;
    }
    return count;
}

// smallest eigenvalue of the symmetric tridiagonal (a, b) by bisection inside its
// Gershgorin interval
static double smallest_eig(const std::vector<double> &a, const std::vector<double> &b) {
    double lo = INFINITY, hi = -INFINITY;
    for (size_t i = 0; i < a.size(); ++i) {
        const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i < b.size() ? std::fabs(b[i]) : 0.0);
        lo = std::min(lo, a[i] - r);
        hi = std::max(hi, a[i] + r);
    }
    for (int it = 0; it < 300 && hi - lo > 1e-15 * std::max(std::fabs(hi), std::fabs(lo)); ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (sturm_count(a, b, mid) >= 1) hi = mid;
        else lo = mid;
    }
    return 0.5 * (lo + hi);
}

int csr_bounds(int64_t n, const int64_t *rowptr, const int32_t *colidx, const double *val, double scale,
               double *lmin, double *lmax, int *steps_out) {
    // Gershgorin upper bound
    double gmax = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) s += std::fabs(scale * val[e]);
        gmax = std::max(gmax, s);
    }
    // Lanczos from a fixed +-1 vector (SplitMix64 bits)
    std::vector<double> v(n), vp(n, 0.0), w(n);
    uint64_t st = 0x9e3779b97f4a7c15ull;
    for (int64_t i = 0; i < n; ++i) {
        st += 0x9e3779b97f4a7c15ull;
        uint64_t z = st;
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        z ^= z >> 31;
        v[i] = (z & 1) ? 1.0 : -1.0;
    }
    const double v0 = 1.0 / std::sqrt((double)n);
    for (double &x : v) x *= v0;
    const double nnz = (double)rowptr[n];
    const int64_t cap = std::max<int64_t>(300, (int64_t)(4e9 / (2.0 * nnz + 10.0 * (double)n)));
    std::vector<double> alpha, beta;
    std::vector<std::pair<int64_t, double>> hist;   // (steps, smallest Ritz value) at each check
    double b = 0.0, theta = 0.0;
    bool converged = false;
    int64_t next_check = 20, k = 0;
    while (k < cap) {
        for (int64_t i = 0; i < n; ++i) {
            double s = 0.0;
            for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) s += scale * val[e] * v[colidx[e]];
            w[i] = s;
        }
        double a = 0.0;
        for (int64_t i = 0; i < n; ++i) a += v[i] * w[i];
        for (int64_t i = 0; i < n; ++i) w[i] -= a * v[i] + b * vp[i];
        double nb = 0.0;
        for (int64_t i = 0; i < n; ++i) nb += w[i] * w[i];
        nb = std::sqrt(nb);
        alpha.push_back(a);
        ++k;
        const bool invariant = !(nb > 1e-14 * std::max(std::fabs(a), 1e-300));  // Krylov space closed
        if (k >= next_check || k == cap || invariant) {
            next_check = std::max(k + 10, (int64_t)(1.05 * (double)k));
            theta = smallest_eig(alpha, beta);
            double ref = NAN;
            for (const auto &h : hist)
                if (h.first <= k / 2) ref = h.second;
            hist.emplace_back(k, theta);
            if (invariant || (k >= 60 && ref == ref && theta >= (1.0 - 1e-3) * ref)) {
                converged = true;
                break;
            }
        }
        beta.push_back(nb);
        b = nb;
        for (int64_t i = 0; i < n; ++i) {
            vp[i] = v[i];
            v[i] = w[i] / nb;
        }
    }
    if (steps_out) *steps_out = (int)std::min<int64_t>(k, 1 << 30);
    if (!converged) return -2;
    if (!(theta > 0.0) || !(gmax > 0.0)) return -1;
    *lmin = 0.5 * theta;
    *lmax = std::max(gmax, 1.01 * *lmin);
    return 0;
}

}  // namespace ld
