// Spectral interval of a general CSR matrix (the rational log of Sec. 2.1 needs an
// interval [m, M] enclosing the spectrum; grid kinds get exact bounds elsewhere).
//
//   M: Gershgorin, max_i sum_j |Q_ij|, a guaranteed upper bound;
//   m: half the smallest Ritz value of a Lanczos run (at most 80 steps, no
//      reorthogonalisation, a fixed +-1 start vector).  Ritz values lie inside the
//      spectrum, so the smallest one over-estimates lambda_min; halving it guards
//      against a slowly converging lower end at the price of a slightly wider interval.
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

int csr_bounds(int64_t n, const int64_t *rowptr, const int32_t *colidx, const double *val, double scale,
               double *lmin, double *lmax) {
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
    std::vector<double> alpha, beta;
    const int steps = (int)std::min<int64_t>(n, 80);
    double b = 0.0;
    for (int j = 0; j < steps; ++j) {
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
        if (!(nb > 1e-14 * std::max(std::fabs(a), 1e-300)) || j + 1 == steps) break;
        beta.push_back(nb);
        b = nb;
        for (int64_t i = 0; i < n; ++i) {
            vp[i] = v[i];
            v[i] = w[i] / nb;
        }
    }
    // smallest eigenvalue of the tridiagonal by bisection inside its Gershgorin interval
    double lo = INFINITY, hi = -INFINITY;
    for (size_t i = 0; i < alpha.size(); ++i) {
        const double r = (i > 0 ? std::fabs(beta[i - 1]) : 0.0) + (i < beta.size() ? std::fabs(beta[i]) : 0.0);
        lo = std::min(lo, alpha[i] - r);
        hi = std::max(hi, alpha[i] + r);
    }
    for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(std::fabs(hi), 1e-300); ++it) {
        const double mid = 0.5 * (lo + hi);
        if (sturm_count(alpha, beta, mid) >= 1) hi = mid;
        else lo = mid;
    }
    const double theta = 0.5 * (lo + hi);
    if (!(theta > 0.0) || !(gmax > 0.0)) return -1;
    *lmin = 0.5 * theta;
    *lmax = std::max(gmax, 1.01 * *lmin);
    return 0;
}

}  // namespace ld
