// Quadrature nodes of the rational approximation of log (Sec. 2.1, Eq. "eq_rat_app").
//
// log(Q) v = (1/2 pi i) oint log(z) (zI - Q)^{-1} v dz over a contour around the
// spectrum [m, M] that avoids (-inf, 0].  Following Hale, Higham & Trefethen's
// square-root construction: with z = w^2 the integrand becomes
// 4 w log(w) (w^2 I - Q)^{-1} v on a w-contour around [a, b] = [sqrt m, sqrt M];
// the rectangle [-K, K] x [0, K'] is mapped onto the upper half w-plane by
// u = sn(t | k^2), w = sqrt(ab)(1/k + u)/(1/k - u), k = (r-1)/(r+1), r = sqrt(b/a),
// and the midpoint rule on Im t = K'/2 with N points, plus the conjugate half,
// gives log(Q)v ~ Re sum_j alpha_j (Q - sigma_j I)^{-1} v with
//   sigma_j = w_j^2,  alpha_j = -(4 i h / pi) w_j log(w_j) w'(t_j),  h = 2K/N.
//
// Elliptic functions are computed here from their textbook definitions:
//   K(m) = pi / (2 AGM(1, sqrt(1-m)))                       (A&S 17.6)
//   sn, cn, dn of real argument by the descending AGM scale  (A&S 16.4)
//   complex argument x + iy by the addition formulas        (A&S 16.21)
#include <cmath>
#include <complex>
#include <vector>

#include "internal.h"

namespace ld {

static double agm(double a, double b) {
    for (int it = 0; it < 64; ++it) {
        double an = 0.5 * (a + b);
        double bn = std::sqrt(a * b);
        a = an;
        b = bn;
        if (std::fabs(a - b) <= 1e-17 * a) break;
    }
    return 0.5 * (a + b);
}

double ellip_k(double m) { return M_PI / (2.0 * agm(1.0, std::sqrt(1.0 - m))); }

// Jacobi sn, cn, dn of real u, parameter 0 <= m < 1, by the AGM scale (A&S 16.4.3).
void jacobi_real(double u, double m, double *sn, double *cn, double *dn) {
    if (m < 1e-300) {
        *sn = std::sin(u);
        *cn = std::cos(u);
        *dn = 1.0;
        return;
    }
    double a[40], c[40];
    a[0] = 1.0;
    double b = std::sqrt(1.0 - m);
    c[0] = std::sqrt(m);
    int N = 0;
    while (N < 38 && std::fabs(c[N]) > 1e-17) {
        double an = 0.5 * (a[N] + b);
        double cn_ = 0.5 * (a[N] - b);
        b = std::sqrt(a[N] * b);
        ++N;
        a[N] = an;
        c[N] = cn_;
    }
    double phi = std::ldexp(a[N] * u, N);
    for (int i = N; i >= 1; --i) phi = 0.5 * (phi + std::asin(c[i] * std::sin(phi) / a[i]));
    double s = std::sin(phi);
    *sn = s;
    *cn = std::cos(phi);
    *dn = std::sqrt(1.0 - m * s * s);
}

// sn, cn, dn at x + i y (A&S 16.21.1-4).
static void jacobi_complex(double x, double y, double m, std::complex<double> *sn,
                           std::complex<double> *cn, std::complex<double> *dn) {
    double s, c, d, s1, c1, d1;
    jacobi_real(x, m, &s, &c, &d);
    jacobi_real(y, 1.0 - m, &s1, &c1, &d1);
    double den = c1 * c1 + m * s * s * s1 * s1;
    *sn = std::complex<double>(s * d1, c * d * s1 * c1) / den;
    *cn = std::complex<double>(c * c1, -s * d * s1 * d1) / den;
    *dn = std::complex<double>(d * c1 * d1, -m * s * c * s1) / den;
}

int hht_log_nodes(double lmin, double lmax, int N, std::complex<double> *sigma,
                  std::complex<double> *alpha) {
    if (!(lmin > 0.0) || !(lmax >= lmin) || N < 1) return -1;
    const double a = std::sqrt(lmin), b = std::sqrt(lmax);
    const double r = std::sqrt(b / a);
    const double k = (r - 1.0) / (r + 1.0);
    if (!(k > 0.0)) return -1;
    const double m = k * k;
    const double K = ellip_k(m);
    const double Kp = ellip_k(1.0 - m);
    const double h = 2.0 * K / N;
    const double g = std::sqrt(a * b);
    const std::complex<double> I(0.0, 1.0);
    for (int j = 0; j < N; ++j) {
        double x = -K + (j + 0.5) * h;
        std::complex<double> sn, cn, dn;
        jacobi_complex(x, 0.5 * Kp, m, &sn, &cn, &dn);
        std::complex<double> den = 1.0 / k - sn;
        std::complex<double> w = g * (1.0 / k + sn) / den;
        std::complex<double> dw = g * (2.0 / k) * cn * dn / (den * den);
        sigma[j] = w * w;
        alpha[j] = -(4.0 * h / M_PI) * I * w * std::log(w) * dw;
    }
    return 0;
}

// The same contour and nodes for f(z) = z^{-1/2}: after z = w^2 the integrand is
// 2 (w^2 I - Q)^{-1} (principal branch, Re w > 0), so
//   Q^{-1/2} v ~ Re sum_j beta_j (Q - sigma_j I)^{-1} v,  beta_j = -(2 i h / pi) w'(t_j).
int hht_invsqrt_nodes(double lmin, double lmax, int N, std::complex<double> *sigma,
                      std::complex<double> *beta) {
    if (!(lmin > 0.0) || !(lmax >= lmin) || N < 1) return -1;
    const double a = std::sqrt(lmin), b = std::sqrt(lmax);
    const double r = std::sqrt(b / a);
    const double k = (r - 1.0) / (r + 1.0);
    if (!(k > 0.0)) return -1;
    const double m = k * k;
    const double K = ellip_k(m);
    const double Kp = ellip_k(1.0 - m);
    const double h = 2.0 * K / N;
    const double g = std::sqrt(a * b);
    const std::complex<double> I(0.0, 1.0);
    for (int j = 0; j < N; ++j) {
        double x = -K + (j + 0.5) * h;
        std::complex<double> sn, cn, dn;
        jacobi_complex(x, 0.5 * Kp, m, &sn, &cn, &dn);
        std::complex<double> den = 1.0 / k - sn;
        std::complex<double> w = g * (1.0 / k + sn) / den;
        std::complex<double> dw = g * (2.0 / k) * cn * dn / (den * den);
        sigma[j] = w * w;
        beta[j] = -(2.0 * h / M_PI) * I * dw;
    }
    return 0;
}

double hht_certificate(double lmin, double lmax, int N, const std::complex<double> *sigma,
                       const std::complex<double> *alpha) {
    const int S = 2001;
    double worst = 0.0;
    const double l0 = std::log(lmin), l1 = std::log(lmax);
    for (int s = 0; s < S; ++s) {
        double lam = std::exp(l0 + (l1 - l0) * s / (S - 1));
        double f = 0.0;
        for (int j = 0; j < N; ++j) f += std::real(alpha[j] / (lam - sigma[j]));
        double e = std::fabs(f - std::log(lam));
        if (e > worst) worst = e;
    }
    return worst;
}

}  // namespace ld
