// General-mesh input on the host: the SPDE precision matrices of a triangulation as CSR.
//
// Piecewise-linear finite elements with natural (Neumann) boundary: lumped mass
// C~ = diag(c), c_i = a third of the area of every triangle at vertex i; stiffness
// G_ij = sum over triangles T of |T| grad(phi_i) . grad(phi_j).  On a triangle with edge
// vectors e_i opposite vertex i, grad(phi_i) is e_i turned by 90 degrees over 2|T|, so the
// element stiffness is e_i . e_j / (4 |T|).  The model tau (kappa^2 - Laplacian) of Sec. 3
// (with kappa^2 for the paper's kappa) gives
//     Q = tau (kappa^2 C~ + G)                      first order,
//     Q = tau K C~^{-1} K,   K = kappa^2 C~ + G     second order (Matern alpha = 2).
// Rows come out with sorted column indices; entries that sum to exactly zero are dropped
// (on right triangles the coupling across the hypotenuse vanishes).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "internal.h"

namespace ld {

namespace {

// CSR with sorted rows, built from per-row (column, value) lists
struct Rows {
    std::vector<std::vector<std::pair<int64_t, double>>> r;
    explicit Rows(int64_t n) : r((size_t)n) {}
    void add(int64_t i, int64_t j, double v) { r[(size_t)i].emplace_back(j, v); }
    // merge duplicates in place (sum), sort by column, drop exact zeros
    void compress() {
        for (auto &row : r) {
            std::sort(row.begin(), row.end(),
                      [](const std::pair<int64_t, double> &a, const std::pair<int64_t, double> &b) {
                          return a.first < b.first;
                      });
            size_t o = 0;
            for (size_t k = 0; k < row.size();) {
                const int64_t j = row[k].first;
                double s = 0.0;
                while (k < row.size() && row[k].first == j) s += row[k++].second;
                if (s != 0.0) row[o++] = {j, s};
            }
            row.resize(o);
        }
    }
};

}  // namespace

int fem_spde(int64_t n, const double *xy, int64_t m, const int64_t *tri, double kappa2, int alpha,
             double tau, std::vector<int64_t> &rowptr, std::vector<int32_t> &colidx,
             std::vector<double> &val) {
    std::vector<double> c((size_t)n, 0.0);
    Rows K(n);
    for (int64_t t = 0; t < m; ++t) {
        const int64_t v[3] = {tri[3 * t], tri[3 * t + 1], tri[3 * t + 2]};
        for (int k = 0; k < 3; ++k)
            if (v[k] < 0 || v[k] >= n) return -1;
        double e[3][2];
        for (int k = 0; k < 3; ++k) {   // e_k = p_{k+2} - p_{k+1}, opposite vertex k
            const int64_t a = v[(k + 1) % 3], b = v[(k + 2) % 3];
            e[k][0] = xy[2 * b] - xy[2 * a];
            e[k][1] = xy[2 * b + 1] - xy[2 * a + 1];
        }
        // twice the signed area: cross(p1 - p0, p2 - p0) = cross(e_2, -e_1)
        const double area2 = e[2][0] * (-e[1][1]) - e[2][1] * (-e[1][0]);
        if (!(area2 != 0.0) || !std::isfinite(area2)) return -2;
        const double area = 0.5 * std::fabs(area2);
        for (int i = 0; i < 3; ++i) {
            c[(size_t)v[i]] += area / 3.0;
            for (int j = 0; j < 3; ++j)
                K.add(v[i], v[j], (e[i][0] * e[j][0] + e[i][1] * e[j][1]) / (4.0 * area));
        }
    }
    for (int64_t i = 0; i < n; ++i) {
        if (!(c[(size_t)i] > 0.0)) return -3;   // a vertex in no triangle
        K.add(i, i, kappa2 * c[(size_t)i]);
    }
    K.compress();
    Rows Q(n);
    if (alpha == 1) {
        for (int64_t i = 0; i < n; ++i)
            for (const auto &q : K.r[(size_t)i]) Q.add(i, q.first, tau * q.second);
    } else {
        // row i of K C~^{-1} K: sum over k in row i of K of (K_ik / c_k) * row k of K,
        // accumulated in a dense scratch row with a list of touched columns
        std::vector<double> acc((size_t)n, 0.0);
        std::vector<char> hit((size_t)n, 0);
        std::vector<int64_t> cols;
        for (int64_t i = 0; i < n; ++i) {
            cols.clear();
            for (const auto &ik : K.r[(size_t)i]) {
                const double s = ik.second / c[(size_t)ik.first];
                for (const auto &kj : K.r[(size_t)ik.first]) {
                    if (!hit[(size_t)kj.first]) {
                        hit[(size_t)kj.first] = 1;
                        cols.push_back(kj.first);
                    }
                    acc[(size_t)kj.first] += s * kj.second;
                }
            }
            for (int64_t j : cols) {
                Q.add(i, j, tau * acc[(size_t)j]);
                acc[(size_t)j] = 0.0;
                hit[(size_t)j] = 0;
            }
        }
    }
    Q.compress();
    rowptr.assign((size_t)n + 1, 0);
    for (int64_t i = 0; i < n; ++i) rowptr[(size_t)i + 1] = rowptr[(size_t)i] + (int64_t)Q.r[(size_t)i].size();
    const int64_t nnz = rowptr[(size_t)n];
    colidx.resize((size_t)nnz);
    val.resize((size_t)nnz);
    for (int64_t i = 0; i < n; ++i) {
        int64_t o = rowptr[(size_t)i];
        for (const auto &q : Q.r[(size_t)i]) {
            colidx[(size_t)o] = (int32_t)q.first;
            val[(size_t)o] = q.second;
            ++o;
        }
    }
    return 0;
}

}  // namespace ld
