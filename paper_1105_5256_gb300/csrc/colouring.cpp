// Probing-vector colourings (Sec. 2.1).
//
// The probing vectors are the indicator vectors of the colour classes of a
// distance-d colouring of the graph of Q: any two vertices joined by a path of
// at most d edges get different colours (equivalently a neighbour colouring of
// the graph of Q^d).  The colouring is greedy in natural vertex order: vertex i
// takes the smallest colour not used by an already coloured vertex within
// distance d.  Colourings depend only on the sparsity pattern, so a context
// computes one at creation and keeps it (Sec. 3 stores colourings for reuse).
//
// Grid kinds avoid a graph search: on the lattice the graph distance is the
// (torus) L1 distance for the 5- and 7-point stencils and ceil(L1 / 2) for the
// 13-point square, so the distance-d ball is a fixed set of lattice offsets.
#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <vector>

#include "internal.h"

namespace ld {

int colour_csr(int64_t n, const int64_t *rowptr, const int32_t *colidx, int d,
               int32_t *colour) {
    std::vector<int64_t> seen(n, -1), frontier, next;
    std::vector<int64_t> used;  // used[c] == i  <=> colour c taken near vertex i
    int ncol = 0;
    for (int64_t i = 0; i < n; ++i) colour[i] = -1;
    for (int64_t i = 0; i < n; ++i) {
        frontier.assign(1, i);
        seen[i] = i;
        for (int depth = 0; depth < d && !frontier.empty(); ++depth) {
            next.clear();
            for (int64_t u : frontier) {
                for (int64_t e = rowptr[u]; e < rowptr[u + 1]; ++e) {
                    int64_t w = colidx[e];
                    if (seen[w] == i) continue;
                    seen[w] = i;
                    next.push_back(w);
                    int32_t cw = colour[w];
                    if (cw >= 0) {
                        if ((size_t)cw >= used.size()) used.resize((size_t)cw + 1, -1);
                        used[cw] = i;
                    }
                }
            }
            frontier.swap(next);
        }
        int32_t c = 0;
        while ((size_t)c < used.size() && used[c] == i) ++c;
        colour[i] = c;
        ncol = std::max(ncol, c + 1);
    }
    return ncol;
}

int colour_grid(int kind, const int32_t dims[3], int periodic, int d, int32_t *colour) {
    const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    const int R = (kind == KIND_2D13_SQ) ? 2 * d : d;   // L1 radius of the ball
    const bool is3d = (kind == KIND_3D7);
    struct Off { int dx, dy, dz; };
    std::vector<Off> offs;
    for (int dz = is3d ? -R : 0; dz <= (is3d ? R : 0); ++dz)
        for (int dy = -R; dy <= R; ++dy)
            for (int dx = -R; dx <= R; ++dx) {
                if (std::abs(dx) + std::abs(dy) + std::abs(dz) > R) continue;
                if (dx == 0 && dy == 0 && dz == 0) continue;
                if (!periodic) {
                    // only offsets that can reach an earlier vertex in natural order
                    bool earlier = dz < 0 || (dz == 0 && (dy < 0 || (dy == 0 && dx < 0)));
                    if (!earlier) continue;
                }
                offs.push_back({dx, dy, dz});
            }
    const int64_t n = nx * ny * nz;
    // Vertices whose ball needs no bounds or wrap logic take a fast path: their coloured
    // neighbours are i + back[k], the same set the general path finds.  Without wrap the
    // earlier half-ball must lie inside the grid; on a torus the whole ball must (a later
    // offset that wraps lands on an earlier vertex).
    std::vector<int64_t> back;
    for (const Off &o : offs)
        if (o.dz < 0 || (o.dz == 0 && (o.dy < 0 || (o.dy == 0 && o.dx < 0))))
            back.push_back(o.dx + nx * (o.dy + ny * (int64_t)o.dz));
    std::vector<int64_t> used;
    int ncol = 0;
    for (int64_t i = 0; i < n; ++i) colour[i] = -1;
    int64_t i = 0;
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x, ++i) {
                bool inside = x >= R && x + R < nx && y >= R;
                if (is3d) inside = inside && y + R < ny && z >= R;
                if (periodic) inside = inside && y + R < ny && (!is3d || z + R < nz);
                if (inside) {
                    for (const int64_t dj : back) {
                        const int32_t cj = colour[i + dj];
                        if ((size_t)cj >= used.size()) used.resize((size_t)cj + 1, -1);
                        used[cj] = i;
                    }
                    int32_t c = 0;
                    while ((size_t)c < used.size() && used[c] == i) ++c;
                    colour[i] = c;
                    ncol = std::max(ncol, c + 1);
                    continue;
                }
                for (const Off &o : offs) {
                    int64_t xx = x + o.dx, yy = y + o.dy, zz = z + o.dz;
                    if (periodic) {
                        xx = ((xx % nx) + nx) % nx;
                        yy = ((yy % ny) + ny) % ny;
                        zz = ((zz % nz) + nz) % nz;
                    } else if (xx < 0 || xx >= nx || yy < 0 || yy >= ny || zz < 0 || zz >= nz) {
                        continue;
                    }
                    int64_t j = xx + nx * (yy + ny * zz);
                    if (j >= i) continue;   // not yet coloured (or the vertex itself)
                    int32_t cj = colour[j];
                    if ((size_t)cj >= used.size()) used.resize((size_t)cj + 1, -1);
                    used[cj] = i;
                }
                int32_t c = 0;
                while ((size_t)c < used.size() && used[c] == i) ++c;
                colour[i] = c;
                ncol = std::max(ncol, c + 1);
            }
    return ncol;
}

// Graph distances from vertex j in the graph of Q, -1 beyond max_d.  Grid kinds use
// the lattice distance (as for the colouring); CSR a breadth-first search.
void graph_distances(int kind, const int32_t dims[3], int periodic, int64_t n, const int64_t *rowptr,
                     const int32_t *colidx, int64_t j, int max_d, int32_t *dist) {
    for (int64_t i = 0; i < n; ++i) dist[i] = -1;
    if (kind == KIND_CSR) {
        std::vector<int64_t> frontier(1, j), next;
        dist[j] = 0;
        for (int d = 1; d <= max_d && !frontier.empty(); ++d) {
            next.clear();
            for (int64_t u : frontier)
                for (int64_t e = rowptr[u]; e < rowptr[u + 1]; ++e) {
                    const int64_t w = colidx[e];
                    if (dist[w] < 0) {
                        dist[w] = d;
                        next.push_back(w);
                    }
                }
            frontier.swap(next);
        }
        return;
    }
    const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    const int64_t jx = j % nx, jy = (j / nx) % ny, jz = j / (nx * ny);
    auto axis = [&](int64_t a, int64_t b, int64_t len) {
        int64_t dd = a > b ? a - b : b - a;
        if (periodic && len - dd < dd) dd = len - dd;
        return dd;
    };
    int64_t i = 0;
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x, ++i) {
                int64_t l1 = axis(x, jx, nx) + axis(y, jy, ny) + axis(z, jz, nz);
                const int64_t d = kind == KIND_2D13_SQ ? (l1 + 1) / 2 : l1;
                if (d <= max_d) dist[i] = (int32_t)d;
            }
}

}  // namespace ld
