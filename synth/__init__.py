"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module only draws random numbers and lays out problem descriptions; it
holds none of the log-determinant method's arithmetic (no colouring, no
quadrature, no Krylov recurrence; the only assembly is the graph Laplacian of
a drawn edge list).  Every generator is a pure function of its seed, so the
oracle and the CUDA path see identical inputs.

The workloads mirror the spatial GMRF models the paper uses (the SPDE model
tau (kappa - Laplacian) u = W on regular grids, Sec. 3; the Gauss-linear
posterior precision Q_x + A^T Q_1 A, Sec. 1): regular 2D/3D lattices with a
5-, 13- or 7-point structure, scalar or spatially varying kappa^2 and a
random observation pattern.
"""
from __future__ import annotations

from dataclasses import dataclass
import numpy as np

KIND_CSR = 0
KIND_2D5 = 1
KIND_2D13_SQ = 2
KIND_3D7 = 3


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence(int(seed)))


def kappa2_draws(seed: int, count: int, lo: float = 0.01, hi: float = 1.0) -> np.ndarray:
    """kappa^2 drawn log-uniformly in [lo, hi]."""
    g = rng(seed)
    return np.exp(g.uniform(np.log(lo), np.log(hi), size=count))


def obs_mask(seed: int, n: int, frac: float = 0.1) -> np.ndarray:
    """uint8 mask with exactly round(frac*n) observed nodes, from a seeded permutation."""
    g = rng(seed)
    m = np.zeros(n, dtype=np.uint8)
    k = int(round(frac * n))
    m[g.permutation(n)[:k]] = 1
    return m


def _box_mean_same(z: np.ndarray, w: int) -> np.ndarray:
    """Truncated ('same'-size, renormalised by the in-grid count) w^d box mean."""
    h = w // 2
    out = z.astype(np.float64)
    for ax in range(z.ndim):
        n = out.shape[ax]
        c = np.cumsum(out, axis=ax)
        pad_shape = list(out.shape)
        pad_shape[ax] = 1
        c = np.concatenate([np.zeros(pad_shape), c], axis=ax)
        idx = np.arange(n)
        hi = np.minimum(idx + h + 1, n)
        lo = np.maximum(idx - h, 0)
        s = np.take(c, hi, axis=ax) - np.take(c, lo, axis=ax)
        cnt_shape = [1] * out.ndim
        cnt_shape[ax] = n
        out = s / (hi - lo).reshape(cnt_shape)
    return out


def log_kappa2_field(seed: int, dims, mean: float = -2.0, sd: float = 1.0, box: int = 5) -> np.ndarray:
    """Seeded smooth Gaussian field for log kappa^2(s).

    i.i.d. N(0,1) on the grid, smoothed by a truncated box mean of side `box`,
    standardised to empirical mean 0 / sd 1, then mean + sd*z.  Returned in
    natural (x fastest) order, flattened.  dims = (nx, ny[, nz]).
    """
    g = rng(seed)
    shape = tuple(int(d) for d in reversed(dims))  # (nz, ny, nx): x fastest
    z = g.standard_normal(shape)
    z = _box_mean_same(z, box)
    z = (z - z.mean()) / z.std()
    return (mean + sd * z).reshape(-1)


def kappa2_field(seed: int, dims, mean: float = -2.0, sd: float = 1.0, box: int = 5) -> np.ndarray:
    return np.exp(log_kappa2_field(seed, dims, mean, sd, box))


@dataclass(frozen=True)
class GridInstance:
    """One GMRF on a regular grid: Q = scale*(kappa2*I - Lap [+ tau*diag(mask)]) or its square."""
    kind: int
    dims: tuple
    kappa2: float
    periodic: bool = False
    tau: float = 0.0
    scale: float = 1.0
    distance: int = 2

    @property
    def n(self) -> int:
        n = 1
        for d in self.dims:
            n *= int(d)
        return n


def batch_instances(seed: int, count: int = 256, side_lo: int = 32, side_hi: int = 512):
    """Batch of independent 2D GMRFs of uneven size.

    Grid side uniform on {side_lo..side_hi}; stencil 5-point (probing distance 4)
    or 13-point Matern (distance 2) by a fair coin; kappa^2 log-uniform in
    [0.01, 1].
    """
    g = rng(seed)
    sides = g.integers(side_lo, side_hi + 1, size=count)
    coin = g.integers(0, 2, size=count)
    k2 = np.exp(g.uniform(np.log(0.01), np.log(1.0), size=count))
    out = []
    for s, c, k in zip(sides, coin, k2):
        kind = KIND_2D5 if c == 0 else KIND_2D13_SQ
        out.append(GridInstance(kind=kind, dims=(int(s), int(s)), kappa2=float(k),
                                distance=4 if kind == KIND_2D5 else 2))
    return out


def random_probe_block(seed: int, n: int, c: int, dtype=np.float64) -> np.ndarray:
    """Dense random block (n x c) for operator-level parity (SpMM)."""
    g = rng(seed)
    return g.standard_normal((n, c)).astype(dtype)


def rademacher_block(seed: int, n: int, s: int) -> np.ndarray:
    """n x s block of independent +-1 entries, each sign with probability 1/2 (the
    random vectors of the Hutchinson estimator, drawn here and passed in)."""
    g = rng(seed)
    return np.where(g.random((n, s)) < 0.5, -1.0, 1.0)


def random_sparse_spd_pattern(seed: int, n: int, avg_deg: int = 6):
    """Seeded irregular symmetric graph for general-CSR inputs.

    Returns (rows, cols, weights) of the strictly-lower edges of a random
    geometric-like graph (each vertex links to a few random near indices),
    with positive weights.  The caller turns it into a weighted graph
    Laplacian plus a diagonal shift, which is SPD.
    """
    g = rng(seed)
    rows, cols = [], []
    for i in range(1, n):
        k = int(g.integers(1, avg_deg // 2 + 2))
        span = max(1, min(i, 4 * avg_deg))
        js = np.unique(i - 1 - g.integers(0, span, size=k))
        js = js[js >= 0]
        rows.extend([i] * len(js))
        cols.extend(js.tolist())
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    w = g.uniform(0.5, 1.5, size=rows.size)
    return rows, cols, w


def torus_edges(nx: int, ny: int):
    """Unit-weight edges (i < j) of the nx x ny periodic 4-neighbour lattice, x fastest;
    with csr_from_edges(..., kappa2) this is kappa2 I - Lap on the torus as a CSR matrix."""
    idx = np.arange(nx * ny).reshape(ny, nx)
    right = np.stack([idx.ravel(), np.roll(idx, -1, axis=1).ravel()], axis=1)
    down = np.stack([idx.ravel(), np.roll(idx, -1, axis=0).ravel()], axis=1)
    e = np.concatenate([right, down])
    e = np.sort(e, axis=1)
    e = np.unique(e, axis=0)
    return e[:, 0], e[:, 1], np.ones(len(e))


def csr_from_edges(n: int, rows, cols, w, diag_shift) -> tuple:
    """Assemble CSR (int64 rowptr, int32 colidx, f64 val) of L_w + diag(diag_shift).

    L_w is the weighted graph Laplacian of the given edge list.  This is input
    construction for the general-CSR path, not part of the method.
    """
    diag_shift = np.broadcast_to(np.asarray(diag_shift, dtype=np.float64), (n,))
    deg = np.zeros(n)
    np.add.at(deg, rows, w)
    np.add.at(deg, cols, w)
    r = np.concatenate([rows, cols, np.arange(n)])
    c = np.concatenate([cols, rows, np.arange(n)])
    v = np.concatenate([-w, -w, deg + diag_shift])
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    # merge duplicates
    key = r * n + c
    uk, start = np.unique(key, return_index=True)
    vs = np.add.reduceat(v, start)
    rr = uk // n
    cc = uk % n
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rr + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr.astype(np.int64), cc.astype(np.int32), vs.astype(np.float64)


def perturbed_triangulation(seed: int, nx: int, ny: int, jitter: float = 0.15):
    """Seeded unstructured triangulation of the unit square (general-mesh input).

    Vertices start on the nx x ny lattice (x fastest, spacing 1/(nx-1), 1/(ny-1)).
    Interior vertices move by uniform(-jitter, jitter) lattice spacings in x and y;
    edge vertices move only along their edge and corners stay, so the domain is the
    unit square exactly.  Each cell is cut along one of its two diagonals by a fair
    coin.  jitter <= 0.15 keeps every triangle counter-clockwise and non-degenerate.
    Returns (points float64 n x 2, triangles int64 m x 3, counter-clockwise).
    """
    g = rng(seed)
    hx, hy = 1.0 / (nx - 1), 1.0 / (ny - 1)
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny))
    ix, iy = ix.ravel(), iy.ravel()
    dx = g.uniform(-jitter, jitter, size=ix.size) * hx
    dy = g.uniform(-jitter, jitter, size=ix.size) * hy
    dx[(ix == 0) | (ix == nx - 1)] = 0.0
    dy[(iy == 0) | (iy == ny - 1)] = 0.0
    pts = np.stack([ix * hx + dx, iy * hy + dy], axis=1)
    cx, cy = np.meshgrid(np.arange(nx - 1), np.arange(ny - 1))
    a = (cx + nx * cy).ravel()
    b, c, d = a + 1, a + nx, a + nx + 1          # a b on the lower row, c d above
    coin = g.integers(0, 2, size=a.size).astype(bool)
    t1 = np.where(coin[:, None], np.stack([a, b, d], 1), np.stack([a, b, c], 1))
    t2 = np.where(coin[:, None], np.stack([a, d, c], 1), np.stack([b, d, c], 1))
    return pts, np.concatenate([t1, t2]).astype(np.int64)
