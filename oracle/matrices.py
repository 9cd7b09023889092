"""Oracle: the precision matrices Q as explicit sparse matrices (test infrastructure).

The models are the paper's SPDE prior tau (kappa - Laplacian) u = W discretised
on a regular grid (Sec. 3), its Matern alpha=2 square, a spatially varying
kappa^2, and the Gauss-linear posterior precision Q_p = Q_x + A^T Q_1 A with
A observing a subset of nodes and Q_1 = tau I (Sec. 1).

Construction is by Kronecker sums of 1D second-difference matrices and by a
sparse matrix product for the square -- deliberately nothing like the CUDA
path's hand-expanded stencil coefficients.

Readings (the paper leaves these open):
  * natural order: vertex index = x + nx*(y + ny*z);
  * non-periodic boundary = Dirichlet truncation (out-of-grid neighbours
    dropped, diagonal kept at kappa^2 + 2*dim), which keeps Q an SPD
    M-matrix with a sine-transform eigenbasis;
  * the 13-point Matern precision is the exact product Q1 @ Q1 of the
    truncated 5-point Q1 = kappa^2 I - Laplacian;
  * the prior scale multiplies the whole matrix.

General meshes (the SPDE route the paper cites for sparse precisions, Sec. 1):
piecewise-linear finite elements on a triangulation, natural (Neumann)
boundary, lumped mass C~ (each triangle gives a third of its area to each of
its vertices), stiffness G_ij = integral of grad(phi_i) . grad(phi_j);
Q = tau (kappa^2 C~ + G) for the first-order model and
Q = tau K C~^{-1} K with K = kappa^2 C~ + G for the second-order one.  The
hat-function gradients come from inverting each triangle's vertex matrix, one
triangle at a time.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

KIND_CSR, KIND_2D5, KIND_2D13_SQ, KIND_3D7 = 0, 1, 2, 3


def second_difference_1d(n: int, periodic: bool) -> sp.csr_matrix:
    """T = tridiag(-1, 2, -1); periodic adds the wrap-around entries (summed)."""
    T = sp.lil_matrix((n, n))
    for i in range(n):
        T[i, i] += 2.0
        for j in (i - 1, i + 1):
            if periodic:
                T[i, j % n] += -1.0
            elif 0 <= j < n:
                T[i, j] += -1.0
    return T.tocsr()


def neg_laplacian(dims, periodic: bool) -> sp.csr_matrix:
    """-Laplacian as the Kronecker sum of 1D second differences, x fastest."""
    dims = [int(d) for d in dims]
    n = int(np.prod(dims))
    L = sp.csr_matrix((n, n))
    for ax, nd in enumerate(dims):
        left = int(np.prod(dims[ax + 1:]))   # slower axes
        right = int(np.prod(dims[:ax]))      # faster axes
        L = L + sp.kron(sp.kron(sp.identity(left), second_difference_1d(nd, periodic)),
                        sp.identity(right))
    return L.tocsr()


def precision(kind: int, dims, kappa2, periodic: bool = False, tau: float = 0.0,
              mask=None, scale: float = 1.0) -> sp.csr_matrix:
    """Q for one grid model.

    kind 1 (2D 5-point) / 3 (3D 7-point): scale*(diag(kappa2) - Lap + tau*diag(mask)).
    kind 2 (2D 13-point Matern alpha=2): scale*(kappa2 I - Lap)^2 (matrix product).
    kappa2 is a scalar or a per-vertex array.
    """
    L = neg_laplacian(dims, periodic)
    n = L.shape[0]
    k2 = np.broadcast_to(np.asarray(kappa2, dtype=np.float64), (n,))
    Q1 = (sp.diags(k2) + L).tocsr()
    if kind == KIND_2D13_SQ:
        Q = (Q1 @ Q1).tocsr()
    elif kind in (KIND_2D5, KIND_3D7):
        Q = Q1
    else:
        raise ValueError("kind")
    if mask is not None and tau != 0.0:
        Q = (Q + tau * sp.diags(np.asarray(mask, dtype=np.float64))).tocsr()
    Q = (scale * Q).tocsr()
    Q.eliminate_zeros()
    Q.sort_indices()
    return Q


def bandwidth(Q: sp.csr_matrix) -> int:
    coo = Q.tocoo()
    if coo.nnz == 0:
        return 0
    return int(np.max(np.abs(coo.row - coo.col)))


def to_lower_band(Q: sp.csr_matrix, b: int, dtype=np.float64) -> np.ndarray:
    """Lower band, column-major: entry (i, j), j <= i <= j+b, at A[j*(b+1) + i-j]."""
    n = Q.shape[0]
    A = np.zeros((n, b + 1), dtype=dtype)   # row j of this array = column j of the band
    coo = Q.tocoo()
    sel = coo.row >= coo.col
    A[coo.col[sel], coo.row[sel] - coo.col[sel]] = coo.data[sel]
    return A.reshape(-1)


def csr_arrays(Q: sp.csr_matrix):
    """(int64 rowptr, int32 col, f64 val) of Q."""
    Q = Q.tocsr()
    Q.sort_indices()
    return (Q.indptr.astype(np.int64), Q.indices.astype(np.int32), Q.data.astype(np.float64))


def fem_p1(points: np.ndarray, triangles: np.ndarray):
    """Lumped mass diagonal c (n,) and stiffness G (CSR) of P1 elements, one triangle
    at a time: the hat functions restricted to a triangle are the columns of the
    inverse of [[1, x_k, y_k]]_k (value 1 at their own vertex, 0 at the others)."""
    n = points.shape[0]
    c = np.zeros(n)
    G = {}
    for tri in triangles:
        V = np.array([[1.0, points[k, 0], points[k, 1]] for k in tri])
        area = 0.5 * abs(np.linalg.det(V))
        coef = np.linalg.inv(V)            # column i: (c0, cx, cy) of phi_i on this triangle
        for i in range(3):
            c[tri[i]] += area / 3.0
            for j in range(3):
                gij = area * (coef[1, i] * coef[1, j] + coef[2, i] * coef[2, j])
                key = (int(tri[i]), int(tri[j]))
                G[key] = G.get(key, 0.0) + gij
    r = np.array([k[0] for k in G], dtype=np.int64)
    cc = np.array([k[1] for k in G], dtype=np.int64)
    v = np.array(list(G.values()))
    return c, sp.csr_matrix((v, (r, cc)), shape=(n, n))


def fem_spde_precision(points, triangles, kappa2: float, alpha: int = 1, tau: float = 1.0):
    """Q = tau (kappa^2 C~ + G) (alpha = 1) or tau K C~^{-1} K, K = kappa^2 C~ + G (alpha = 2)."""
    c, G = fem_p1(points, triangles)
    K = (kappa2 * sp.diags(c) + G).tocsr()
    if alpha == 1:
        Q = tau * K
    elif alpha == 2:
        Q = tau * (K @ sp.diags(1.0 / c) @ K)
    else:
        raise ValueError("alpha must be 1 or 2")
    Q = Q.tocsr()
    Q.sort_indices()
    return Q
