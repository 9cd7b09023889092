"""General-mesh input: SPDE precision matrices from a triangulation (host preprocessing).

The paper motivates sparse precision matrices by the SPDE construction of Gaussian
fields (Sec. 1) and fits the model tau (kappa - Laplacian) u = W (Sec. 3).  On a
regular grid the library has stencil kinds; on an unstructured triangulation the
same model becomes a general CSR matrix through piecewise-linear finite elements:

    C~  lumped mass, diagonal: a third of each triangle's area to each of its vertices;
    G   stiffness, G_ij = sum over triangles T of |T| grad(phi_i) . grad(phi_j),
        natural (Neumann) boundary;
    Q = tau (kappa^2 C~ + G)                        (alpha = 1)
    Q = tau K C~^{-1} K,   K = kappa^2 C~ + G       (alpha = 2).

On triangle T with edge vectors e_i opposite vertex i (counter-clockwise order),
grad(phi_i) is e_i rotated by 90 degrees over 2|T|, so the element stiffness is
e_i . e_j / (4 |T|).  Assembly is vectorised over triangles; the result feeds
ld_create as an LD_CSR matrix (the kernels never see the mesh).
"""
from __future__ import annotations

import numpy as np


def fem_p1(points, triangles):
    """(lumped mass c (n,), stiffness (rowptr int64, colidx int32, val f64)) of P1 elements.
    Triangles may come in either orientation."""
    import scipy.sparse as sp
    P = np.ascontiguousarray(points, dtype=np.float64)
    T = np.ascontiguousarray(triangles, dtype=np.int64)
    if P.ndim != 2 or P.shape[1] != 2 or T.ndim != 2 or T.shape[1] != 3:
        raise ValueError("points must be n x 2 and triangles m x 3")
    n = P.shape[0]
    if T.size and (T.min() < 0 or T.max() >= n):
        raise ValueError("triangle vertex index out of range")
    p0, p1, p2 = P[T[:, 0]], P[T[:, 1]], P[T[:, 2]]
    e = np.stack([p2 - p1, p0 - p2, p1 - p0], axis=1)          # m x 3 x 2, e_i opposite vertex i
    area2 = e[:, 2, 0] * (-e[:, 1, 1]) - e[:, 2, 1] * (-e[:, 1, 0])   # cross(p1 - p0, p2 - p0)
    if np.any(area2 == 0.0):
        raise ValueError("degenerate triangle")
    area = 0.5 * np.abs(area2)
    K = np.einsum("mid,mjd->mij", e, e) / (4.0 * area)[:, None, None]
    c = np.zeros(n)
    np.add.at(c, T.ravel(), np.repeat(area / 3.0, 3))
    rows = np.repeat(T, 3, axis=1).ravel()
    cols = np.tile(T, (1, 3)).ravel()
    G = sp.coo_matrix((K.ravel(), (rows, cols)), shape=(n, n)).tocsr()
    G.sum_duplicates()
    G.sort_indices()
    return c, (G.indptr.astype(np.int64), G.indices.astype(np.int32), G.data.astype(np.float64))


def spde_csr(points, triangles, kappa2: float, alpha: int = 1, tau: float = 1.0):
    """CSR arrays (rowptr, colidx, val) of the alpha = 1 or 2 SPDE precision on the mesh."""
    import scipy.sparse as sp
    if alpha not in (1, 2):
        raise ValueError("alpha must be 1 or 2")
    if not (kappa2 > 0.0 and tau > 0.0):
        raise ValueError("kappa2 and tau must be positive")
    c, (rp, ci, vv) = fem_p1(points, triangles)
    n = c.size
    if np.any(c <= 0.0):
        raise ValueError("vertex outside every triangle")
    K = sp.csr_matrix((vv, ci, rp), shape=(n, n)) + sp.diags(kappa2 * c)
    Q = tau * (K if alpha == 1 else K @ sp.diags(1.0 / c) @ K)
    Q = sp.csr_matrix(Q)
    Q.sum_duplicates()
    Q.sort_indices()
    return Q.indptr.astype(np.int64), Q.indices.astype(np.int32), Q.data.astype(np.float64)


def spde_matrix(points, triangles, kappa2: float, alpha: int = 1, tau: float = 1.0):
    """ld_matrix (LD_CSR) of the SPDE precision on the mesh; returns (Matrix, arrays kept alive)
    like grid_matrix / csr_matrix."""
    from . import csr_matrix
    return csr_matrix(*spde_csr(points, triangles, kappa2, alpha, tau))
