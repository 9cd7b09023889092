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

The assembly is the library's `ld_spde_fem_csr` (host C++); this module marshals the
arrays.  The result feeds ld_create as an LD_CSR matrix (the kernels never see the mesh).
"""
from __future__ import annotations

import ctypes as C

import numpy as np


def spde_csr(points, triangles, kappa2: float, alpha: int = 1, tau: float = 1.0):
    """CSR arrays (rowptr int64, colidx int32, val float64) of the alpha = 1 or 2 SPDE
    precision on the mesh (points n x 2, triangles m x 3 vertex indices)."""
    from . import _check, _ptr, library
    P = np.ascontiguousarray(points, dtype=np.float64)
    T = np.ascontiguousarray(triangles, dtype=np.int64)
    if P.ndim != 2 or P.shape[1] != 2 or T.ndim != 2 or T.shape[1] != 3:
        raise ValueError("points must be n x 2 and triangles m x 3")
    if alpha not in (1, 2):
        raise ValueError("alpha must be 1 or 2")
    if not (kappa2 > 0.0 and tau > 0.0):
        raise ValueError("kappa2 and tau must be positive")
    n, m = P.shape[0], T.shape[0]
    lib = library()
    nnz = C.c_int64()
    args = (n, _ptr(P), m, _ptr(T), float(kappa2), int(alpha), float(tau))
    _check(lib.ld_spde_fem_csr(*args, 0, None, None, None, C.byref(nnz)))
    rp = np.zeros(n + 1, dtype=np.int64)
    ci = np.zeros(nnz.value, dtype=np.int32)
    vv = np.zeros(nnz.value, dtype=np.float64)
    _check(lib.ld_spde_fem_csr(*args, nnz.value, _ptr(rp), _ptr(ci), _ptr(vv), C.byref(nnz)))
    return rp, ci, vv


def spde_matrix(points, triangles, kappa2: float, alpha: int = 1, tau: float = 1.0):
    """ld_matrix (LD_CSR) of the SPDE precision on the mesh; returns (Matrix, arrays kept alive)
    like grid_matrix / csr_matrix."""
    from . import csr_matrix
    return csr_matrix(*spde_csr(points, triangles, kappa2, alpha, tau))
