"""Oracle: probing vectors from a distance-d greedy colouring (test infrastructure).

Sec. 2.1: probing vectors v_c are indicator vectors of the colour classes of a
neighbour colouring of the graph induced by Q^d, i.e. a distance-d colouring
of the graph of Q (vertices at graph distance <= d get different colours).
Reading: natural vertex order, each vertex takes the smallest colour unused
within distance d (greedy; the paper names greedy colourings but no order).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import _native


def colour_greedy(Q: sp.csr_matrix, d: int) -> np.ndarray:
    """int32 colour per vertex (plain C BFS, natural order)."""
    Q = Q.tocsr()
    n = Q.shape[0]
    rowptr = Q.indptr.astype(np.int64)
    col = Q.indices.astype(np.int32)
    out = np.empty(n, dtype=np.int32)
    nc = _native.lib().or_colour_greedy(n, _native.ptr(rowptr), _native.ptr(col), int(d),
                                        _native.ptr(out))
    if nc < 0:
        raise MemoryError("colouring")
    return out


def distance_pattern(Q: sp.csr_matrix, d: int) -> sp.csr_matrix:
    """Boolean pattern of vertex pairs at graph distance <= d: (I + |A|)^d."""
    A = Q.tocsr().copy()
    A.data = np.ones_like(A.data)
    n = A.shape[0]
    B = (sp.identity(n, format="csr") + A).astype(bool).astype(np.int8)
    P = sp.identity(n, format="csr", dtype=np.int8)
    for _ in range(d):
        P = (P @ B)
        P.data = np.ones_like(P.data)
    return P.tocsr()


def is_valid_colouring(Q: sp.csr_matrix, d: int, colour: np.ndarray) -> bool:
    """No two distinct vertices within graph distance d share a colour."""
    P = distance_pattern(Q, d).tocoo()
    off = P.row != P.col
    colour = np.asarray(colour)
    return bool(np.all(colour[P.row[off]] != colour[P.col[off]]))


def probing_vectors(colour: np.ndarray) -> np.ndarray:
    """Dense (n, C) block of 0/1 indicator columns (small cases only)."""
    colour = np.asarray(colour)
    C = int(colour.max()) + 1 if colour.size else 0
    V = np.zeros((colour.size, C))
    V[np.arange(colour.size), colour] = 1.0
    return V
