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


# ---------------------------------------------------------------- distance selection
# Sec. 2.1 (heuristic for the power p of Q^p whose graph the colouring follows):
# solve for a column x = Q^{-1} e_j, or here y = log(Q) e_j, and take
#     p = min { d(l, j) : |y_l| < eps },
# d the graph distance in the graph of Q.  Reading: eps is relative to |y_j| (the
# paper's eps is unnormalised; relative makes p independent of the scale of Q).

def graph_distances(Q: sp.csr_matrix, j: int, max_d: int) -> np.ndarray:
    """Breadth-first graph distances from vertex j over the pattern of Q (int64;
    -1 beyond max_d)."""
    Q = Q.tocsr()
    n = Q.shape[0]
    dist = np.full(n, -1, dtype=np.int64)
    dist[j] = 0
    frontier = [int(j)]
    for d in range(1, max_d + 1):
        nxt = []
        for u in frontier:
            for w in Q.indices[Q.indptr[u]:Q.indptr[u + 1]]:
                if dist[w] < 0:
                    dist[w] = d
                    nxt.append(int(w))
        frontier = nxt
        if not frontier:
            break
    return dist


def decay_profile(y: np.ndarray, dist: np.ndarray, j: int, max_d: int) -> np.ndarray:
    """profile[d] = max over vertices at graph distance d of |y_l| / |y_j|."""
    y = np.abs(np.asarray(y)) / abs(y[j])
    prof = np.zeros(max_d + 1)
    for d in range(max_d + 1):
        sel = dist == d
        prof[d] = y[sel].max() if np.any(sel) else 0.0
    return prof


def decay_distance(y: np.ndarray, dist: np.ndarray, j: int, eps: float) -> int:
    """min { d(l, j) : |y_l| < eps |y_j| } over vertices within the distances given
    (-1 when none qualifies)."""
    ratio = np.abs(np.asarray(y)) / abs(y[j])
    sel = (dist >= 0) & (ratio < eps)
    return int(dist[sel].min()) if np.any(sel) else -1
