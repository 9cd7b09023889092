"""Test helper: a context's colouring, checked against the oracle's.

The GPU parity tests compute their expected values from the probing vectors of a
colouring.  That colouring is the oracle's own greedy distance-d colouring of the
oracle's matrix (Sec. 2.1: natural vertex order, smallest free colour); the
library's colouring, which the GPU solve used, must equal it bit for bit.
"""
import numpy as np

import paper_1105_5256_gb300 as L
from oracle import probing


def checked_colouring(ctx, Q, d):
    col, _ = L.ld_get_colouring(ctx)
    ref = probing.colour_greedy(Q, d)
    assert np.array_equal(col, ref), "library colouring differs from the oracle's greedy colouring"
    return ref, int(ref.max()) + 1


def checked_on_subbox(col, dims, d, box=20):
    """Large 3D grids: the colouring restricted to the leading box^3 corner must be a
    valid distance-d colouring of that sub-lattice (a necessary condition)."""
    from oracle import matrices as om
    nx, ny, nz = dims
    c = np.asarray(col).reshape(nz, ny, nx)[:box, :box, :box].reshape(-1)
    Qs = om.precision(om.KIND_3D7, (box, box, box), 1.0)
    assert probing.is_valid_colouring(Qs, d, c)
