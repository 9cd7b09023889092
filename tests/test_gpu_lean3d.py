"""GPU: the lean 3D pass (7-point kind, FP32 vectors, four state words per vertex and
probing vector per CG pass; Q p recomputed from the state) against the oracle and the
stored-w 3D pass.

The lean pass is the same one-reduction CG as the stored-w pass in exact arithmetic
(Sec. 2.1: the seed CG on Q x = v_c drives every shifted system); only rounding differs.
Scalar-kappa^2 cases compare the per-colour terms with the oracle's exact rational target
from the sine / Fourier closed form (no Krylov error) at the mixed-precision bar 2e-5, and
the two passes with each other.  The cases cover the pass's geometry: grids narrower than
a CTA tile (28 x 12 own columns) and several tiles in x and y, ragged edges, tori (wrapped
halos), z segments, tiles of 2 and 4 columns, the kept seed solution (gradient), and a
kappa^2 field against exact sparse-LU solves.
"""
import numpy as np
import pytest

import paper_1105_5256_gb300 as L
import synth
from colour_check import checked_colouring
from oracle import closed_forms as cf
from oracle import hht
from oracle import matrices as om
from oracle import method as mt
from oracle import probing

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_5256_gb300 import _build
    _build.build()
    return L.library()


CASES = [
    # dims, periodic, tile width, distance
    ((61, 29, 23), False, 2, 2),     # three x tiles, three y tiles (ragged), many z planes
    ((61, 29, 23), False, 4, 2),
    ((20, 10, 9), False, 4, 3),      # narrower than one tile
    ((30, 26, 18), True, 4, 2),      # torus: wrapped 2-wide halos
    ((17, 13, 40), True, 2, 2),      # odd torus narrower than a tile, tall
    ((90, 40, 6), False, 2, 1),      # thin in z
]


def run(dims, per, T, d, k2, lattice_pass, keep_x0=0):
    ctx = L.ld_create(L.grid_matrix(om.KIND_3D7, dims, k2, periodic=per), d, 20, 1e-6,
                      L.options(precision=L.LD_MIXED, engine=1, tile_width=T, lattice_pass=lattice_pass,
                                keep_x0=keep_x0))
    val, info = L.ld_logdet(ctx)
    terms, seeds = L.ld_column_terms(ctx)
    return ctx, val, info, terms, seeds


@pytest.mark.parametrize("dims,per,T,d", CASES)
def test_lean3d_matches_oracle_and_stored_w_pass(dims, per, T, d):
    k2 = 0.2
    ctx, val, info, terms, seeds = run(dims, per, T, d, k2, 0)
    assert info["pass_words"] == 4 and info["tile_width"] == T
    col, _ = checked_colouring(ctx, om.precision(om.KIND_3D7, dims, k2, periodic=per), d)
    lo, hi = mt.spectral_bounds(om.KIND_3D7, dims, k2, periodic=per)
    s, a = hht.log_nodes(lo, hi, 20)
    ref = cf.probed_value(om.KIND_3D7, dims, k2, per, col, lambda lam: hht.f_N(lam, s, a), per_colour=True)
    assert np.abs(terms - ref).max() <= 2e-5 * np.abs(ref).max()
    assert abs(val - ref.sum()) <= 2e-5 * abs(ref.sum())
    seed_ref = cf.probed_value(om.KIND_3D7, dims, k2, per, col, lambda lam: 1.0 / lam, per_colour=True)
    assert np.abs(seeds - seed_ref).max() <= 2e-5 * np.abs(seed_ref).max()
    _, val_w, info_w, terms_w, _ = run(dims, per, T, d, k2, 1)
    assert info_w["pass_words"] == 6
    assert np.abs(terms - terms_w).max() <= 2e-5 * np.abs(ref).max()
    assert abs(info["iters"] - info_w["iters"]) <= max(5, info_w["iters"] // 10)


@pytest.mark.parametrize("T", [2, 4])
def test_lean3d_keeps_the_seed_solution(T):
    """x_k = x_{k-1} + alpha p_{k-1} inside the lean pass: the gradient d log det / d kappa^2
    = sum_c v_c^T x_c equals the probed tr(Q^{-1}) of the closed form."""
    dims, k2 = (45, 20, 14), 0.1
    ctx = L.ld_create(L.grid_matrix(om.KIND_3D7, dims, k2), 2, 20, 1e-6,
                      L.options(precision=L.LD_MIXED, engine=1, tile_width=T, keep_x0=1))
    val, info = L.ld_logdet(ctx)
    assert info["pass_words"] == 6
    g = L.ld_grad(ctx, [L.LD_P_KAPPA2])
    col, _ = L.ld_get_colouring(ctx)
    gref = cf.probed_value(om.KIND_3D7, dims, k2, False, col, lambda lam: 1.0 / lam)
    assert abs(g[0] - gref) <= 2e-5 * abs(gref)


def test_lean3d_kappa2_field_against_sparse_lu():
    """A seeded kappa^2 field (the 3D non-stationary model): terms against exact sparse-LU
    rational solves on the oracle's nodes, the field-scale gradient against exact solves,
    and the stored-w pass beside."""
    dims = (30, 20, 16)
    f = synth.kappa2_field(7, dims)
    Q = om.precision(om.KIND_3D7, dims, f)
    out = {}
    for lp in (0, 1):
        ctx = L.ld_create(L.grid_matrix(om.KIND_3D7, dims, 1.0, kappa2_field=f), 2, 20, 1e-7,
                          L.options(precision=L.LD_MIXED, engine=1, tile_width=4, lattice_pass=lp))
        v, g, info = L.ld_logdet_grad(ctx, [L.LD_P_KAPPA2])
        out[lp] = (v, g, info, L.ld_column_terms(ctx)[0])
        col, _ = checked_colouring(ctx, Q, 2)
    assert out[0][2]["pass_words"] == 6 and out[1][2]["pass_words"] == 8
    lo, hi = mt.spectral_bounds(om.KIND_3D7, dims, f)
    s, a = hht.log_nodes(lo, hi, 20)
    ref = mt.probed_rational_splu(Q, col, s, a, per_colour=True)
    import scipy.sparse.linalg as spla
    V = probing.probing_vectors(col)
    X = spla.splu(Q.tocsc()).solve(V)
    gref = float(np.sum((f[:, None] * V) * X))
    for lp in (0, 1):
        v, g, info, terms = out[lp]
        assert np.abs(terms - ref).max() <= 2e-5 * np.abs(ref).max()
        assert abs(g[0] - gref) <= 2e-5 * abs(gref)
    assert np.abs(out[0][3] - out[1][3]).max() <= 2e-5 * np.abs(ref).max()


def test_lean3d_repeated_solves_are_deterministic():
    dims, k2 = (33, 30, 12), 0.3
    ctx = L.ld_create(L.grid_matrix(om.KIND_3D7, dims, k2), 2, 20, 1e-6,
                      L.options(precision=L.LD_MIXED, engine=1, tile_width=4))
    v1, i1 = L.ld_logdet(ctx)
    L.ld_logdet_grad(ctx, [L.LD_P_KAPPA2, L.LD_P_SCALE])
    v2, i2 = L.ld_logdet(ctx)
    assert i1["pass_words"] == 4 and i2["pass_words"] == 4
    assert v1 == v2
