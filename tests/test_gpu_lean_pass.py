"""GPU: the lean lattice pass (four state words per vertex and probing vector per CG
iteration; Q p recomputed from the state) against the oracle and the stored-w pass.

The lean pass is the same one-reduction CG as the stored-w pass in exact arithmetic
(Sec. 2.1: the seed CG on Q x = v_c drives every shifted system); only rounding
differs.  Each case runs both passes on the same grid and colouring and compares the
per-colour terms with the oracle's exact rational target from the sine / Fourier
closed form (no Krylov error), at the mixed-precision bar 2e-5, and the two passes with
each other.  The cases cover the pass's geometry: grids whose width is not a multiple
of the strip width (ragged last strip, idle warps), odd widths (one lattice column per
thread) and even widths (two), tiles of 2 and 4 columns, tori, one-strip grids narrower
than a CTA, tall grids split into many row segments, and the kept seed solution.
"""
import numpy as np
import pytest

import paper_1105_5256_gb300 as L
from oracle import closed_forms as cf
from oracle import hht
from oracle import matrices as om
from oracle import method as mt
from colour_check import checked_colouring

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
    # kind, dims, periodic, tile width
    (om.KIND_2D13_SQ, (1024, 300), False, 2),   # 2 columns a thread, ragged last strip
    (om.KIND_2D13_SQ, (333, 257), False, 2),    # odd width at T = 2: one column a thread
    (om.KIND_2D13_SQ, (130, 96), True, 4),      # torus, 4-column tiles, 1 column a thread
    (om.KIND_2D13_SQ, (201, 150), True, 4),     # odd torus narrower than a strip
    (om.KIND_2D5, (520, 260), False, 2),
    (om.KIND_2D5, (255, 300), False, 4),        # odd width, T = 4
    (om.KIND_2D5, (64, 512), True, 2),          # torus wrapped 4 times by one strip, tall
    (om.KIND_2D5, (97, 61), True, 4),           # odd torus, wrapped twice
    (om.KIND_2D5, (10, 700), False, 2),         # one mostly idle strip, many segments
]


def lean_applies(dims, T):
    """The lean pass runs for FP32 tiles of 2 or 4 columns on any 2D lattice (two lattice
    columns a thread at T = 2 on even widths, one otherwise)."""
    return T in (2, 4)


def run(kind, dims, per, T, k2, d, lattice_pass, keep_x0=0):
    ctx = L.ld_create(L.grid_matrix(kind, dims, k2, periodic=per), d, 20, 1e-6,
                      L.options(precision=L.LD_MIXED, engine=1, tile_width=T,
                                lattice_pass=lattice_pass, keep_x0=keep_x0))
    val, info = L.ld_logdet(ctx)
    terms, seeds = L.ld_column_terms(ctx)
    return ctx, val, info, terms, seeds


@pytest.mark.parametrize("kind,dims,per,T", CASES)
def test_lean_pass_matches_oracle_and_stored_w_pass(kind, dims, per, T):
    k2 = 0.05
    d = 2 if kind == om.KIND_2D13_SQ else 4
    ctx, val, info, terms, seeds = run(kind, dims, per, T, k2, d, 0)
    assert info["pass_words"] == (4 if lean_applies(dims, T) else 6) and info["tile_width"] == T
    col, _ = checked_colouring(ctx, om.precision(kind, dims, k2, periodic=per), d)
    lo, hi = mt.spectral_bounds(kind, dims, k2, periodic=per)
    s, a = hht.log_nodes(lo, hi, 20)
    ref = cf.probed_value(kind, dims, k2, per, col, lambda lam: hht.f_N(lam, s, a), per_colour=True)
    assert np.abs(terms - ref).max() <= 2e-5 * np.abs(ref).max()
    assert abs(val - ref.sum()) <= 2e-5 * abs(ref.sum())
    seed_ref = cf.probed_value(kind, dims, k2, per, col, lambda lam: 1.0 / lam, per_colour=True)
    assert np.abs(seeds - seed_ref).max() <= 2e-5 * np.abs(seed_ref).max()
    _, val_w, info_w, terms_w, _ = run(kind, dims, per, T, k2, d, 1)
    assert info_w["pass_words"] == 6
    assert np.abs(terms - terms_w).max() <= 2e-5 * np.abs(ref).max()
    # the same CG: iteration counts agree up to FP32 rounding near the tolerance
    assert abs(info["iters"] - info_w["iters"]) <= max(5, info_w["iters"] // 10)


def test_lean_pass_keeps_the_seed_solution_on_the_5_point_kind():
    """x_k = x_{k-1} + alpha p_{k-1} inside the lean 5-point pass (6 words with x): the
    gradient d log det / d kappa^2 = sum_c v_c^T x_c from the kept solution equals the
    probed tr(Q^{-1}) of the closed form; the Matern kind keeps x through the stored-w
    pass (8 words)."""
    dims, k2 = (300, 222), 0.05
    ctx = L.ld_create(L.grid_matrix(om.KIND_2D5, dims, k2), 4, 20, 1e-6,
                      L.options(precision=L.LD_MIXED, engine=1, keep_x0=1))
    val, info = L.ld_logdet(ctx)
    assert info["pass_words"] == 6
    g = L.ld_grad(ctx, [L.LD_P_KAPPA2])
    col, _ = L.ld_get_colouring(ctx)
    gref = cf.probed_value(om.KIND_2D5, dims, k2, False, col, lambda lam: 1.0 / lam)
    assert abs(g[0] - gref) <= 2e-5 * abs(gref)
    ctx2 = L.ld_create(L.grid_matrix(om.KIND_2D13_SQ, (130, 120), 0.3), 2, 20, 1e-6,
                       L.options(precision=L.LD_MIXED, engine=1, keep_x0=1))
    _, info2 = L.ld_logdet(ctx2)
    assert info2["pass_words"] == 8
    _, info3 = L.ld_logdet(L.ld_create(L.grid_matrix(om.KIND_2D13_SQ, (130, 120), 0.3), 2, 20, 1e-6,
                                       L.options(precision=L.LD_MIXED, engine=1)))
    assert info3["pass_words"] == 4


def test_lean_pass_repeated_solves_are_deterministic():
    """The same context solved twice (and after switching to a kept x and back) gives
    bit-identical results: fixed reduction order, no state carried between solves."""
    dims, k2 = (200, 150), 0.1
    ctx = L.ld_create(L.grid_matrix(om.KIND_2D13_SQ, dims, k2), 2, 20, 1e-6,
                      L.options(precision=L.LD_MIXED, engine=1))
    v1, i1 = L.ld_logdet(ctx)
    L.ld_logdet_grad(ctx, [L.LD_P_KAPPA2])          # keeps x: stored-w pass
    v2, i2 = L.ld_logdet(ctx)
    assert i1["pass_words"] == 4 and i2["pass_words"] == 4
    assert v1 == v2


@pytest.mark.parametrize("dims,per", [((260, 130), False), ((120, 90), True), ((97, 64), False)])
def test_lean_pass_masked_posterior_diagonal_from_codes(dims, per):
    """Gauss-linear posterior Q = kappa^2 I - Lap + tau diag(mask) (Sec. 1): the lean pass
    forms kappa^2 + tau mask_i from the mask bit of its lane codes (halo and wrapped columns
    included); terms against the exact sparse-LU rational target and against the stored-w
    pass, which reads the diagonal as a word, with the gradients (kappa^2, tau)."""
    import synth
    from oracle import probing
    import scipy.sparse.linalg as spla
    n = dims[0] * dims[1]
    k2, tau = 0.1, 4.0
    mask = synth.obs_mask(11, n, 0.1)
    Q = om.precision(om.KIND_2D5, dims, k2, periodic=per, tau=tau, mask=mask)
    out = {}
    for lp in (0, 1):
        ctx = L.ld_create(L.grid_matrix(om.KIND_2D5, dims, k2, periodic=per, tau=tau, obs_mask=mask), 4, 20,
                          1e-7, L.options(precision=L.LD_MIXED, engine=1, tile_width=2, lattice_pass=lp))
        v, g, info = L.ld_logdet_grad(ctx, [L.LD_P_KAPPA2, L.LD_P_TAU])
        out[lp] = (v, g, info, L.ld_column_terms(ctx)[0])
        col, _ = checked_colouring(ctx, Q, 4)
    assert out[0][2]["pass_words"] == 6 and out[1][2]["pass_words"] == 8
    lo, hi = mt.spectral_bounds(om.KIND_2D5, dims, k2, periodic=per, tau=tau, mask=mask)
    s, a = hht.log_nodes(lo, hi, 20)
    ref = mt.probed_rational_splu(Q, col, s, a, per_colour=True)
    V = probing.probing_vectors(col)
    X = spla.splu(Q.tocsc()).solve(V)
    gref = [float(np.sum(V * X)), float(np.sum((mask[:, None] * V) * X))]
    for lp in (0, 1):
        v, g, info, terms = out[lp]
        assert np.abs(terms - ref).max() <= 2e-5 * np.abs(ref).max()
        for got, r in zip(g, gref):
            assert abs(got - r) <= 2e-5 * abs(r)
    assert np.abs(out[0][3] - out[1][3]).max() <= 2e-5 * np.abs(ref).max()
