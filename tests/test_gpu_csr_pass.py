"""GPU: the CSR pass of the grid engine (a streaming CG step, then the product by row
groups of T lanes with the six dots and the multi-shift tail) against the oracle.

Target: the per-colour rational terms sum_l Re alpha_l v_c^T (Q - sigma_l I)^{-1} v_c
(Sec. 2.1, Eq. of the rational approximation) from exact sparse-LU solves on the oracle's
own nodes for the same interval, so only the CG stopping error separates the two:
  FP64   |term_c - ref_c| <= 50 tol |ref_c| + 1e-12 sum |ref|
  mixed  |term_c - ref_c| <= 2e-5 max |ref|   (FP32 vectors, FP64 scalars)
Every tile width of both precisions runs (T = 6 and T = 3 leave lanes of each warp idle),
on a FEM mesh (rows of about 20 entries: several T-wide chunks a row) and on an irregular
pattern with rows of 2 to about 30 entries; the kept seed solutions give the scale
gradient, which probing makes exact: d log det / ds = tr(Q^{-1} Q / s) = n / s.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import paper_1105_5256_gb300 as L
import synth
from colour_check import checked_colouring
from oracle import hht
from oracle import matrices as om
from oracle import method as mt

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_5256_gb300 import _build
    _build.build()
    return L.library()


def interval(Q):
    """[0.9 lambda_min, Gershgorin] from a shift-invert Lanczos run and the row sums."""
    lmin = spla.eigsh(Q.tocsc(), k=1, sigma=0.0, which="LM", return_eigenvectors=False)[0]
    return 0.9 * float(lmin), float(np.abs(Q).sum(axis=1).max())


def mesh_q():
    p, t = synth.perturbed_triangulation(21, 120, 110)
    h = 1.0 / 119
    return om.fem_spde_precision(p, t, 0.3 / h ** 2, 2, 1.0)


def irregular_q():
    n = 20000
    rows, cols, w = synth.random_sparse_spd_pattern(23, n, 24)
    rp, ci, vv = synth.csr_from_edges(n, rows, cols, w, 0.05)
    return sp.csr_matrix((vv, ci, rp), shape=(n, n))


_cache = {}


def problem(name):
    if name not in _cache:
        Q = mesh_q() if name == "mesh" else irregular_q()
        Q.sort_indices()
        _cache[name] = (Q, interval(Q))
    return _cache[name]


def run(Q, lo, hi, prec, T, d, keep_x0=0, scale=1.0):
    tol = 1e-10 if prec == L.LD_FP64 else 1e-6
    rp, ci, vv = om.csr_arrays(Q)
    ctx = L.ld_create(L.csr_matrix(rp, ci, vv, scale=scale), d, 24, tol,
                      L.options(precision=prec, engine=1, tile_width=T, lambda_min=lo * scale,
                                lambda_max=hi * scale, keep_x0=keep_x0))
    return ctx, tol


@pytest.mark.parametrize("name,d", [("mesh", 2), ("irregular", 1)])
@pytest.mark.parametrize("prec,T", [(L.LD_MIXED, 2), (L.LD_MIXED, 4), (L.LD_MIXED, 6), (L.LD_MIXED, 8),
                                    (L.LD_FP64, 1), (L.LD_FP64, 2), (L.LD_FP64, 3), (L.LD_FP64, 4)])
def test_csr_pass_terms_match_sparse_lu(name, d, prec, T):
    Q, (lo, hi) = problem(name)
    ctx, tol = run(Q, lo, hi, prec, T, d)
    val, info = L.ld_logdet(ctx)
    assert info["engine"] == 1 and info["tile_width"] == T
    col, _ = checked_colouring(ctx, Q, d)
    key = (name, "ref")
    if key not in _cache:   # the same colouring for every tile width
        s, a = hht.log_nodes(lo, hi, 24)
        _cache[key] = (col, mt.probed_rational_splu(Q, col, s, a, per_colour=True))
    assert np.array_equal(_cache[key][0], col)
    ref = _cache[key][1]
    terms, _ = L.ld_column_terms(ctx)
    if prec == L.LD_FP64:
        assert np.all(np.abs(terms - ref) <= 50 * tol * np.abs(ref) + 1e-12 * np.abs(ref).sum())
    else:
        assert np.abs(terms - ref).max() <= 2e-5 * np.abs(ref).max()
    assert abs(val - ref.sum()) <= 2e-5 * np.abs(ref).sum()


@pytest.mark.parametrize("prec,T", [(L.LD_MIXED, 6), (L.LD_FP64, 3)])
def test_csr_pass_kept_seed_solutions_give_the_scale_gradient(prec, T):
    """Q = s Q0 with s = 2: the kept x gives d log det / ds = sum_c v_c^T Q^{-1} Q0 v_c,
    which is n / s for any colouring; the value equals the solve without kept x."""
    Q, (lo, hi) = problem("irregular")
    n = Q.shape[0]
    ctx, tol = run(Q, lo, hi, prec, T, 1, keep_x0=1, scale=2.0)
    v, g, info = L.ld_logdet_grad(ctx, [L.LD_P_SCALE])
    assert info["engine"] == 1
    bar = 1e-8 if prec == L.LD_FP64 else 2e-5
    assert abs(g[0] - n / 2.0) <= bar * n / 2.0
    plain, _ = run(Q, lo, hi, prec, T, 1, scale=2.0)
    v2, _ = L.ld_logdet(plain)
    assert v == v2
