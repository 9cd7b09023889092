"""Full-size parity at the configuration bench.py times (Matern alpha=2, 1024 x 1024).

The oracle's exact probed rational target per colour, sum_k f_N(lambda_k) |u_k^T v_c|^2 by an
orthonormal DST-I (Sec. 2.1), is compared with the GPU's per-colour terms and total, in the
launch configuration of the bench (distance-2 colouring, N = 20, automatic tile width), for
the mixed-precision form and the plain FP64 form.  The probing error against the exact log
det is printed beside, not asserted.
"""
import numpy as np
import pytest

import paper_1105_5256_gb300 as L
import synth
from oracle import closed_forms as cf
from oracle import hht
from oracle import method as mt
from oracle import matrices as om
from colour_check import checked_colouring

pytestmark = pytest.mark.gpu

DIMS, DIST, NSHIFT = (1024, 1024), 2, 20
KIND = L.LD_STENCIL_2D13_SQ


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_5256_gb300 import _build
    _build.build()
    return L.library()


def target(k2, col):
    lo, hi = mt.spectral_bounds(KIND, DIMS, k2)
    s, a = hht.log_nodes(lo, hi, NSHIFT)
    return cf.probed_value(KIND, DIMS, k2, False, col, lambda lam: hht.f_N(lam, s, a),
                           per_colour=True)


@pytest.mark.parametrize("prec,tol", [(L.LD_MIXED, 1e-6), (L.LD_FP64, 1e-8)])
def test_matern_1024_against_spectral_oracle(prec, tol):
    k2 = float(synth.kappa2_draws(2, 16)[1])
    ctx = L.ld_create(L.grid_matrix(KIND, DIMS, k2), DIST, NSHIFT, tol, L.options(precision=prec))
    val, info = L.ld_logdet(ctx)
    col, nc = checked_colouring(ctx, om.precision(KIND, DIMS, k2), DIST)
    assert nc == 18
    terms, _ = L.ld_column_terms(ctx)
    ref = target(k2, col)
    if prec == L.LD_FP64:
        assert abs(val - ref.sum()) <= 50 * tol * np.abs(ref).sum()
        assert np.abs(terms - ref).max() <= 50 * tol * np.abs(ref).max()
    else:
        assert abs(val - ref.sum()) <= 2e-5 * abs(ref.sum())
        assert np.abs(terms - ref).max() <= 2e-5 * np.abs(ref).max()
    exact = cf.logdet(KIND, DIMS, k2, False)
    print("kappa2 %.4f  gpu %.6f  target %.6f  rel %.2e  exact %.6f  probing rel %.2e  iters %d"
          % (k2, val, ref.sum(), (val - ref.sum()) / ref.sum(), exact, (ref.sum() - exact) / exact,
             info["iters"]))


def test_gradient_fullsize_periodic_5pt():
    """tr(Q^{-1}) probed (d log det / d kappa2) at 1024^2 on a torus, projected seed sums."""
    dims, k2, tol = (1024, 1024), 0.05, 1e-8
    ctx = L.ld_create(L.grid_matrix(L.LD_STENCIL_2D5, dims, k2, periodic=True), 4, NSHIFT, tol)
    v, g, info = L.ld_logdet_grad(ctx, [L.LD_P_KAPPA2])
    col, _ = checked_colouring(ctx, om.precision(om.KIND_2D5, dims, k2, periodic=True), 4)
    gref = cf.probed_value(L.LD_STENCIL_2D5, dims, k2, True, col, lambda lam: 1.0 / lam)
    assert abs(g[0] - gref) <= 1e-6 * abs(gref)
