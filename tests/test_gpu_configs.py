"""The Gauss-linear posterior and 3D non-stationary workloads (GPU).

Gauss-linear posterior (Sec. 1, Q_p = Q_x + tau A^T A, A observing 10% of the nodes):
  * 2048 x 2048: d log det / d kappa^2 against a central finite difference of the
    FP64 log det (h = 1e-4 relative; E = I commutes with Q, so the difference of the
    probed estimator equals the probed trace up to quadrature and CG error);
  * 128 x 128: both gradients against the oracle's probed traces (exact solves), with
    the gap to the exact tr(Q^{-1} E) (Takahashi selected inverse) reported.
3D 7-point with a kappa^2 field (log kappa^2 = -2 + smoothed N(0,1)):
  * 256^3 with a constant field, sampled colour terms against the 3D DST oracle;
  * 16 x 14 x 12 with the seeded field against exact banded shifted solves.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import paper_1105_5256_gb300 as L
import synth
from oracle import closed_forms as cf
from oracle import hht
from oracle import matrices as om
from oracle import method as mt
from oracle import probing
from colour_check import checked_colouring, checked_on_subbox

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_5256_gb300 import _build
    _build.build()
    return L.library()


def test_posterior_2048_gradient_vs_finite_difference():
    dims, k2, tau, h, tol = (2048, 2048), 0.1, 4.0, 1e-4, 1e-9
    n = dims[0] * dims[1]
    mask = synth.obs_mask(4, n, 0.1)
    ctx = L.ld_create(L.grid_matrix(L.LD_STENCIL_2D5, dims, k2, tau=tau, obs_mask=mask), 4, 20, tol,
                      L.options(precision=L.LD_FP64, keep_x0=1))
    v, g, info = L.ld_logdet_grad(ctx, [L.LD_P_KAPPA2, L.LD_P_TAU])
    L.ld_set_params(ctx, k2 * (1 + h), tau)
    up = L.ld_logdet(ctx)[0]
    L.ld_set_params(ctx, k2 * (1 - h), tau)
    dn = L.ld_logdet(ctx)[0]
    fd = (up - dn) / (2 * k2 * h)
    print("2048^2 posterior: logdet %.6f  d/dkappa2 %.6f  FD %.6f  d/dtau %.6f  iters %d"
          % (v, g[0], fd, g[1], info["iters"]))
    assert abs(g[0] - fd) <= 1e-6 * abs(fd)
    assert g[1] > 0 and np.isfinite(g[1])


@pytest.mark.parametrize("prec", [L.LD_FP64, L.LD_MIXED])
def test_posterior_128_gradients_vs_oracle_traces(prec):
    dims, k2, tau = (128, 128), 0.1, 4.0
    n = 128 * 128
    mask = synth.obs_mask(4, n, 0.1)
    tol = 1e-10 if prec == L.LD_FP64 else 1e-6
    ctx = L.ld_create(L.grid_matrix(L.LD_STENCIL_2D5, dims, k2, tau=tau, obs_mask=mask), 4, 20, tol,
                      L.options(precision=prec))
    v, g, _ = L.ld_logdet_grad(ctx, [L.LD_P_KAPPA2, L.LD_P_TAU])
    Q = om.precision(om.KIND_2D5, dims, k2, tau=tau, mask=mask)
    col, _ = checked_colouring(ctx, Q, 4)
    V = probing.probing_vectors(col)
    X = sp.linalg.splu(Q.tocsc()).solve(V)
    probed_k2 = float(np.sum(V * X))
    probed_tau = float(np.sum((mask[:, None] * V) * X))
    rel = 1e-8 if prec == L.LD_FP64 else 2e-5
    assert abs(g[0] - probed_k2) <= rel * abs(probed_k2)
    assert abs(g[1] - probed_tau) <= rel * abs(probed_tau)
    Z, b = mt.selected_inverse(Q)
    exact_k2 = mt.trace_inv_times(Z, b, sp.identity(n))
    exact_tau = mt.trace_inv_times(Z, b, sp.diags(mask.astype(float)))
    print("128^2 posterior: d/dkappa2 %.4f probed-exact %.2e | d/dtau %.4f probed-exact %.2e"
          % (g[0], (probed_k2 - exact_k2) / exact_k2, g[1], (probed_tau - exact_tau) / exact_tau))


def test_3d_256_constant_field_sampled_colours():
    dims, tol = (256, 256, 256), 1e-6
    n = 256 ** 3
    k2 = float(np.exp(-2.0))
    field = np.ones(n)
    ctx = L.ld_create(L.grid_matrix(L.LD_STENCIL_3D7, dims, k2, kappa2_field=field), 6, 32, tol,
                      L.options(precision=L.LD_MIXED))
    v, info = L.ld_logdet(ctx)
    col, nc = L.ld_get_colouring(ctx)
    checked_on_subbox(col, dims, 6)
    terms, _ = L.ld_column_terms(ctx)
    lo, hi = mt.spectral_bounds(om.KIND_3D7, dims, k2)
    s, a = hht.log_nodes(lo, hi, 32)
    pick = [0, nc // 2, nc - 1]
    ref = cf.probed_value(om.KIND_3D7, dims, k2, False, col, lambda lam: hht.f_N(lam, s, a),
                          per_colour=True, colours=pick)
    for c in pick:
        assert abs(terms[c] - ref[c]) <= 2e-5 * abs(ref[c]), c
    exact = cf.logdet(om.KIND_3D7, dims, k2, False)
    print("256^3: %d colours, %d iters, %.1f ms, logdet %.2f, exact %.2f (probing+quadrature rel %.2e)"
          % (nc, info["iters"], info["ms"], v, exact, (v - exact) / exact))


@pytest.mark.parametrize("prec", [L.LD_FP64, L.LD_MIXED])
def test_3d_seeded_field_exact_solves_and_gradient(prec):
    dims = (16, 14, 12)
    f = synth.kappa2_field(5, dims)
    tol = 1e-10 if prec == L.LD_FP64 else 1e-6
    ctx = L.ld_create(L.grid_matrix(L.LD_STENCIL_3D7, dims, 1.0, kappa2_field=f), 6, 32, tol,
                      L.options(precision=prec, keep_x0=1))
    v, g, info = L.ld_logdet_grad(ctx, [L.LD_P_KAPPA2])
    Q = om.precision(om.KIND_3D7, dims, f)
    col, _ = checked_colouring(ctx, Q, 6)
    lo, hi = mt.spectral_bounds(om.KIND_3D7, dims, f)
    s, a = hht.log_nodes(lo, hi, 32)
    ref = mt.probed_rational_band(Q, col, s, a, per_colour=True)
    terms, _ = L.ld_column_terms(ctx)
    if prec == L.LD_FP64:
        assert abs(v - ref.sum()) <= 50 * tol * np.abs(ref).sum()
    else:
        assert abs(v - ref.sum()) <= 2e-5 * abs(ref.sum())
    # d/dc of kappa^2 = c * field at c = 1: probed tr(Q^{-1} diag(field))
    V = probing.probing_vectors(col)
    X = sp.linalg.splu(Q.tocsc()).solve(V)
    gref = float(np.sum((f[:, None] * V) * X))
    assert abs(g[0] - gref) <= (1e-8 if prec == L.LD_FP64 else 2e-5) * abs(gref)


@pytest.mark.parametrize("prec", [L.LD_FP64, L.LD_MIXED])
@pytest.mark.parametrize("dims,per", [((33, 8, 6), False), ((9, 8, 7), True), ((64, 7, 4), False)])
def test_3d_streaming_engine_matches_exact_solves(dims, per, prec):
    """The multi-CTA engine on small 3D grids with a kappa^2 field and an observation mask,
    against exact banded shifted solves: FP64 through the stored-w plane-streaming kernel,
    mixed precision through the lean 3D pass (tiles of 4, the field and mask in its
    diagonal term, the seed solution kept for the gradient)."""
    n = int(np.prod(dims))
    f = synth.kappa2_field(6, dims)
    mask = synth.obs_mask(7, n, 0.1)
    fp64 = prec == L.LD_FP64
    tol = 1e-10 if fp64 else 1e-7
    ctx = L.ld_create(L.grid_matrix(L.LD_STENCIL_3D7, dims, 0.7, periodic=per, kappa2_field=f,
                                    tau=2.0, obs_mask=mask), 2, 20, tol,
                      L.options(precision=prec, engine=1, keep_x0=1, tile_width=0 if fp64 else 4))
    v, g, info = L.ld_logdet_grad(ctx, [L.LD_P_KAPPA2, L.LD_P_TAU])
    assert fp64 or info["pass_words"] == 6
    Q = om.precision(om.KIND_3D7, dims, 0.7 * f, periodic=per, tau=2.0, mask=mask)
    col, _ = checked_colouring(ctx, Q, 2)
    lo, hi = mt.spectral_bounds(om.KIND_3D7, dims, 0.7 * f, periodic=per, tau=2.0, mask=mask)
    s, a = hht.log_nodes(lo, hi, 20)
    if per:   # wrap-around entries make the band as wide as the matrix: dense route
        ref = np.array([mt.probed_dense(Q, col, lambda lam: hht.f_N(lam, s, a))])
    else:
        ref = mt.probed_rational_band(Q, col, s, a, per_colour=True)
    assert abs(v - ref.sum()) <= (50 * tol if fp64 else 2e-5) * np.abs(ref).sum()
    V = probing.probing_vectors(col)
    X = sp.linalg.splu(Q.tocsc()).solve(V)
    gbar = 1e-8 if fp64 else 2e-5
    assert abs(g[0] - float(np.sum((f[:, None] * V) * X))) <= gbar * abs(g[0])
    assert abs(g[1] - float(np.sum((mask[:, None] * V) * X))) <= gbar * abs(g[1])
