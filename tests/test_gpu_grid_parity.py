"""GPU parity of the multi-CTA grid engine on the posterior, field and 3D workloads.

Every case here forces the grid engine (engine = 1: the lattice-streaming pass kernels
with their tile-group graphs), the path the bench times, and compares it with the
oracle element by element:

  * Gauss-linear posterior Q_p = kappa^2 I - Lap + tau diag(mask) (Sec. 1), 10 % of the
    nodes observed, at 256^2 and 512^2: per-colour terms against the exact rational
    target (sparse-LU shifted solves), the seed projections v_c^T Q^{-1} v_c and both
    gradients (kappa^2, tau) against exact probed traces, in FP64 and in mixed
    precision with reliable updates and the kept seed solution;
  * a 2D kappa^2 field (log kappa^2 = -2 + smoothed N(0,1), 5^2 box), Dirichlet and
    periodic, with the gradient with respect to the field's scale;
  * the 3D 7-point kappa^2 field at 32^3, distance 6, N = 32: every colour's term
    against the oracle's CG-M method reference (O4) run to 1e-12, the gradient
    against exact sparse solves, and the exact log det (band Cholesky, O1) beside;
  * the 2048^2 posterior in the bench's launch configuration (mixed, reliable
    updates, tol 1e-9, gradient): sampled colours against O4 run to 1e-12.

Tolerances (the parity bar of every GPU test): FP64 |term - ref| <= 50 tol max|ref|
elementwise and 50 tol sum|ref| for the total; mixed precision 2e-5 relative.  The
per-colour seed projections v_c^T x_c that ld_column_terms reports are the FP64 scalar
recurrence pi_0 += alpha_k v^T p_k driven by the CG's own recursion, so in mixed
precision they carry the FP32 recursion's drift (measured 1e-7 to 6e-7 relative, with or
without reliable updates) and are held to the mixed bar; the gradients of the mixed
runs with reliable updates come from the kept FP64 seed solution x_hi and meet exact
probed traces to 1e-7 (FP64: 1e-8).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import paper_1105_5256_gb300 as L
import synth
from oracle import hht
from oracle import matrices as om
from oracle import method as mt
from oracle import probing
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


def exact_traces(Q, col, diags):
    """Probed traces sum_c (E v_c)^T Q^{-1} v_c for diagonal E = diag(e) (e in diags),
    and the per-colour seed projections v_c^T Q^{-1} v_c, from a sparse LU of Q."""
    V = probing.probing_vectors(col)
    X = spla.splu(Q.tocsc(), permc_spec="MMD_AT_PLUS_A").solve(V)
    seeds = np.sum(V * X, axis=0)
    return seeds, [float(np.sum((np.asarray(e, float)[:, None] * V) * X)) for e in diags]


def check_terms(prec, tol, terms, val, ref):
    if prec == L.LD_FP64:
        assert np.abs(terms - ref).max() <= 50 * tol * np.abs(ref).max()
        assert abs(val - ref.sum()) <= 50 * tol * np.abs(ref).sum()
    else:
        assert np.abs(terms - ref).max() <= 2e-5 * np.abs(ref).max()
        assert abs(val - ref.sum()) <= 2e-5 * abs(ref.sum())


# ------------------------------------------------------------------ posterior, 256^2 / 512^2
_POSTERIOR = {}


def posterior_oracle(side):
    """Exact per-colour rational targets, seed projections and probed traces of the
    seeded posterior on a side x side grid (cached: shared by both precisions)."""
    if side in _POSTERIOR:
        return _POSTERIOR[side]
    dims, k2, tau = (side, side), 0.1, 4.0
    n = side * side
    mask = synth.obs_mask(4, n, 0.1)
    Q = om.precision(om.KIND_2D5, dims, k2, tau=tau, mask=mask)
    col = probing.colour_greedy(Q, 4)
    lo, hi = mt.spectral_bounds(om.KIND_2D5, dims, k2, tau=tau, mask=mask)
    s, a = hht.log_nodes(lo, hi, 20)
    terms = mt.probed_rational_splu(Q, col, s, a, per_colour=True)
    seeds, (g_k2, g_tau) = exact_traces(Q, col, [np.ones(n), mask])
    _POSTERIOR[side] = dict(Q=Q, col=col, mask=mask, terms=terms, seeds=seeds, grad=(g_k2, g_tau),
                            k2=k2, tau=tau, dims=dims)
    return _POSTERIOR[side]


@pytest.mark.parametrize("mode", ["fp64", "mixed_reliable"])
@pytest.mark.parametrize("side", [256, 512])
def test_posterior_grid_engine_against_exact_solves(side, mode):
    o = posterior_oracle(side)
    if mode == "fp64":
        prec, tol, opts = L.LD_FP64, 1e-10, dict(keep_x0=0)
    else:
        prec, tol, opts = L.LD_MIXED, 1e-9, dict(keep_x0=1, reliable_delta=1e-2)
    ctx = L.ld_create(L.grid_matrix(L.LD_STENCIL_2D5, o["dims"], o["k2"], tau=o["tau"],
                                    obs_mask=o["mask"]), 4, 20, tol,
                      L.options(precision=prec, engine=1, **opts))
    val, g, info = L.ld_logdet_grad(ctx, [L.LD_P_KAPPA2, L.LD_P_TAU])
    assert info["engine"] == 1 and info["bulk_rows"] in (0, 1)
    checked_colouring(ctx, o["Q"], 4)
    terms, seeds = L.ld_column_terms(ctx)
    check_terms(prec, tol, terms, val, o["terms"])
    rel = 1e-8 if prec == L.LD_FP64 else 1e-7
    srel = 1e-8 if prec == L.LD_FP64 else 2e-5
    assert np.abs(seeds - o["seeds"]).max() <= srel * np.abs(o["seeds"]).max()
    for got, ref in zip(g, o["grad"]):
        assert abs(got - ref) <= rel * abs(ref)
    if mode == "mixed_reliable":
        assert info["reliable_updates"] >= 1 and info["rel_resid_max"] <= 10 * tol
    print("posterior %d^2 %s: logdet %.6f (target %.6f), grad %s, %d iters, %d reliable updates"
          % (side, mode, val, o["terms"].sum(), g, info["iters"], info["reliable_updates"]))


# ------------------------------------------------------------------ 2D kappa^2 field
@pytest.mark.parametrize("prec", [L.LD_FP64, L.LD_MIXED])
@pytest.mark.parametrize("dims,per", [((300, 200), False), ((128, 96), True)])
def test_2d_kappa2_field_grid_engine(dims, per, prec):
    n = dims[0] * dims[1]
    f = synth.kappa2_field(8, dims)
    c = 0.7
    tol = 1e-10 if prec == L.LD_FP64 else 1e-6
    ctx = L.ld_create(L.grid_matrix(L.LD_STENCIL_2D5, dims, c, periodic=per, kappa2_field=f), 4, 20,
                      tol, L.options(precision=prec, engine=1, keep_x0=1))
    val, g, info = L.ld_logdet_grad(ctx, [L.LD_P_KAPPA2])
    assert info["engine"] == 1
    Q = om.precision(om.KIND_2D5, dims, c * f, periodic=per)
    col, _ = checked_colouring(ctx, Q, 4)
    lo, hi = mt.spectral_bounds(om.KIND_2D5, dims, c * f, periodic=per)
    s, a = hht.log_nodes(lo, hi, 20)
    ref = mt.probed_rational_splu(Q, col, s, a, per_colour=True)
    terms, _ = L.ld_column_terms(ctx)
    check_terms(prec, tol, terms, val, ref)
    _, (gref,) = exact_traces(Q, col, [f])      # d/dc of kappa^2 = c f: probed tr(Q^{-1} diag f)
    assert abs(g[0] - gref) <= (1e-8 if prec == L.LD_FP64 else 2e-5) * abs(gref)


# ------------------------------------------------------------------ 3D field, 32^3
_FIELD32 = {}


def field32_oracle():
    if _FIELD32:
        return _FIELD32
    dims = (32, 32, 32)
    f = synth.kappa2_field(5, dims)
    Q = om.precision(om.KIND_3D7, dims, f)
    col = probing.colour_greedy(Q, 6)
    lo, hi = mt.spectral_bounds(om.KIND_3D7, dims, f)
    o4 = mt.logdet_method(Q, col, lo, hi, 32, 1e-12, per_colour=True)
    _, (gref,) = exact_traces(Q, col, [f])
    _FIELD32.update(dims=dims, f=f, Q=Q, col=col, terms=o4["terms"], grad=gref,
                    exact=mt.exact_logdet_band(Q))
    return _FIELD32


@pytest.mark.parametrize("prec", [L.LD_FP64, L.LD_MIXED])
def test_3d_field_32cube_every_colour(prec):
    """configs' 3D non-stationary model at 32^3 with the full seeded field (d = 6,
    N = 32): every colour against the oracle's CG-M reference, the gradient with
    respect to the field scale against exact solves, the exact log det beside."""
    o = field32_oracle()
    tol = 1e-10 if prec == L.LD_FP64 else 1e-6
    ctx = L.ld_create(L.grid_matrix(L.LD_STENCIL_3D7, o["dims"], 1.0, kappa2_field=o["f"]), 6, 32,
                      tol, L.options(precision=prec, engine=1, keep_x0=1))
    val, g, info = L.ld_logdet_grad(ctx, [L.LD_P_KAPPA2])
    assert info["engine"] == 1
    checked_colouring(ctx, o["Q"], 6)
    terms, _ = L.ld_column_terms(ctx)
    check_terms(prec, tol, terms, val, o["terms"])
    assert abs(g[0] - o["grad"]) <= (1e-8 if prec == L.LD_FP64 else 2e-5) * abs(o["grad"])
    # probing + quadrature error against the exact log det: reported, and small
    err = (val - o["exact"]) / o["exact"]
    print("32^3 field: %d colours, logdet %.6f, exact %.6f (probing+quadrature rel %.2e), %d iters"
          % (len(terms), val, o["exact"], err, info["iters"]))
    assert abs(err) < 1e-2


# ------------------------------------------------------------------ 2048^2, bench configuration
_P2048 = {}


def posterior2048_oracle():
    if _P2048:
        return _P2048
    dims, k2, tau = (2048, 2048), 0.1, 4.0
    n = dims[0] * dims[1]
    mask = synth.obs_mask(4, n, 0.1)
    Q = om.precision(om.KIND_2D5, dims, k2, tau=tau, mask=mask)
    col = probing.colour_greedy(Q, 4)
    C = int(col.max()) + 1
    pick = [0, C // 2, C - 1]
    lo, hi = mt.spectral_bounds(om.KIND_2D5, dims, k2, tau=tau, mask=mask)
    o4 = mt.logdet_method(Q, col, lo, hi, 20, 1e-12, per_colour=True, colours=pick)
    _P2048.update(dims=dims, k2=k2, tau=tau, mask=mask, Q=Q, col=col, pick=pick,
                  terms=o4["terms"], seeds=o4["seeds"])
    return _P2048


@pytest.mark.parametrize("prec", [L.LD_MIXED, L.LD_FP64])
def test_posterior_2048_sampled_colours_against_cgm_reference(prec):
    """The 2048^2 posterior as the bench runs it (mixed: reliable updates, tol 1e-9,
    gradient; FP64 beside): three sampled colours' terms and seed projections against
    the oracle's CG-M run to 1e-12 on the same probing vectors."""
    o = posterior2048_oracle()
    tol = 1e-9
    opts = dict(reliable_delta=1e-2) if prec == L.LD_MIXED else {}
    ctx = L.ld_create(L.grid_matrix(L.LD_STENCIL_2D5, o["dims"], o["k2"], tau=o["tau"],
                                    obs_mask=o["mask"]), 4, 20, tol,
                      L.options(precision=prec, keep_x0=1, **opts))
    val, g, info = L.ld_logdet_grad(ctx, [L.LD_P_KAPPA2, L.LD_P_TAU])
    assert info["engine"] == 1
    col, _ = L.ld_get_colouring(ctx)
    assert np.array_equal(col, o["col"])
    terms, seeds = L.ld_column_terms(ctx)
    for c in o["pick"]:
        ref, sref = o["terms"][c], o["seeds"][c]
        if prec == L.LD_FP64:
            assert abs(terms[c] - ref) <= 50 * tol * abs(ref), c
            assert abs(seeds[c] - sref) <= 1e-8 * abs(sref), c
        else:
            assert abs(terms[c] - ref) <= 2e-5 * abs(ref), c
            assert abs(seeds[c] - sref) <= 2e-5 * abs(sref), c
    print("2048^2 posterior (%s): logdet %.4f, %d iters, sampled colours %s ok"
          % ("mixed" if prec == L.LD_MIXED else "fp64", val, info["iters"], o["pick"]))
