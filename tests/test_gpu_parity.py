"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

The method's target for a given colouring and node set is
    P_{d,N} = sum_c Re sum_l alpha_l v_c^T (Q - sigma_l I)^{-1} v_c
(Sec. 2.1, Eqs. "eq_logdet_ident" and "eq_rat_app"); the oracle computes it
with no Krylov error (spectral closed forms, dense or banded exact solves), so
the GPU result differs from it only by the CG stopping error.  Tolerances:
  FP64   |gpu - P| <= 50 * tol * sum_c |term_c|   (each shifted residual <= tol)
  mixed  |gpu - P| <= 2e-5 * |P|                  (FP32 vectors, FP64 scalars)
The exact log det (closed form / band Cholesky) and the probing and quadrature
errors are reported beside, not asserted against the CG tolerance.
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


def fN(sigma, alpha):
    return lambda lam: hht.f_N(lam, sigma, alpha)


def spectral_target(kind, dims, k2, per, col, sigma, alpha, scale=1.0, per_colour=False):
    return cf.probed_value(kind, dims, k2, per, col, fN(sigma, alpha), scale=scale,
                           per_colour=per_colour)


# ------------------------------------------------------------------ operator
@pytest.mark.parametrize("prec", [L.LD_FP64, L.LD_MIXED])
@pytest.mark.parametrize("kind,dims,per,ncols", [
    (om.KIND_2D5, (37, 23), False, 5),
    (om.KIND_2D5, (16, 9), True, 3),
    (om.KIND_2D5, (1, 7), True, 2),
    (om.KIND_2D13_SQ, (29, 31), False, 7),
    (om.KIND_2D13_SQ, (6, 5), True, 4),
    (om.KIND_2D13_SQ, (2, 3), True, 1),
    (om.KIND_3D7, (7, 6, 5), False, 9),
    (om.KIND_3D7, (4, 3, 5), True, 2),
])
def test_spmm_matches_sparse_matvec(prec, kind, dims, per, ncols):
    k2 = 0.37
    Q = om.precision(kind, dims, k2, periodic=per, scale=1.3)
    ctx = L.ld_create(L.grid_matrix(kind, dims, k2, periodic=per, scale=1.3), 1, 4, 1e-6,
                      L.options(precision=prec))
    X = synth.random_probe_block(3, Q.shape[0], ncols)
    Y = L.ld_apply(ctx, X)
    ref = Q @ X
    tol = 1e-13 if prec == L.LD_FP64 else 3e-6
    assert np.abs(Y - ref).max() <= tol * np.abs(ref).max()


@pytest.mark.parametrize("prec", [L.LD_FP64, L.LD_MIXED])
def test_spmm_field_mask_and_csr(prec):
    dims = (13, 11, 6)
    n = int(np.prod(dims))
    f = synth.kappa2_field(5, dims)
    mask = synth.obs_mask(4, n, 0.1)
    Q = om.precision(om.KIND_3D7, dims, 0.8 * f, tau=4.0, mask=mask)
    ctx = L.ld_create(L.grid_matrix(om.KIND_3D7, dims, 0.8, kappa2_field=f, tau=4.0, obs_mask=mask),
                      1, 4, 1e-6, L.options(precision=prec))
    X = synth.random_probe_block(4, n, 6)
    tol = 1e-13 if prec == L.LD_FP64 else 3e-6
    ref = Q @ X
    assert np.abs(L.ld_apply(ctx, X) - ref).max() <= tol * np.abs(ref).max()
    rows, cols, w = synth.random_sparse_spd_pattern(12, 500)
    rp, ci, vv = synth.csr_from_edges(500, rows, cols, w, 0.3)
    Qc = sp.csr_matrix((vv, ci, rp), shape=(500, 500))
    ctx2 = L.ld_create(L.csr_matrix(rp, ci, vv, scale=1.5), 1, 4, 1e-6,
                       L.options(precision=prec, lambda_min=0.1, lambda_max=40.0))
    X2 = synth.random_probe_block(5, 500, 5)
    ref2 = 1.5 * (Qc @ X2)
    assert np.abs(L.ld_apply(ctx2, X2) - ref2).max() <= tol * np.abs(ref2).max()


# ------------------------------------------------------------------ small periodic (64^2)
@pytest.mark.parametrize("engine", [1, 2])
def test_periodic_64_distance4_fp64(engine):
    dims, k2 = (64, 64), 0.5
    tol = 1e-10
    ctx = L.ld_create(L.grid_matrix(om.KIND_2D5, dims, k2, periodic=True), 4, 20, tol,
                      L.options(engine=engine))
    val, info = L.ld_logdet(ctx)
    col, nc = L.ld_get_colouring(ctx)
    Q = om.precision(om.KIND_2D5, dims, k2, periodic=True)
    assert np.array_equal(col, probing.colour_greedy(Q, 4))
    lo, hi = mt.spectral_bounds(om.KIND_2D5, dims, k2, periodic=True)
    s, a = hht.log_nodes(lo, hi, 20)
    target = spectral_target(om.KIND_2D5, dims, k2, True, col, s, a, per_colour=True)
    assert abs(val - target.sum()) <= 50 * tol * np.abs(target).sum()
    terms, seed = L.ld_column_terms(ctx)
    assert np.abs(terms - target).max() <= 50 * tol * np.abs(target).max()
    seed_ref = cf.probed_value(om.KIND_2D5, dims, k2, True, col, lambda x: 1 / x, per_colour=True)
    assert np.abs(seed - seed_ref).max() <= 50 * tol * np.abs(seed_ref).max()
    assert info["n_colours"] == 25 and info["engine"] == engine


def test_full_probing_equals_exact_logdet():
    """d >= diameter: one colour per vertex, the probed value is tr log Q exactly
    (Sec. 2.1, unit-vector trace); FP64 GPU within 1e-6 relative of the closed form."""
    dims, k2 = (64, 64), 0.5
    ctx = L.ld_create(L.grid_matrix(om.KIND_2D5, dims, k2, periodic=True), 64, 20, 1e-10)
    val, info = L.ld_logdet(ctx)
    assert info["n_colours"] == 4096
    exact = cf.logdet(om.KIND_2D5, dims, k2, True)
    assert abs(val - exact) <= 1e-6 * abs(exact)


def test_engines_agree_and_are_deterministic():
    dims, k2 = (48, 40), 0.2
    vals = []
    for eng in (1, 2, 1):
        ctx = L.ld_create(L.grid_matrix(om.KIND_2D13_SQ, dims, k2), 2, 16, 1e-9,
                          L.options(engine=eng))
        vals.append(L.ld_logdet(ctx)[0])
    assert vals[0] == vals[2]
    assert abs(vals[0] - vals[1]) <= 1e-11 * abs(vals[0])


# ------------------------------------------------------------------ Matern, Dirichlet
@pytest.mark.parametrize("prec,tol", [(L.LD_FP64, 1e-9), (L.LD_MIXED, 1e-6)])
@pytest.mark.parametrize("dims,k2", [((96, 80), 0.05), ((33, 47), 0.6)])
def test_matern_dirichlet(prec, tol, dims, k2):
    kind = om.KIND_2D13_SQ
    ctx = L.ld_create(L.grid_matrix(kind, dims, k2), 2, 20, tol, L.options(precision=prec))
    val, info = L.ld_logdet(ctx)
    col, _ = checked_colouring(ctx, om.precision(kind, dims, k2), 2)
    lo, hi = mt.spectral_bounds(kind, dims, k2)
    s, a = hht.log_nodes(lo, hi, 20)
    target = spectral_target(kind, dims, k2, False, col, s, a, per_colour=True)
    if prec == L.LD_FP64:
        assert abs(val - target.sum()) <= 50 * tol * np.abs(target).sum()
    else:
        assert abs(val - target.sum()) <= 2e-5 * abs(target.sum())


# ------------------------------------------------------------------ non-separable cases
@pytest.mark.parametrize("prec", [L.LD_FP64, L.LD_MIXED])
def test_3d_field_against_exact_shifted_solves(prec):
    dims = (10, 9, 8)
    f = synth.kappa2_field(5, dims)
    tol = 1e-10 if prec == L.LD_FP64 else 1e-6
    ctx = L.ld_create(L.grid_matrix(om.KIND_3D7, dims, 1.0, kappa2_field=f), 3, 24, tol,
                      L.options(precision=prec))
    val, info = L.ld_logdet(ctx)
    Q = om.precision(om.KIND_3D7, dims, f)
    col, _ = checked_colouring(ctx, Q, 3)
    lo, hi = mt.spectral_bounds(om.KIND_3D7, dims, f)
    s, a = hht.log_nodes(lo, hi, 24)
    target = mt.probed_rational_band(Q, col, s, a, per_colour=True)
    bound = 50 * tol * np.abs(target).sum() if prec == L.LD_FP64 else 2e-5 * abs(target.sum())
    assert abs(val - target.sum()) <= bound


def test_masked_posterior_against_exact_shifted_solves():
    dims = (40, 36)
    n = 1440
    mask = synth.obs_mask(4, n, 0.1)
    k2, tau, tol = 0.1, 4.0, 1e-10
    ctx = L.ld_create(L.grid_matrix(om.KIND_2D5, dims, k2, tau=tau, obs_mask=mask), 4, 20, tol)
    val, info = L.ld_logdet(ctx)
    Q = om.precision(om.KIND_2D5, dims, k2, tau=tau, mask=mask)
    col, _ = checked_colouring(ctx, Q, 4)
    lo, hi = mt.spectral_bounds(om.KIND_2D5, dims, k2, tau=tau, mask=mask)
    s, a = hht.log_nodes(lo, hi, 20)
    target = mt.probed_rational_band(Q, col, s, a, per_colour=True)
    assert abs(val - target.sum()) <= 50 * tol * np.abs(target).sum()


def test_csr_against_exact_shifted_solves():
    n = 600
    rows, cols, w = synth.random_sparse_spd_pattern(21, n)
    rp, ci, vv = synth.csr_from_edges(n, rows, cols, w, 0.2)
    Q = sp.csr_matrix((vv, ci, rp), shape=(n, n))
    ev = np.linalg.eigvalsh(Q.toarray())
    lo, hi = 0.9 * ev.min(), 1.1 * ev.max()
    tol = 1e-10
    ctx = L.ld_create(L.csr_matrix(rp, ci, vv), 2, 20, tol,
                      L.options(lambda_min=lo, lambda_max=hi))
    val, info = L.ld_logdet(ctx)
    col, _ = L.ld_get_colouring(ctx)
    assert np.array_equal(col, probing.colour_greedy(Q, 2))
    s, a = hht.log_nodes(lo, hi, 20)
    target = mt.probed_rational_band(Q, col, s, a, per_colour=True)
    assert abs(val - target.sum()) <= 50 * tol * np.abs(target).sum()
    # dense brute force of the same rational target
    dense = mt.probed_dense(Q, col, fN(s, a))
    assert abs(target.sum() - dense) <= 1e-10 * abs(dense)


# ------------------------------------------------------------------ partial sums, errors
def test_partial_colour_ranges_sum_to_total():
    dims = (50, 50)
    ctx = L.ld_create(L.grid_matrix(om.KIND_2D5, dims, 0.3), 4, 16, 1e-10)
    total, info = L.ld_logdet(ctx)
    C = info["n_colours"]
    cuts = [0, 3, 7, C]
    parts = [L.ld_logdet_partial(ctx, a, b)[0] for a, b in zip(cuts, cuts[1:])]
    assert abs(sum(parts) - total) <= 1e-14 * abs(total)     # per-column arithmetic is identical


def test_not_spd_reported_and_context_reusable():
    n = 200
    rows, cols, w = synth.random_sparse_spd_pattern(7, n)
    rp, ci, vv = synth.csr_from_edges(n, rows, cols, w, -3.0)   # shifted below zero
    ctx = L.ld_create(L.csr_matrix(rp, ci, vv), 1, 8, 1e-8, L.options(lambda_min=0.1, lambda_max=20))
    with pytest.raises(L.LogDetError) as e:
        L.ld_logdet(ctx)
    assert e.value.status == L.LD_ENOTSPD
    ok = L.ld_create(L.grid_matrix(om.KIND_2D5, (20, 20), 0.5), 2, 8, 1e-8)
    L.ld_logdet(ok)


def test_max_iter_reports_not_converged():
    ctx = L.ld_create(L.grid_matrix(om.KIND_2D13_SQ, (64, 64), 0.01), 2, 20, 1e-10,
                      L.options(max_iter=6, engine=1, chunk_iters=2))
    with pytest.raises(L.LogDetError) as e:
        L.ld_logdet(ctx)
    assert e.value.status == L.LD_ENOTCONV
    L.ld_set_params(ctx, 1.0)
    ctx2 = L.ld_create(L.grid_matrix(om.KIND_2D13_SQ, (64, 64), 1.0), 2, 20, 1e-10)
    L.ld_logdet(ctx2)


# ------------------------------------------------------------------ gradients
def test_gradient_kappa2_projected_and_stored_agree():
    dims, k2 = (64, 48), 0.2
    tol = 1e-10
    ctx = L.ld_create(L.grid_matrix(om.KIND_2D5, dims, k2), 4, 20, tol)
    v1, g1, _ = L.ld_logdet_grad(ctx, [L.LD_P_KAPPA2])
    ctx2 = L.ld_create(L.grid_matrix(om.KIND_2D5, dims, k2), 4, 20, tol, L.options(keep_x0=1))
    v2, _ = L.ld_logdet(ctx2)
    g2 = L.ld_grad(ctx2, [L.LD_P_KAPPA2, L.LD_P_SCALE])
    col, _ = checked_colouring(ctx, om.precision(om.KIND_2D5, dims, k2), 4)
    ref = cf.probed_value(om.KIND_2D5, dims, k2, False, col, lambda x: 1 / x)
    assert abs(g1[0] - ref) <= 1e-8 * abs(ref)
    assert abs(g2[0] - ref) <= 1e-8 * abs(ref)
    n = 64 * 48
    assert abs(g2[1] - n) <= 1e-8 * n          # d/ds log det(sQ) = n/s, probed exactly


def test_gradient_matern_and_mask_against_oracle():
    dims, k2 = (40, 33), 0.1
    tol = 1e-10
    ctx = L.ld_create(L.grid_matrix(om.KIND_2D13_SQ, dims, k2, scale=2.0), 2, 20, tol)
    _, g, _ = L.ld_logdet_grad(ctx, [L.LD_P_KAPPA2, L.LD_P_SCALE])
    col, _ = checked_colouring(ctx, om.precision(om.KIND_2D13_SQ, dims, k2), 2)
    # dQ/dkappa2 = 2 s Q1 shares Q's eigenvectors: probed sum 2 s lambda1 / (s lambda1^2)
    lam1 = lambda lam: np.sqrt(lam / 2.0)
    ref = cf.probed_value(om.KIND_2D13_SQ, dims, k2, False, col, lambda lam: 2.0 * 2.0 * lam1(lam) / lam,
                          scale=2.0)
    assert abs(g[0] - ref) <= 1e-8 * abs(ref)
    assert abs(g[1] - dims[0] * dims[1] / 2.0) <= 1e-8 * dims[0] * dims[1]
    # Gauss-linear posterior: d/dtau = probed tr(Q^-1 diag(mask)), exact solves
    dims2 = (36, 30)
    n2 = 1080
    mask = synth.obs_mask(4, n2, 0.1)
    ctx2 = L.ld_create(L.grid_matrix(om.KIND_2D5, dims2, 0.1, tau=4.0, obs_mask=mask), 4, 20, tol)
    _, g2, _ = L.ld_logdet_grad(ctx2, [L.LD_P_KAPPA2, L.LD_P_TAU])
    Q2 = om.precision(om.KIND_2D5, dims2, 0.1, tau=4.0, mask=mask)
    col2, _ = checked_colouring(ctx2, Q2, 4)
    V = probing.probing_vectors(col2)
    X = np.linalg.solve(Q2.toarray(), V)
    ref_k2 = float(np.sum(V * X))
    ref_tau = float(np.sum((mask[:, None] * V) * X))
    assert abs(g2[0] - ref_k2) <= 1e-8 * abs(ref_k2)
    assert abs(g2[1] - ref_tau) <= 1e-8 * abs(ref_tau)


def test_gradient_matches_finite_difference_of_logdet():
    dims, k2, h = (48, 48), 0.3, 1e-4
    tol = 1e-12
    ctx = L.ld_create(L.grid_matrix(om.KIND_2D5, dims, k2, periodic=True), 6, 24, tol)
    _, g, _ = L.ld_logdet_grad(ctx, [L.LD_P_KAPPA2])
    L.ld_set_params(ctx, k2 * (1 + h))
    up = L.ld_logdet(ctx)[0]
    L.ld_set_params(ctx, k2 * (1 - h))
    dn = L.ld_logdet(ctx)[0]
    fd = (up - dn) / (2 * k2 * h)
    assert abs(g[0] - fd) <= 1e-6 * abs(fd)


def test_autograd_backward_runs_native_gradient():
    import torch
    dims = (32, 32)
    mask = synth.obs_mask(9, 1024, 0.1)
    ctx = L.ld_create(L.grid_matrix(om.KIND_2D5, dims, 0.2, tau=2.0, obs_mask=mask), 4, 16, 1e-10,
                      L.options(keep_x0=1))
    k2 = torch.tensor(0.2, dtype=torch.float64, requires_grad=True)
    tau = torch.tensor(2.0, dtype=torch.float64, requires_grad=True)
    sc = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    out = L.LogDet.apply(ctx, k2, tau, sc)
    (3.0 * out).backward()
    ctx2 = L.ld_create(L.grid_matrix(om.KIND_2D5, dims, 0.2, tau=2.0, obs_mask=mask), 4, 16, 1e-10)
    v, g, _ = L.ld_logdet_grad(ctx2, [L.LD_P_KAPPA2, L.LD_P_TAU, L.LD_P_SCALE])
    assert abs(out.item() - v) <= 1e-12 * abs(v)
    assert abs(k2.grad.item() - 3 * g[0]) <= 1e-10 * abs(g[0])
    assert abs(tau.grad.item() - 3 * g[1]) <= 1e-10 * abs(g[1])
    assert abs(sc.grad.item() - 3 * 1024) <= 1e-6 * 1024


def test_bounded_device_wait_reports_timeout_and_context_stays_usable():
    """A device wait that nothing completes gives up after its limit and the host reads
    LD_ETIMEOUT; the device then runs an ordinary evaluation (failure path of the
    bulk-copy waits, tested without a fault)."""
    import time
    t0 = time.perf_counter()
    with pytest.raises(L.LogDetError) as e:
        L.ld_wait_selftest(50_000_000)          # 50 ms
    assert e.value.status == L.LD_ETIMEOUT
    assert time.perf_counter() - t0 < 5.0
    dims = (32, 32)
    Q = om.precision(om.KIND_2D5, dims, 0.5, periodic=True)
    col = probing.colour_greedy(Q, 2)
    ctx = L.ld_create(L.grid_matrix(om.KIND_2D5, dims, 0.5, periodic=True), 2, 24, 1e-10,
                      L.options(colouring=col))
    v, _ = L.ld_logdet(ctx)
    ref = cf.probed_value(om.KIND_2D5, dims, 0.5, True, col, np.log)
    assert abs(v - ref) <= 1e-7 * abs(ref)



@pytest.mark.parametrize("engine", [1, 2])
def test_periodic_64_as_csr_matches_closed_form_probing(engine):
    """The first configuration as given: kappa^2 I - Lap on the 64 x 64 torus as a general
    CSR matrix, distance 4, 20 shifts, tol 1e-10, FP64, against the spectral oracle."""
    dims, k2, tol = (64, 64), 0.5, 1e-10
    rows, cols, w = synth.torus_edges(*dims)
    rp, ci, vv = synth.csr_from_edges(4096, rows, cols, w, k2)
    Q = sp.csr_matrix((vv, ci, rp), shape=(4096, 4096))
    assert abs(Q - om.precision(om.KIND_2D5, dims, k2, periodic=True)).max() == 0
    col = probing.colour_greedy(Q, 4)
    ctx = L.ld_create(L.csr_matrix(rp, ci, vv), 4, 20, tol,
                      L.options(engine=engine, colouring=col, lambda_min=k2, lambda_max=k2 + 8.0))
    val, info = L.ld_logdet(ctx)
    s, a = hht.log_nodes(k2, k2 + 8.0, 20)
    target = spectral_target(om.KIND_2D5, dims, k2, True, col, s, a, per_colour=True)
    assert abs(val - target.sum()) <= 50 * tol * np.abs(target).sum()


def test_csr_with_library_bounds_matches_exact_probing():
    """A CSR matrix without user bounds: the library's interval (Gershgorin, Lanczos) must
    enclose the spectrum, so the result is the exact probed log det to the quadrature and
    CG accuracy (N = 24 shifts: certificate far below the CG tolerance)."""
    n = 600
    rows, cols, w = synth.random_sparse_spd_pattern(21, n)
    rp, ci, vv = synth.csr_from_edges(n, rows, cols, w, 0.2)
    Q = sp.csr_matrix((vv, ci, rp), shape=(n, n))
    col = probing.colour_greedy(Q, 2)
    ctx = L.ld_create(L.csr_matrix(rp, ci, vv), 2, 24, 1e-11, L.options(colouring=col))
    val, info = L.ld_logdet(ctx)
    ev = np.linalg.eigvalsh(Q.toarray())
    assert info["lambda_min"] <= ev.min() and info["lambda_max"] >= ev.max()
    ref = mt.probed_dense(Q, col, np.log)
    assert abs(val - ref) <= 1e-8 * abs(ref)


def test_automatic_shift_count_follows_the_interval():
    """n_shifts = 0: the context uses the node count ld_auto_shifts gives for its interval
    (the smallest N whose quadrature certificate meets 1e-10 |log M - log m|); the result
    is the oracle's rational target for that N, and a wider interval after ld_set_params
    raises N."""
    kind, dims, k2, tol = om.KIND_2D13_SQ, (96, 80), 0.05, 1e-9
    ctx = L.ld_create(L.grid_matrix(kind, dims, k2), 2, 0, tol, L.options(precision=L.LD_FP64))
    val, info = L.ld_logdet(ctx)
    N = info["n_shifts"]
    assert N == L.ld_auto_shifts(info["lambda_min"], info["lambda_max"])
    lo, hi = mt.spectral_bounds(kind, dims, k2)
    s, a = hht.log_nodes(lo, hi, N)
    col, _ = checked_colouring(ctx, om.precision(kind, dims, k2), 2)
    target = spectral_target(kind, dims, k2, False, col, s, a, per_colour=True)
    assert abs(val - target.sum()) <= 50 * tol * np.abs(target).sum()
    assert info["quad_cert"] <= 2e-10 * abs(np.log(hi) - np.log(lo))
    L.ld_set_params(ctx, 0.002)
    _, info2 = L.ld_logdet(ctx)
    assert info2["n_shifts"] > N
    assert info2["n_shifts"] == L.ld_auto_shifts(info2["lambda_min"], info2["lambda_max"])
