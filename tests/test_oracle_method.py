"""Pins for the oracle's colouring, rational nodes and multi-shift CG.

Each check is against something other than the oracle itself: closed-form
colourings, a brute-force distance pattern, scipy.linalg.logm, Jacobi-function
identities, dense complex solves, and the full-probing invariant
(Sec. 2.1: sum_j e_j^T log(Q) e_j = tr log Q).
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import closed_forms as cf
from oracle import hht
from oracle import matrices as om
from oracle import method as mt
from oracle import probing
from oracle.cgm import cgm


# ---------------------------------------------------------------- colouring
def path_graph(n):
    return sp.diags([np.full(n - 1, -1.0), np.full(n, 2.5), np.full(n - 1, -1.0)], [-1, 0, 1]).tocsr()


@pytest.mark.parametrize("d", [0, 1, 2, 3, 5])
def test_path_colouring_is_i_mod_d_plus_1(d):
    col = probing.colour_greedy(path_graph(23), d)
    assert np.array_equal(col, np.arange(23) % (d + 1))


def test_grid_distance_one_is_checkerboard():
    Q = om.precision(om.KIND_2D5, (9, 7), 0.5)
    col = probing.colour_greedy(Q, 1).reshape(7, 9)
    y, x = np.mgrid[0:7, 0:9]
    assert np.array_equal(col, (x + y) % 2)


def test_full_probing_when_distance_exceeds_diameter():
    Q = om.precision(om.KIND_2D5, (5, 4), 0.5)
    col = probing.colour_greedy(Q, 7)   # diameter = 4 + 3
    assert np.array_equal(np.sort(col), np.arange(20))


@pytest.mark.parametrize("kind,dims,per,d", [
    (om.KIND_2D5, (40, 33), False, 4),
    (om.KIND_2D5, (64, 64), True, 4),
    (om.KIND_2D13_SQ, (30, 31), False, 2),
    (om.KIND_3D7, (9, 8, 7), False, 3),
])
def test_colouring_valid_and_class_sum(kind, dims, per, d):
    Q = om.precision(kind, dims, 0.5, periodic=per)
    col = probing.colour_greedy(Q, d)
    assert probing.is_valid_colouring(Q, d, col)
    V = probing.probing_vectors(col)
    assert np.array_equal(V.sum(axis=1), np.ones(Q.shape[0]))


def test_colour_count_independent_of_grid_size():
    """Sec. 3: the number of colours barely depends on the discretisation."""
    counts = [int(probing.colour_greedy(om.precision(om.KIND_2D5, (s, s), 0.5), 4).max()) + 1
              for s in (32, 64, 128)]
    assert max(counts) - min(counts) <= 2


def test_invalid_colouring_detected():
    Q = om.precision(om.KIND_2D5, (6, 6), 0.5)
    col = probing.colour_greedy(Q, 2)
    col[7] = col[8]
    assert not probing.is_valid_colouring(Q, 2, col)


# ---------------------------------------------------------------- nodes
def test_jacobi_identities_complex():
    m = 0.37
    x = np.linspace(-1.5, 1.5, 11)
    sn, cn, dn = hht.jacobi_complex(x, 0.6, m)
    assert np.allclose(sn ** 2 + cn ** 2, 1, atol=1e-13)
    assert np.allclose(dn ** 2 + m * sn ** 2, 1, atol=1e-13)
    # d sn / dt = cn dn along the real direction
    e = 1e-6
    snp, _, _ = hht.jacobi_complex(x + e, 0.6, m)
    snm, _, _ = hht.jacobi_complex(x - e, 0.6, m)
    assert np.allclose((snp - snm) / (2 * e), cn * dn, atol=1e-8)


@pytest.mark.parametrize("N", [12, 20])
def test_rational_log_matches_logm(N):
    g = np.random.default_rng(0)
    B = g.standard_normal((40, 40))
    A = B @ B.T / 40 + 0.3 * np.eye(40)
    lam = np.linalg.eigvalsh(A)
    s, a = hht.log_nodes(lam.min(), lam.max(), N)
    F = sum(np.real(al * np.linalg.inv(A - si * np.eye(40))) for si, al in zip(s, a))
    err = np.abs(F - sla.logm(A)).max()
    assert err <= 200 * hht.rate_bound(lam.min(), lam.max(), N) + 1e-13


@pytest.mark.parametrize("m,M,N", [(0.5, 8.5, 8), (0.5, 8.5, 16), (1e-4, 64.2, 20),
                                   (1e-4, 64.2, 32), (0.01, 12.0, 10)])
def test_certificate_follows_two_pi_squared_rate(m, M, N):
    """Error decays like exp(-2 pi^2 N/(log(M/m)+6)) (constant < 200), far faster
    than the exp(-2 pi N/(...)) the paper prints."""
    s, a = hht.log_nodes(m, M, N)
    cert = hht.certificate(m, M, s, a)
    assert cert <= 200 * hht.rate_bound(m, M, N) + 2e-15
    printed = np.exp(-2 * np.pi * N / (np.log(M / m) + 6))
    assert cert < printed


def test_nodes_enclose_spectrum_and_avoid_negative_axis():
    s, a = hht.log_nodes(0.5, 8.5, 20)
    w = np.sqrt(s)
    assert np.all(np.imag(s) > 0)            # upper half of the contour
    assert np.all(np.real(w) > 0)


# ---------------------------------------------------------------- CG-M
def test_cgm_matches_dense_complex_solves():
    Q = om.precision(om.KIND_2D5, (10, 9), 0.5)
    A = Q.toarray()
    lmin, lmax = mt.spectral_bounds(om.KIND_2D5, (10, 9), 0.5)
    sigma, alpha = hht.log_nodes(lmin, lmax, 12)
    g = np.random.default_rng(1)
    v = (g.random(90) < 0.2).astype(float)
    res = cgm(Q.dot, v, -sigma, 1e-13, 1000, keep_vectors=True)
    for l, sg in enumerate(sigma):
        x = np.linalg.solve(A - sg * np.eye(90), v.astype(complex))
        assert np.abs(res["xs"][l] - x).max() <= 1e-10 * np.abs(x).max()
        assert abs(res["pi"][l] - v @ x) <= 1e-10 * abs(v @ x)
    x0 = np.linalg.solve(A, v)
    assert np.abs(res["x0"] - x0).max() <= 1e-10 * np.abs(x0).max()


def test_cgm_projected_equals_vector_form():
    Q = om.precision(om.KIND_2D13_SQ, (12, 11), 0.1)
    lmin, lmax = mt.spectral_bounds(om.KIND_2D13_SQ, (12, 11), 0.1)
    sigma, _ = hht.log_nodes(lmin, lmax, 16)
    v = np.zeros(132)
    v[::7] = 1.0
    res = cgm(Q.dot, v, -sigma, 1e-12, 5000, keep_vectors=True)
    proj_from_vec = res["xs"] @ v
    assert np.abs(res["pi"] - proj_from_vec).max() <= 1e-11 * np.abs(proj_from_vec).max()


def test_cgm_detects_indefinite():
    from oracle.cgm import NotSPD
    A = sp.diags([1.0, 2.0, -1.0]).tocsr()
    with pytest.raises(NotSPD):
        cgm(A.dot, np.ones(3), np.array([0.1 + 0.1j]), 1e-10, 100)


def test_spectral_bounds_enclose_closed_form_spectrum():
    for kind, dims, per in [(om.KIND_2D5, (64, 64), True), (om.KIND_2D5, (31, 17), False),
                            (om.KIND_2D13_SQ, (40, 40), False), (om.KIND_3D7, (7, 6, 5), False)]:
        lo, hi = mt.spectral_bounds(kind, dims, 0.2, periodic=per)
        elo, ehi = cf.extreme_eigs(kind, dims, 0.2, per)
        assert lo <= elo * (1 + 1e-12) and hi >= ehi * (1 - 1e-12)
        assert abs(lo - elo) <= 1e-12 * elo and abs(hi - ehi) <= 1e-12 * ehi


# ---------------------------------------------------------------- method end to end
def test_full_probing_method_equals_exact_logdet():
    """d >= diameter gives unit vectors: the probed value is tr log Q exactly; the
    method then differs only by quadrature and CG tolerance."""
    dims = (6, 5)
    Q = om.precision(om.KIND_2D5, dims, 0.5)
    col = probing.colour_greedy(Q, 20)
    lo, hi = mt.spectral_bounds(om.KIND_2D5, dims, 0.5)
    res = mt.logdet_method(Q, col, lo, hi, 20, 1e-12)
    exact = cf.logdet(om.KIND_2D5, dims, 0.5, False)
    assert abs(res["logdet"] - exact) <= 1e-9 * abs(exact)


def test_method_equals_exact_rational_target():
    """CG-M probed value == exact banded solves of the same shifted systems."""
    dims = (16, 14)
    mask = np.zeros(224, np.uint8)
    mask[::9] = 1
    Q = om.precision(om.KIND_2D5, dims, 0.1, tau=4.0, mask=mask)
    col = probing.colour_greedy(Q, 4)
    lo, hi = mt.spectral_bounds(om.KIND_2D5, dims, 0.1, tau=4.0, mask=mask)
    res = mt.logdet_method(Q, col, lo, hi, 20, 1e-12, per_colour=True)
    exact_terms = mt.probed_rational_band(Q, col, res["sigma"], res["alpha"], per_colour=True)
    assert np.abs(res["terms"] - exact_terms).max() <= 1e-9 * np.abs(exact_terms).max()
    # and the rational target is within quadrature error of the exact probed log
    pd = mt.probed_dense(Q, col, np.log)
    cert = hht.certificate(lo, hi, res["sigma"], res["alpha"])
    assert abs(float(exact_terms.sum()) - pd) <= 224 * cert + 1e-9


def test_probing_error_shrinks_with_distance():
    """Sec. 3 / Table 1 trend: larger colouring distance, closer to exact."""
    dims = (48, 48)
    Q = om.precision(om.KIND_2D5, dims, 0.05, periodic=True)
    exact = cf.logdet(om.KIND_2D5, dims, 0.05, True)
    errs = []
    for d in (2, 4, 6, 8):
        col = probing.colour_greedy(Q, d)
        errs.append(abs(cf.probed_value(om.KIND_2D5, dims, 0.05, True, col, np.log) - exact))
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:]))


def test_banded_shifted_solves_equal_dense_rational_target():
    """Complex-symmetric banded LDL^T quadratic forms == dense eigendecomposition of f_N."""
    n = 150
    import synth
    rows, cols, w = synth.random_sparse_spd_pattern(31, n)
    rp, ci, vv = synth.csr_from_edges(n, rows, cols, w, 0.4)
    Q = sp.csr_matrix((vv, ci, rp), shape=(n, n))
    ev = np.linalg.eigvalsh(Q.toarray())
    sigma, alpha = hht.log_nodes(0.9 * ev.min(), 1.1 * ev.max(), 16)
    col = probing.colour_greedy(Q, 2)
    band = mt.probed_rational_band(Q, col, sigma, alpha)
    dense = mt.probed_dense(Q, col, lambda lam: hht.f_N(lam, sigma, alpha))
    assert abs(band - dense) <= 1e-11 * abs(dense)


@pytest.mark.parametrize("case", ["posterior2d", "field3d", "matern_periodic"])
def test_sparse_lu_rational_target_equals_banded_and_dense(case):
    """SuperLU shifted solves give the same rational target as the plain-C banded
    LDL^T (an independent factorisation and ordering) and as dense eigh of f_N."""
    import synth
    if case == "posterior2d":
        dims, kind, per = (30, 26), om.KIND_2D5, False
        n = 780
        mask = synth.obs_mask(4, n, 0.1)
        Q = om.precision(kind, dims, 0.1, tau=4.0, mask=mask)
        lo, hi = mt.spectral_bounds(kind, dims, 0.1, tau=4.0, mask=mask)
        d = 4
    elif case == "field3d":
        dims, kind, per = (7, 6, 5), om.KIND_3D7, False
        f = synth.kappa2_field(5, dims)
        Q = om.precision(kind, dims, f)
        lo, hi = mt.spectral_bounds(kind, dims, f)
        d = 3
    else:
        dims, kind, per = (12, 10), om.KIND_2D13_SQ, True
        Q = om.precision(kind, dims, 0.2, periodic=True)
        lo, hi = mt.spectral_bounds(kind, dims, 0.2, periodic=True)
        d = 2
    col = probing.colour_greedy(Q, d)
    sigma, alpha = hht.log_nodes(lo, hi, 20)
    lu = mt.probed_rational_splu(Q, col, sigma, alpha, per_colour=True)
    dense_total = mt.probed_dense(Q, col, lambda lam: hht.f_N(lam, sigma, alpha))
    assert abs(lu.sum() - dense_total) <= 1e-11 * abs(dense_total)
    if not per:   # wrap-around entries make the band as wide as the matrix
        band = mt.probed_rational_band(Q, col, sigma, alpha, per_colour=True)
        assert np.abs(lu - band).max() <= 1e-11 * np.abs(band).max()


def test_method_on_a_subset_of_colours_equals_exact_solves():
    """CG-M run for chosen probing vectors only: each chosen term equals the exact
    rational target's term, the skipped ones are NaN and the seed projections are
    v_c^T Q^{-1} v_c from a sparse LU solve."""
    import synth
    dims = (20, 18)
    n = 360
    f = synth.kappa2_field(9, dims)
    Q = om.precision(om.KIND_2D5, dims, f)
    col = probing.colour_greedy(Q, 3)
    lo, hi = mt.spectral_bounds(om.KIND_2D5, dims, f)
    pick = [0, 5, int(col.max())]
    res = mt.logdet_method(Q, col, lo, hi, 20, 1e-13, per_colour=True, colours=pick)
    exact = mt.probed_rational_band(Q, col, res["sigma"], res["alpha"], per_colour=True)
    V = probing.probing_vectors(col)
    X = sp.linalg.splu(Q.tocsc()).solve(V)
    seeds = np.sum(V * X, axis=0)
    for c in pick:
        assert abs(res["terms"][c] - exact[c]) <= 1e-10 * abs(exact[c])
        assert abs(res["seeds"][c] - seeds[c]) <= 1e-10 * abs(seeds[c])
    skipped = [c for c in range(int(col.max()) + 1) if c not in pick]
    assert np.all(np.isnan(res["terms"][skipped]))
    assert abs(res["logdet"] - exact[pick].sum()) <= 1e-10 * np.abs(exact[pick]).sum()


@pytest.mark.parametrize("what", ["field", "mask", "both"])
@pytest.mark.parametrize("kind,dims,per", [(om.KIND_2D5, (9, 7), False), (om.KIND_2D5, (8, 6), True),
                                          (om.KIND_3D7, (5, 4, 6), False),
                                          (om.KIND_2D13_SQ, (7, 9), False)])
def test_spectral_bounds_enclose_field_and_mask_spectrum(kind, dims, per, what):
    """With a kappa^2 field and/or an observation mask the interval [m, M] must still
    enclose the spectrum (dense eigvalsh), and each end must lie within the field's
    spread (plus tau) of it.  A bound built from the wrong end of the field, or one
    that drops the mask's tau, fails one of the two."""
    import synth
    if kind == om.KIND_2D13_SQ and what != "field":
        pytest.skip("the Matern kind has no observation term")
    n = int(np.prod(dims))
    f = 0.6 * synth.kappa2_field(11, dims, sd=2.0) if what != "mask" else np.full(n, 0.3)
    mask = synth.obs_mask(12, n, 0.5) if what != "field" else None
    tau = 10.0 if mask is not None else 0.0
    Q = om.precision(kind, dims, f, periodic=per, tau=tau, mask=mask)
    ev = np.linalg.eigvalsh(Q.toarray())
    lo, hi = mt.spectral_bounds(kind, dims, f, periodic=per, tau=tau, mask=mask)
    assert lo <= ev.min() * (1 + 1e-12) and ev.max() <= hi * (1 + 1e-12)
    spread = f.max() - f.min() + tau
    if kind == om.KIND_2D13_SQ:   # bounds of the square: compare square roots
        assert np.sqrt(lo) >= np.sqrt(ev.min()) - spread and np.sqrt(hi) <= np.sqrt(ev.max()) + spread
    else:
        assert lo >= ev.min() - spread and hi <= ev.max() + spread


# ---------------------------------------------------------------- distance selection
@pytest.mark.parametrize("kind,dims,per", [(om.KIND_2D5, (12, 10), False), (om.KIND_2D5, (9, 8), True),
                                          (om.KIND_2D13_SQ, (11, 9), False)])
def test_log_column_matches_dense_logm(kind, dims, per):
    Q = om.precision(kind, dims, 0.3, periodic=per)
    L = sla.logm(Q.toarray()).real
    for j in (0, 17, Q.shape[0] - 1):
        assert np.abs(cf.log_column(kind, dims, 0.3, per, j) - L[:, j]).max() <= 1e-12


@pytest.mark.parametrize("kind,dims,per", [(om.KIND_2D5, (13, 11), False), (om.KIND_2D5, (10, 9), True),
                                          (om.KIND_2D13_SQ, (12, 10), False), (om.KIND_3D7, (6, 5, 4), False)])
def test_graph_distances_are_lattice_distances(kind, dims, per):
    """Graph distance on the lattice = (torus) L1 distance for 5/7 points, ceil(L1/2) for
    the 13-point square."""
    Q = om.precision(kind, dims, 0.3, periodic=per)
    j = Q.shape[0] // 2 + 1
    dist = probing.graph_distances(Q, j, 50)
    coords = np.array(np.unravel_index(np.arange(Q.shape[0]), tuple(reversed(dims)))).T
    cj = coords[j]
    diff = np.abs(coords - cj)
    if per:
        diff = np.minimum(diff, np.array(tuple(reversed(dims))) - diff)
    l1 = diff.sum(axis=1)
    ref = (l1 + 1) // 2 if kind == om.KIND_2D13_SQ else l1
    assert np.array_equal(dist, ref)


def test_decay_distance_definition_on_a_path():
    """Path graph: y_l = 10^-|l-j|; the first vertex below eps sits at distance ceil(-log10 eps)."""
    n, j = 30, 12
    Q = path_graph(n)
    dist = probing.graph_distances(Q, j, n)
    y = 10.0 ** (-np.abs(np.arange(n) - j))
    for eps, p in ((0.5, 1), (1e-3 * 1.5, 3), (1e-6 * 0.99, 7)):
        assert probing.decay_distance(y, dist, j, eps) == p
    prof = probing.decay_profile(y, dist, j, 5)
    assert np.allclose(prof, 10.0 ** -np.arange(6))
    assert probing.decay_distance(y, dist, j, 1e-40) == -1



# ---------------------------------------------------------------- Hutchinson (Eq. "eq_est_eq")
def test_quadratic_forms_match_dense_logm():
    import synth
    for kind, dims, per in ((om.KIND_2D5, (11, 9), True), (om.KIND_2D13_SQ, (10, 8), False)):
        Q = om.precision(kind, dims, 0.4, periodic=per)
        Z = synth.rademacher_block(3, Q.shape[0], 5)
        ref = np.einsum("ik,ij,jk->k", Z, sla.logm(Q.toarray()).real, Z)
        assert np.abs(cf.quadratic_forms(kind, dims, 0.4, per, Z) - ref).max() <= 1e-10 * np.abs(ref).max()


def test_hutchinson_is_unbiased_on_average():
    """E[z^T log(Q) z] = tr log Q for Rademacher z: the mean over many draws approaches it."""
    import synth
    dims = (16, 16)
    Z = synth.rademacher_block(4, 256, 4000)
    q = cf.quadratic_forms(om.KIND_2D5, dims, 0.5, True, Z)
    exact = cf.logdet(om.KIND_2D5, dims, 0.5, True)
    assert abs(q.mean() - exact) <= 4 * q.std() / np.sqrt(q.size)



# ---------------------------------------------------------------- sampling and likelihood
@pytest.mark.parametrize("N", [16, 24])
def test_invsqrt_nodes_match_dense_inverse_sqrt(N):
    g = np.random.default_rng(5)
    B = g.standard_normal((30, 30))
    A = B @ B.T / 30 + 0.2 * np.eye(30)
    lam, U = np.linalg.eigh(A)
    s, b = hht.invsqrt_nodes(lam.min(), lam.max(), N)
    F = sum(np.real(bb * np.linalg.inv(A - ss * np.eye(30))) for ss, bb in zip(s, b))
    ref = U @ np.diag(lam ** -0.5) @ U.T
    cert = hht.invsqrt_certificate(lam.min(), lam.max(), s, b)
    assert np.abs(F - ref).max() <= 10 * cert * np.abs(ref).max() + 1e-13
    assert cert <= 200 * hht.rate_bound(lam.min(), lam.max(), N) + 1e-15
    # same poles as the log approximation
    s2, _ = hht.log_nodes(lam.min(), lam.max(), N)
    assert np.allclose(s, s2, rtol=0, atol=1e-14 * np.abs(s2).max())


def test_apply_function_matches_dense():
    dims = (9, 7)
    Q = om.precision(om.KIND_2D13_SQ, dims, 0.3)
    lam, U = np.linalg.eigh(Q.toarray())
    V = np.random.default_rng(2).standard_normal((63, 3))
    ref = U @ np.diag(lam ** -0.5) @ U.T @ V
    got = cf.apply_function(om.KIND_2D13_SQ, dims, 0.3, False, V, lambda x: x ** -0.5)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_gaussian_loglik_matches_dense_formula():
    from scipy.stats import multivariate_normal
    dims = (6, 5)
    Q = om.precision(om.KIND_2D5, dims, 0.7, scale=2.0)
    Y = np.random.default_rng(8).standard_normal((30, 2))
    ref = sum(multivariate_normal(np.zeros(30), np.linalg.inv(Q.toarray())).logpdf(Y[:, k]) for k in range(2))
    assert abs(mt.gaussian_loglik(Q, Y) - ref) <= 1e-10 * abs(ref)
