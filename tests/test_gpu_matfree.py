"""GPU parity of the matrix-free operator path (ld_create_matfree): the caller supplies
only W = Q P (Sec. 1: the method touches Q through products), the library runs CG with
the projected multi-shift recurrences of Sec. 2.1 in its own kernels.

The caller's product here is a dense torch matmul of the oracle's matrix.  Targets:
  * the exact probed value P_d = sum_c v_c^T log(Q) v_c from dense eigh (oracle), with the
    oracle's greedy colouring: |mf - P_d| <= 50 tol sum_c |term_c| + 100 n rate(M/m, N)
    (the CG stopping error and the quadrature bound, as the CSR parity tests);
  * per-colour terms against the oracle's rational target on the same nodes, and the
    seed projections v_c^T Q^{-1} v_c against dense solves;
  * the fused CSR path on the same colouring and interval, to the same tolerance;
  * the gradient sum_c v_c^T E_j Q^{-1} v_c through the caller's derivative products
    (E_j = dQ/d eta_j) against dense solves, and ld_grad on kept seed solutions;
  * the vector form log(Q) V and Q^{-1/2} V against dense eigh of the rational functions.
Error paths: a failing callback, an operator that is not SPD, max_iter, a gradient
without derivative products, and the entry points a matrix-free context does not support.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import paper_1105_5256_gb300 as L
import synth
from oracle import hht
from oracle import matrices as om
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


def dense_matvec(Q, sign=1.0):
    import torch
    Qd = torch.tensor(sign * Q.toarray(), dtype=torch.float64, device="cuda")

    def mv(P, W):
        torch.matmul(Qd, P, out=W)
    return mv


def exact_terms(Q, colour, f=np.log):
    lam, U = np.linalg.eigh(Q.toarray())
    F = (U * f(lam)) @ U.T
    return np.array([F[np.ix_(i, i)].sum() for i in
                     (np.nonzero(colour == c)[0] for c in range(int(colour.max()) + 1))]), lam


def mesh_problem(alpha, k2, d):
    p, t = synth.perturbed_triangulation(3, 31, 27)
    Q = om.fem_spde_precision(p, t, k2, alpha)
    return Q, probing.colour_greedy(Q, d)


@pytest.mark.parametrize("alpha,k2,d", [(1, 10.0, 2), (2, 10.0, 1), (1, 0.5, 3)])
def test_matfree_matches_exact_probing_and_csr_path(alpha, k2, d):
    Q, col = mesh_problem(alpha, k2, d)
    n, tol, N = Q.shape[0], 1e-10, 32
    terms, lam = exact_terms(Q, col)
    lo, hi = 0.9 * lam.min(), 1.1 * lam.max()
    ctx = L.ld_create_matfree(n, dense_matvec(Q), col, lo, hi, N, tol)
    val, info = L.ld_logdet(ctx)
    assert info["engine"] == 3 and info["iters"] > 0 and info["gpu_launches"] >= 3 * info["iters"]
    assert info["n_colours"] == int(col.max()) + 1 and info["n_shifts"] == N
    P = terms.sum()
    bound = 50 * tol * np.abs(terms).sum() + 100 * n * hht.rate_bound(lo, hi, N)
    assert abs(val - P) <= bound
    # per colour against the oracle's rational target on its own nodes for the same interval
    s, a = hht.log_nodes(lo, hi, N)
    rterms, _ = exact_terms(Q, col, lambda x: hht.f_N(x, s, a))
    got, seed = L.ld_column_terms(ctx)
    assert np.all(np.abs(got - rterms) <= 50 * tol * np.abs(rterms) + 1e-12 * np.abs(rterms).sum())
    # seed system followed to tol: |v^T (x - Q^{-1} v)| <= ||v|| ||Q^{-1}|| tol ||v||
    V = probing.probing_vectors(col)
    sref = np.sum(V * np.linalg.solve(Q.toarray(), V), axis=0)
    assert np.all(np.abs(seed - sref) <= 10 * tol * V.sum(axis=0) / lam.min())
    # the fused CSR path on the same colouring and interval
    rp, ci, vv = om.csr_arrays(Q)
    csr = L.ld_create(L.csr_matrix(rp, ci, vv), d, N, tol,
                      L.options(colouring=col, lambda_min=lo, lambda_max=hi))
    ref, _ = L.ld_logdet(csr)
    assert abs(val - ref) <= 2 * bound


def test_matfree_partial_ranges_add_up_and_repeat():
    Q, col = mesh_problem(1, 10.0, 2)
    n = Q.shape[0]
    lam = np.linalg.eigvalsh(Q.toarray())
    ctx = L.ld_create_matfree(n, dense_matvec(Q), col, 0.9 * lam.min(), 1.1 * lam.max(), 24, 1e-10)
    total, _ = L.ld_logdet(ctx)
    again, _ = L.ld_logdet(ctx)
    assert abs(again - total) <= 1e-13 * abs(total)
    C = int(col.max()) + 1
    cuts = [0, 1, C // 2, C]
    parts = [L.ld_logdet_partial(ctx, a, b)[0] for a, b in zip(cuts, cuts[1:])]
    assert abs(sum(parts) - total) <= 1e-12 * abs(total)


def test_matfree_error_paths_leave_the_context_usable():
    Q, col = mesh_problem(1, 10.0, 2)
    n = Q.shape[0]
    lam = np.linalg.eigvalsh(Q.toarray())
    lo, hi = 0.9 * lam.min(), 1.1 * lam.max()
    good = dense_matvec(Q)
    state = {"fail": True}

    def flaky(P, W):
        if state["fail"]:
            raise RuntimeError("planted failure")
        good(P, W)

    ctx = L.ld_create_matfree(n, flaky, col, lo, hi, 16, 1e-8)
    with pytest.raises(L.LogDetError) as e:
        L.ld_logdet(ctx)
    assert e.value.status == L.LD_ECALLBACK
    assert isinstance(ctx.matvec_error, RuntimeError)
    state["fail"] = False
    val, _ = L.ld_logdet(ctx)
    assert np.isfinite(val)

    neg = L.ld_create_matfree(n, dense_matvec(Q, -1.0), col, lo, hi, 16, 1e-8)
    with pytest.raises(L.LogDetError) as e:
        L.ld_logdet(neg)
    assert e.value.status == L.LD_ENOTSPD

    short = L.ld_create_matfree(n, good, col, lo, hi, 16, 1e-8, L.options(max_iter=3))
    with pytest.raises(L.LogDetError) as e:
        L.ld_logdet(short)
    assert e.value.status == L.LD_ENOTCONV

    for call in (lambda: L.ld_set_params(ctx, 1.0),
                 lambda: L.ld_apply(ctx, np.ones((n, 1)))):
        with pytest.raises(L.LogDetError) as e:
            call()
        assert e.value.status == L.LD_EUNSUPPORTED
    # a gradient needs the caller's derivative products, ld_grad a kept seed solution
    for call in (lambda: L.ld_logdet_grad(ctx, [0]), lambda: L.ld_grad(ctx, [0])):
        with pytest.raises(L.LogDetError) as e:
            call()
        assert e.value.status == L.LD_EINVAL
    c2, nc = L.ld_get_colouring(ctx)
    assert np.array_equal(c2, col) and nc == int(col.max()) + 1


def mesh_family():
    """Q(eta) = eta_1 Q_mesh + eta_0 diag(m) with the mesh precision of an alpha = 1 FEM
    SPDE and a 0/1 observation mask (the Gauss-linear posterior of Sec. 3 on a mesh) at
    eta = (4, 1); dQ/d eta_0 = diag(m), dQ/d eta_1 = Q_mesh."""
    Qm, col = mesh_problem(1, 10.0, 2)
    n = Qm.shape[0]
    mask = synth.obs_mask(5, n, 0.2).astype(float)
    Q = (Qm + 4.0 * sp.diags(mask)).tocsr()
    return Q, Qm, mask, col


def derivative_products(Qm, mask):
    import torch
    Qd = torch.tensor(Qm.toarray(), dtype=torch.float64, device="cuda")
    md = torch.tensor(mask, dtype=torch.float64, device="cuda")[:, None]

    def dmv(j, X, Y):
        if j == 0:
            torch.mul(md, X, out=Y)
        else:
            torch.matmul(Qd, X, out=Y)
    return dmv


def test_matfree_gradient_through_derivative_products():
    """d log det / d eta_j ~ sum_c v_c^T E_j Q^{-1} v_c with the caller's E_j X (Sec. 3's
    likelihood gradient) against dense solves; the value equals the plain solve's bit for
    bit; ld_grad on the seed solutions kept by a keep_x0 solve repeats it bit for bit."""
    Q, Qm, mask, col = mesh_family()
    n, tol, N = Q.shape[0], 1e-10, 24
    lam = np.linalg.eigvalsh(Q.toarray())
    lo, hi = 0.9 * lam.min(), 1.1 * lam.max()
    ctx = L.ld_create_matfree(n, dense_matvec(Q), col, lo, hi, N, tol)
    plain, _ = L.ld_logdet(ctx)
    L.ld_matfree_set_derivative(ctx, derivative_products(Qm, mask), 2)
    val, g, info = L.ld_logdet_grad(ctx, [0, 1])
    assert val == plain
    V = probing.probing_vectors(col)
    X = np.linalg.solve(Q.toarray(), V)
    E = [np.diag(mask), Qm.toarray()]
    gref = np.array([np.sum(V * (Ej @ X)) for Ej in E])
    for j in range(2):
        bound = 10 * tol * np.linalg.norm(E[j], 2) * V.sum() / lam.min()
        assert abs(g[j] - gref[j]) <= bound, (j, g[j], gref[j], bound)
    # E_1 = Q_mesh = Q - 4 diag(m): the two parts add up to the probed trace of I, n
    assert abs(4.0 * g[0] + g[1] - n) <= 1e-6 * n
    g10 = L.ld_grad(ctx, [1, 0])
    assert g10[0] == g[1] and g10[1] == g[0]
    kept = L.ld_create_matfree(n, dense_matvec(Q), col, lo, hi, N, tol, L.options(keep_x0=1))
    L.ld_matfree_set_derivative(kept, derivative_products(Qm, mask), 2)
    v2, _ = L.ld_logdet(kept)
    assert v2 == plain
    assert np.array_equal(L.ld_grad(kept, [0, 1]), g)
    with pytest.raises(L.LogDetError) as e:
        L.ld_grad(kept, [2])
    assert e.value.status == L.LD_EINVAL

    def failing(j, X, Y):
        raise RuntimeError("planted derivative failure")
    L.ld_matfree_set_derivative(kept, failing, 1)
    with pytest.raises(L.LogDetError) as e:
        L.ld_grad(kept, [0])
    assert e.value.status == L.LD_ECALLBACK


@pytest.mark.parametrize("ncols", [1, 3, 40])
def test_matfree_vector_form_matches_dense_functions(ncols):
    """log(Q) V and Q^{-1/2} V by the vector form of CG-M with the caller's product
    (Sec. 2.1, Eq. of the rational approximation) against U f_N(Lambda) U^T V for the same
    rational functions; 40 columns are more than the mesh's colours and wider than a warp."""
    Q, _, _, col = mesh_family()
    n, tol, N = Q.shape[0], 1e-11, 24
    lam, U = np.linalg.eigh(Q.toarray())
    lo, hi = 0.9 * lam.min(), 1.1 * lam.max()
    ctx = L.ld_create_matfree(n, dense_matvec(Q), col, lo, hi, N, tol)
    Vb = synth.random_probe_block(8, n, ncols)
    Y, info = L.ld_logmv(ctx, Vb)
    assert info["iters"] > 0
    s, a = hht.log_nodes(lo, hi, N)
    ref = (U * hht.f_N(lam, s, a)) @ (U.T @ Vb)
    assert np.abs(Y - ref).max() <= 1e-8 * np.abs(ref).max()
    Z, _ = L.ld_invsqrt_mv(ctx, Vb)
    s2, b2 = hht.invsqrt_nodes(lo, hi, N)
    ref2 = (U * hht.f_N(lam, s2, b2)) @ (U.T @ Vb)
    assert np.abs(Z - ref2).max() <= 1e-8 * np.abs(ref2).max()
    # the probing solve still works after the vector form reused the buffers
    val, _ = L.ld_logdet(ctx)
    assert np.isfinite(val)
    # Hutchinson's estimator runs on the same vector form: the sample mean of z^T log(Q) z
    if ncols == 3:
        est, se, samples, _ = L.ld_hutchinson(ctx, Vb)
        assert np.all(np.abs(samples - np.sum(Vb * ref, axis=0)) <= 1e-7 * np.sum(np.abs(Vb * ref), axis=0))
        assert abs(est - samples.mean()) <= 1e-12 * abs(samples).max()
    with pytest.raises(L.LogDetError) as e:
        L.ld_select_distance(ctx, 0, 1e-3)
    assert e.value.status == L.LD_EUNSUPPORTED
