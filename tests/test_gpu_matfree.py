"""GPU parity of the matrix-free operator path (ld_create_matfree): the caller supplies
only W = Q P (Sec. 1: the method touches Q through products), the library runs CG with
the projected multi-shift recurrences of Sec. 2.1 in its own kernels.

The caller's product here is a dense torch matmul of the oracle's matrix.  Targets:
  * the exact probed value P_d = sum_c v_c^T log(Q) v_c from dense eigh (oracle), with the
    oracle's greedy colouring: |mf - P_d| <= 50 tol sum_c |term_c| + 100 n rate(M/m, N)
    (the CG stopping error and the quadrature bound, as the CSR parity tests);
  * per-colour terms against the oracle's rational target on the same nodes;
  * the fused CSR path on the same colouring and interval, to the same tolerance.
Error paths: a failing callback, an operator that is not SPD, max_iter, and the entry
points a matrix-free context does not support.
"""
import numpy as np
import pytest

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
    assert info["engine"] == 3 and info["iters"] > 0 and info["gpu_launches"] > 5 * info["iters"]
    assert info["n_colours"] == int(col.max()) + 1 and info["n_shifts"] == N
    P = terms.sum()
    bound = 50 * tol * np.abs(terms).sum() + 100 * n * hht.rate_bound(lo, hi, N)
    assert abs(val - P) <= bound
    # per colour against the oracle's rational target on its own nodes for the same interval
    s, a = hht.log_nodes(lo, hi, N)
    rterms, _ = exact_terms(Q, col, lambda x: hht.f_N(x, s, a))
    got, seed = L.ld_column_terms(ctx)
    assert np.all(np.abs(got - rterms) <= 50 * tol * np.abs(rterms) + 1e-12 * np.abs(rterms).sum())
    assert np.all(np.isnan(seed))
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
                 lambda: L.ld_logdet_grad(ctx, [L.LD_P_KAPPA2]),
                 lambda: L.ld_logmv(ctx, np.ones((n, 1))),
                 lambda: L.ld_apply(ctx, np.ones((n, 1)))):
        with pytest.raises(L.LogDetError) as e:
            call()
        assert e.value.status == L.LD_EUNSUPPORTED
    c2, nc = L.ld_get_colouring(ctx)
    assert np.array_equal(c2, col) and nc == int(col.max()) + 1
