"""GPU: reliable-update residual replacement in mixed precision.

With FP32 vectors the recursively updated CG residual drifts away from the true
residual v - Q x of the seed solve: the recursion still reports convergence while
the true residual stalls orders of magnitude above the tolerance, and the gradient
Sum_c (E v_c)^T x_c inherits that error.  Reliable updates keep the seed solution
as x_hi (FP64) + x_lo (FP32 correction) and, whenever a column's residual norm has
fallen by reliable_delta, fold x_lo into x_hi and replace the residual by
v - Q x_hi formed in FP64.  Checked here on the Matern alpha = 2 precision
(13-point, kappa^2 = 0.01, condition number about 4e5):
  * the true relative seed residual (reported in FP64 by the library) meets the
    tolerance with updates and does not without them;
  * the gradient d log det / d kappa^2 = Sum_c v_c^T Q^{-1} (2 Q1) v_c matches exact
    sparse solves of the same probing vectors to FP64-level accuracy with updates;
  * the log det stays within the mixed-precision parity tolerance of the oracle's
    rational target, and FP64 runs are unchanged by the option.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import paper_1105_5256_gb300 as L
from oracle import closed_forms as cf
from oracle import hht
from oracle import matrices as om
from oracle import method as mt
from oracle import probing

pytestmark = pytest.mark.gpu

DIMS, K2, DIST, NSHIFT, TOL = (128, 128), 0.01, 2, 20, 1e-8


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_5256_gb300 import _build
    _build.build()
    return L.library()


@pytest.fixture(scope="module")
def oracle():
    kind = om.KIND_2D13_SQ
    Q = om.precision(kind, DIMS, K2)
    col = probing.colour_greedy(Q, DIST)
    V = probing.probing_vectors(col)
    X = spla.splu(Q.tocsc()).solve(V)
    E = 2.0 * om.precision(om.KIND_2D5, DIMS, K2)          # dQ/dkappa^2 = 2 (kappa^2 I - Lap)
    grad = float(np.sum(np.asarray(E @ V) * X))
    lo, hi = mt.spectral_bounds(kind, DIMS, K2)
    s, a = hht.log_nodes(lo, hi, NSHIFT)
    target = cf.probed_value(kind, DIMS, K2, False, col, lambda lam: hht.f_N(lam, s, a))
    return {"col": col, "grad": grad, "target": target}


def run(col, prec, delta, tol=TOL):
    ctx = L.ld_create(L.grid_matrix(L.LD_STENCIL_2D13_SQ, DIMS, K2), DIST, NSHIFT, tol,
                      L.options(precision=prec, engine=1, colouring=col, reliable_delta=delta))
    v, g, info = L.ld_logdet_grad(ctx, [L.LD_P_KAPPA2])
    return v, float(g[0]), info


def test_reliable_updates_restore_true_residual_and_gradient(oracle):
    v0, g0, i0 = run(oracle["col"], L.LD_MIXED, 0.0)
    v1, g1, i1 = run(oracle["col"], L.LD_MIXED, 1e-2)
    print("mixed: true residual %.2e -> %.2e with %d updates; grad rel err %.1e -> %.1e"
          % (i0["rel_resid_max"], i1["rel_resid_max"], i1["reliable_updates"],
             abs(g0 - oracle["grad"]) / oracle["grad"], abs(g1 - oracle["grad"]) / oracle["grad"]))
    assert i0["reliable_updates"] == 0 and i1["reliable_updates"] >= 1
    assert i1["rel_resid_max"] <= 10 * TOL
    assert i0["rel_resid_max"] > 1e3 * i1["rel_resid_max"]          # the drift being repaired
    assert abs(g1 - oracle["grad"]) <= 1e-7 * abs(oracle["grad"])
    for v in (v0, v1):
        assert abs(v - oracle["target"]) <= 2e-5 * abs(oracle["target"])


def test_reliable_updates_leave_fp64_unchanged(oracle):
    v0, g0, i0 = run(oracle["col"], L.LD_FP64, 0.0, tol=1e-9)
    v1, g1, i1 = run(oracle["col"], L.LD_FP64, 1e-2, tol=1e-9)
    assert i0["rel_resid_max"] <= 10 * 1e-9 and i1["rel_resid_max"] <= 10 * 1e-9
    assert abs(v1 - v0) <= 1e-9 * abs(v0)
    assert abs(g1 - g0) <= 1e-8 * abs(g0)
    assert abs(g1 - oracle["grad"]) <= 1e-8 * abs(oracle["grad"])


def test_true_residual_reported_only_with_seed_solutions(oracle):
    ctx = L.ld_create(L.grid_matrix(L.LD_STENCIL_2D13_SQ, DIMS, K2), DIST, NSHIFT, 1e-6,
                      L.options(precision=L.LD_MIXED, engine=1, colouring=oracle["col"]))
    _, info = L.ld_logdet(ctx)
    assert info["rel_resid_max"] == -1.0 and info["reliable_updates"] == 0


def test_reliable_updates_on_the_csr_pass():
    """The CSR pass (streaming step + row-group product) with reliable updates: an
    ill-conditioned FEM alpha = 2 mesh precision Q = s Q0 (s = 2) in mixed precision.  The
    scale gradient d log det / ds = sum_c v_c^T Q^{-1} Q0 v_c is n / s exactly for any
    colouring, so its error measures the kept seed solutions: with updates the true residual
    meets the tolerance and the gradient is FP64-accurate; without them it is not."""
    import synth
    p, t = synth.perturbed_triangulation(31, 60, 55)
    h = 1.0 / 59
    Q = om.fem_spde_precision(p, t, 0.01 / h ** 2, 2, 1.0)
    n = Q.shape[0]
    rp, ci, vv = om.csr_arrays(Q)
    lo = 0.9 * float(spla.eigsh(Q.tocsc(), k=1, sigma=0.0, which="LM", return_eigenvectors=False)[0])
    hi = float(np.abs(Q).sum(axis=1).max())
    out = {}
    for delta in (0.0, 1e-2):
        ctx = L.ld_create(L.csr_matrix(rp, ci, vv, scale=2.0), 2, NSHIFT, TOL,
                          L.options(precision=L.LD_MIXED, engine=1, tile_width=4, reliable_delta=delta,
                                    lambda_min=2.0 * lo, lambda_max=2.0 * hi))
        v, g, info = L.ld_logdet_grad(ctx, [L.LD_P_SCALE])
        out[delta] = (v, float(g[0]), info)
        assert info["engine"] == 1 and info["pass_words"] == 10
    v1, g1, i1 = out[1e-2]
    v0, g0, i0 = out[0.0]
    print("CSR mixed: true residual %.2e -> %.2e with %d updates; grad rel err %.1e -> %.1e"
          % (i0["rel_resid_max"], i1["rel_resid_max"], i1["reliable_updates"],
             abs(g0 - n / 2) / (n / 2), abs(g1 - n / 2) / (n / 2)))
    assert i1["reliable_updates"] >= 1 and i1["rel_resid_max"] <= 10 * TOL
    assert abs(g1 - n / 2) <= 1e-6 * n / 2
    assert abs(v1 - v0) <= 2e-5 * abs(v0)
