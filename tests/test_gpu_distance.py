"""GPU: colouring distance by decay of log(Q) e_j (Sec. 2.1 heuristic).

ld_select_distance forms y = log(Q) e_j with the context's method and returns
p = min { d(l, j) : |y_l| < eps |y_j| } and the decay profile max_{d(l,j)=d} |y_l|/|y_j|.
The oracle forms y exactly (grid eigenbasis, or dense logm for CSR), its own BFS
graph distances, and the same minimum.  Profiles agree to the method's accuracy;
the selected distances agree exactly wherever no ratio lies within 1e-4 (relative)
of eps, which each case checks first.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import paper_1105_5256_gb300 as L
import synth
from oracle import closed_forms as cf
from oracle import matrices as om
from oracle import probing

pytestmark = pytest.mark.gpu

EPS = (1e-1, 1e-2, 1e-3, 1e-4)
MAXD = 24


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_5256_gb300 import _build
    _build.build()
    return L.library()


def check(ctx, Q, y, j):
    dist = probing.graph_distances(Q, j, MAXD)
    prof_ref = probing.decay_profile(y, dist, j, MAXD)
    ratio = np.abs(y) / abs(y[j])
    for eps in EPS:
        near = (dist >= 0) & (np.abs(ratio - eps) <= 1e-4 * eps)
        assert not np.any(near), "eps %g sits on a decay value" % eps
        p_ref = probing.decay_distance(y, dist, j, eps)
        p, prof, _ = L.ld_select_distance(ctx, j, eps, MAXD)
        assert p == p_ref, (eps, p, p_ref)
        assert np.abs(prof - prof_ref).max() <= 1e-7
    return prof_ref


@pytest.mark.parametrize("kind,dims,per,k2,j", [
    (om.KIND_2D5, (64, 64), True, 0.5, 64 * 20 + 7),
    (om.KIND_2D5, (50, 46), False, 0.05, 50 * 23 + 25),
    (om.KIND_2D13_SQ, (48, 40), False, 0.1, 48 * 19 + 30),
])
def test_grid_distance_matches_oracle(kind, dims, per, k2, j):
    ctx = L.ld_create(L.grid_matrix(kind, dims, k2, periodic=per), 2, 24, 1e-11,
                      L.options(precision=L.LD_FP64))
    Q = om.precision(kind, dims, k2, periodic=per)
    y = cf.log_column(kind, dims, k2, per, j)
    prof = check(ctx, Q, y, j)
    assert np.all(np.diff(prof[:8]) < 0)      # decays away from j


def test_csr_distance_matches_oracle():
    n = 300
    rows, cols, w = synth.random_sparse_spd_pattern(5, n)
    rp, ci, vv = synth.csr_from_edges(n, rows, cols, w, 0.5)
    Q = sp.csr_matrix((vv, ci, rp), shape=(n, n))
    ev = np.linalg.eigvalsh(Q.toarray())
    ctx = L.ld_create(L.csr_matrix(rp, ci, vv), 1, 24, 1e-11,
                      L.options(precision=L.LD_FP64, lambda_min=0.9 * ev.min(), lambda_max=1.1 * ev.max()))
    j = 123
    y = sla.logm(Q.toarray()).real[:, j]
    check(ctx, Q, y, j)


def test_distance_grows_as_kappa2_falls():
    """Sec. 3: smaller kappa (longer range) needs a larger colouring distance."""
    dims = (64, 64)
    ps = []
    for k2 in (1.0, 0.1, 0.02):
        ctx = L.ld_create(L.grid_matrix(om.KIND_2D5, dims, k2, periodic=True), 2, 24, 1e-10,
                          L.options(precision=L.LD_FP64))
        ps.append(L.ld_select_distance(ctx, 64 * 32 + 32, 1e-3, 64)[0])
    assert ps[0] < ps[1] < ps[2], ps
