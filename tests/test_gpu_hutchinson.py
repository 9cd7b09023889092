"""GPU: the Hutchinson estimator (Sec. 2.1, Eq. "eq_est_eq") through ld_hutchinson.

Each sample z^T f_N(Q) z (Rademacher z drawn by the seeded generator and passed in)
equals the oracle's exact quadratic form of the same rational function within the
CG tolerance; the estimate is the sample mean, its standard error the sample
deviation / sqrt(s).  The probing estimate of the same model is printed beside
it (its error is the probing bias, deterministic; the Hutchinson error is
statistical and shrinks like 1/sqrt(s)).
"""
import numpy as np
import pytest

import paper_1105_5256_gb300 as L
import synth
from oracle import closed_forms as cf
from oracle import hht
from oracle import matrices as om
from oracle import method as mt

pytestmark = pytest.mark.gpu

DIMS, K2, N, TOL = (64, 64), 0.5, 20, 1e-10


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_5256_gb300 import _build
    _build.build()
    return L.library()


def test_hutchinson_samples_match_oracle_and_estimate_is_consistent():
    kind = om.KIND_2D5
    ctx = L.ld_create(L.grid_matrix(kind, DIMS, K2, periodic=True), 4, N, TOL,
                      L.options(precision=L.LD_FP64))
    Z = synth.rademacher_block(11, 4096, 256)
    est, se, q, info = L.ld_hutchinson(ctx, Z)
    lo, hi = mt.spectral_bounds(kind, DIMS, K2, periodic=True)
    s, a = hht.log_nodes(lo, hi, N)
    ref = cf.quadratic_forms(kind, DIMS, K2, True, Z, lambda lam: hht.f_N(lam, s, a))
    assert np.abs(q - ref).max() <= 50 * TOL * np.abs(ref).max() * 64
    assert abs(est - q.mean()) <= 1e-12 * abs(est)
    assert abs(se - q.std(ddof=1) / np.sqrt(q.size)) <= 1e-9 * se
    exact = cf.logdet(kind, DIMS, K2, True)
    assert abs(est - exact) <= 5 * se
    probed, _ = L.ld_logdet(ctx)
    print("tr log Q %.4f | Hutchinson (256 vectors) %.4f +- %.4f | probing (25 vectors) %.4f"
          % (exact, est, se, probed))
