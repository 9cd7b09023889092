"""Vector form of CG-M (log(Q) v for arbitrary v) and the tile-width autotuner.

ld_logmv must give Re sum_l alpha_l (Q - sigma_l I)^{-1} V (dense complex solves of the
oracle) and, within the quadrature certificate, log(Q) V (scipy.linalg.logm); with the
probing vectors as right-hand sides, v_c^T log(Q) v_c from the vector form must equal the
projected per-colour terms of ld_logdet (the two forms of CG-M in Sec. 2.1 agree).
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import scipy.linalg as sla

import paper_1105_5256_gb300 as L
import synth
from oracle import hht
from oracle import matrices as om
from oracle import method as mt
from oracle import probing
from colour_check import checked_colouring

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_5256_gb300 import _build
    _build.build()
    return L.library()


@pytest.mark.parametrize("kind,dims,per,prec", [
    (om.KIND_2D5, (13, 11), False, L.LD_FP64),
    (om.KIND_2D13_SQ, (10, 9), True, L.LD_FP64),
    (om.KIND_3D7, (5, 4, 6), False, L.LD_MIXED),
])
def test_logmv_matches_dense_rational_and_logm(kind, dims, per, prec):
    k2 = 0.4
    Q = om.precision(kind, dims, k2, periodic=per)
    n = Q.shape[0]
    tol = 1e-11 if prec == L.LD_FP64 else 1e-6
    ctx = L.ld_create(L.grid_matrix(kind, dims, k2, periodic=per), 1, 24, tol,
                      L.options(precision=prec))
    V = synth.random_probe_block(9, n, 5)
    Y, info = L.ld_logmv(ctx, V)
    sigma, alpha = L.ld_get_nodes(ctx)
    A = Q.toarray()
    ref = sum(np.real(al * np.linalg.solve(A - sg * np.eye(n), V.astype(complex)))
              for sg, al in zip(sigma, alpha))
    rel = 1e-8 if prec == L.LD_FP64 else 1e-4
    assert np.abs(Y - ref).max() <= rel * np.abs(ref).max()
    lg = np.real(sla.logm(A)) @ V
    assert np.abs(Y - lg).max() <= info["quad_cert"] * np.abs(V).sum(axis=0).max() + rel * np.abs(lg).max()


def test_vector_form_cross_checks_projected_terms():
    dims, k2 = (24, 20), 0.2
    ctx = L.ld_create(L.grid_matrix(om.KIND_2D13_SQ, dims, k2), 2, 20, 1e-10,
                      L.options(precision=L.LD_FP64))
    L.ld_logdet(ctx)
    terms, _ = L.ld_column_terms(ctx)
    col, nc = checked_colouring(ctx, om.precision(om.KIND_2D13_SQ, dims, k2), 2)
    Vp = probing.probing_vectors(col)
    Y, _ = L.ld_logmv(ctx, Vp)
    vec_terms = np.sum(Vp * Y, axis=0)
    assert np.abs(vec_terms - terms).max() <= 1e-8 * np.abs(terms).max()


def test_autotuner_picks_a_candidate_and_caches(tmp_path):
    cache = tmp_path / "tune.json"
    code = (
        "import paper_1105_5256_gb300 as L\n"
        "m = L.grid_matrix(L.LD_STENCIL_2D13_SQ, (512, 512), 0.3)\n"
        "c = L.ld_create(m, 2, 20, 1e-6, L.options(precision=L.LD_MIXED))\n"
        "v, info = L.ld_logdet(c)\n"
        "print(info['tile_width'])\n")
    env = dict(os.environ, LD_AUTOTUNE_CACHE=str(cache), PYTHONPATH=ROOT)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr
    T = int(out.stdout.strip().splitlines()[-1])
    assert T in (2, 4, 6, 8)
    saved = json.loads(cache.read_text())
    assert list(saved.values()) == [T]
    # a second process reads the cache and makes the same choice
    out2 = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                          timeout=600)
    assert out2.returncode == 0 and int(out2.stdout.strip().splitlines()[-1]) == T
