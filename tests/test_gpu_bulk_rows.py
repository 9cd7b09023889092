"""GPU parity of the 2D pass kernel with lattice rows arriving by bulk (TMA) copies.

The grid engine's 2D pass moves strip rows of r, w, p into shared memory with
bulk copies for packs of 24 bytes or more whenever every row piece is 16-byte
aligned (grids at least one strip wide; an even nx for 24-byte packs),
otherwise with per-thread copies.  These cases cover both, on strip layouts with ragged last strips,
torus wraps on both sides of a strip, FP64 and mixed precision and each pack
size, against the oracle's spectral value of the same rational target
    P_{d,N} = sum_c Re sum_l alpha_l v_c^T (Q - sigma_l I)^{-1} v_c
(Sec. 2.1), with the tolerances of the other parity tests.
"""
import numpy as np
import pytest

import paper_1105_5256_gb300 as L
from oracle import closed_forms as cf
from oracle import hht
from oracle import matrices as om
from oracle import method as mt
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


K5, K13 = L.LD_STENCIL_2D5, L.LD_STENCIL_2D13_SQ
CASES = [
    # kind, dims, periodic, precision, tile width, bulk expected
    (K5, (130, 40), True, L.LD_FP64, 4, 1),       # 32-byte packs, last strip wraps 122 columns
    (K5, (200, 64), True, L.LD_FP64, 3, 1),       # 24-byte packs
    (K13, (250, 31), True, L.LD_MIXED, 8, 1),     # wraps on both sides of a strip
    (K13, (256, 45), False, L.LD_MIXED, 6, 1),    # 24-byte packs, ragged last strip
    (K13, (129, 33), False, L.LD_MIXED, 8, 1),    # odd nx, 32-byte packs
    (K13, (131, 33), False, L.LD_MIXED, 6, 0),    # odd nx, 24-byte packs: per-thread copies
    (K5, (130, 40), True, L.LD_MIXED, 2, 0),      # 8-byte packs: per-thread copies
    (K5, (256, 37), False, L.LD_FP64, 1, 0),
    (K13, (250, 31), True, L.LD_MIXED, 4, 0),     # 16-byte packs
    (K13, (127, 30), True, L.LD_FP64, 4, 0),      # narrower than a strip
]


@pytest.mark.parametrize("kind,dims,per,prec,T,bulk", CASES)
def test_pass_kernel_rows(kind, dims, per, prec, T, bulk):
    k2 = 0.3
    d = 4 if kind == K5 else 2
    tol = 1e-9 if prec == L.LD_FP64 else 1e-6
    col = probing.colour_greedy(om.precision(kind, dims, k2, periodic=per), d)
    ctx = L.ld_create(L.grid_matrix(kind, dims, k2, periodic=per), d, 20, tol,
                      L.options(precision=prec, tile_width=T, engine=1, colouring=col))
    val, info = L.ld_logdet(ctx)
    assert info["bulk_rows"] == bulk
    assert info["tile_width"] == T
    lo, hi = mt.spectral_bounds(kind, dims, k2, periodic=per)
    s, a = hht.log_nodes(lo, hi, 20)
    target = cf.probed_value(kind, dims, k2, per, col, lambda lam: hht.f_N(lam, s, a),
                             per_colour=True)
    if prec == L.LD_FP64:
        assert abs(val - target.sum()) <= 50 * tol * np.abs(target).sum()
    else:
        assert abs(val - target.sum()) <= 2e-5 * abs(target.sum())
    terms, _ = L.ld_column_terms(ctx)
    bound = 50 * tol if prec == L.LD_FP64 else 2e-5
    assert np.abs(terms - target).max() <= bound * np.abs(target).sum()
