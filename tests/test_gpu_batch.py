"""Batched evaluation (many GMRFs of uneven size in one persistent launch).

Each instance of a batch must give what its own context gives (same recurrences,
other stencil kernel: equal up to the CG tolerance), and the oracle's exact probed
rational target (Sec. 2.1) within the parity tolerances of the other GPU tests.
The full-size batch of 256 grids (sides 32..512, 5- or 13-point) is checked on a
sample of instances the oracle computes one by one.
"""
import numpy as np
import pytest

import paper_1105_5256_gb300 as L
import synth
from oracle import closed_forms as cf
from oracle import hht
from oracle import method as mt
from oracle import matrices as om
from colour_check import checked_colouring

pytestmark = pytest.mark.gpu
NSHIFT = 20


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_5256_gb300 import _build
    _build.build()
    return L.library()


def target(inst, col):
    lo, hi = mt.spectral_bounds(inst.kind, inst.dims, inst.kappa2)
    s, a = hht.log_nodes(lo, hi, NSHIFT)
    return cf.probed_value(inst.kind, inst.dims, inst.kappa2, False, col,
                           lambda lam: hht.f_N(lam, s, a))


def make(insts):
    return [L.grid_matrix(i.kind, i.dims, i.kappa2) for i in insts], [i.distance for i in insts]


@pytest.mark.parametrize("prec,tol,rel", [(L.LD_MIXED, 1e-6, 2e-5), (L.LD_FP64, 1e-10, None)])
def test_small_batch_matches_single_contexts_and_oracle(prec, tol, rel):
    insts = synth.batch_instances(7, count=12, side_lo=16, side_hi=72)
    mats, dists = make(insts)
    b = L.ld_batch_create(mats, dists, NSHIFT, tol, L.options(precision=prec))
    vals, grads, info = L.ld_batch_logdet(b, with_grad=True)
    T = info["tile_width"]                 # chosen by the batch tuner from the candidates
    assert T in ((2, 4) if prec == L.LD_MIXED else (1, 2))
    for k, inst in enumerate(insts):
        ctx = L.ld_create(L.grid_matrix(inst.kind, inst.dims, inst.kappa2), inst.distance, NSHIFT,
                          tol, L.options(precision=prec, engine=2, tile_width=T))
        v, _ = L.ld_logdet(ctx)
        terms, _ = L.ld_column_terms(ctx)
        assert abs(vals[k] - v) <= 50 * tol * np.abs(terms).sum()
        col, _ = checked_colouring(ctx, om.precision(inst.kind, inst.dims, inst.kappa2), inst.distance)
        ref = target(inst, col)
        if rel is None:
            assert abs(vals[k] - ref) <= 50 * tol * np.abs(terms).sum()
        else:
            assert abs(vals[k] - ref) <= rel * abs(ref)
        if inst.kind == L.LD_STENCIL_2D5:
            gref = cf.probed_value(inst.kind, inst.dims, inst.kappa2, False, col, lambda lam: 1 / lam)
            assert abs(grads[k] - gref) <= 1e-5 * abs(gref)
        else:
            assert np.isnan(grads[k])


def test_batch_tile_width_explicit_and_tuned_agree():
    """The tuner's choice and every explicit candidate width give the same log dets (the
    columns' recurrences do not depend on how they are grouped into tiles), and a width
    the precision does not offer is rejected before any device work."""
    insts = synth.batch_instances(9, count=8, side_lo=24, side_hi=64)
    mats, dists = make(insts)
    tol = 1e-9
    tuned, _, info = L.ld_batch_logdet(L.ld_batch_create(mats, dists, NSHIFT, tol, L.options(precision=L.LD_FP64)))
    for T in (1, 2):
        vals, _, i2 = L.ld_batch_logdet(L.ld_batch_create(mats, dists, NSHIFT, tol,
                                                          L.options(precision=L.LD_FP64, tile_width=T)))
        assert i2["tile_width"] == T
        assert np.max(np.abs(vals - tuned) / np.abs(tuned)) <= 1e-9
    with pytest.raises(L.LogDetError) as e:
        L.ld_batch_create(mats, dists, NSHIFT, tol, L.options(precision=L.LD_MIXED, tile_width=3))
    assert e.value.status == L.LD_EINVAL


def test_batch_reuse_is_deterministic():
    insts = synth.batch_instances(8, count=6, side_lo=20, side_hi=40)
    mats, dists = make(insts)
    b = L.ld_batch_create(mats, dists, NSHIFT, 1e-8, L.options(precision=L.LD_MIXED))
    v1, _, _ = L.ld_batch_logdet(b)
    v2, _, _ = L.ld_batch_logdet(b)
    assert np.array_equal(v1, v2)


def test_full_batch_256_sampled_against_oracle():
    insts = synth.batch_instances(3, count=256)
    mats, dists = make(insts)
    b = L.ld_batch_create(mats, dists, NSHIFT, 1e-6, L.options(precision=L.LD_MIXED))
    vals, _, info = L.ld_batch_logdet(b)
    assert np.all(np.isfinite(vals))
    g = np.random.default_rng(0)
    for k in g.choice(256, size=6, replace=False):
        inst = insts[k]
        col, _ = L.ld_colour_grid(inst.kind, inst.dims, False, inst.distance)
        ref = target(inst, col)
        assert abs(vals[k] - ref) <= 2e-5 * abs(ref), (k, inst)
    print("batch of 256: %.1f ms, %d instances, max iters %d" % (info["ms"], len(insts), info["iters"]))
