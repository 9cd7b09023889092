"""Pins for the oracle's exact references (band Cholesky, selected inverse, closed forms).

log det Q = tr log Q = sum log lambda (Sec. 2.1, Eq. "eq_logdet_ident") and
log det Q = 2 sum log L_jj (Sec. 2) must agree with each other, with numpy's
slogdet on tiny inputs and with the eigenvalue closed forms at every size the
band Cholesky runs.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import closed_forms as cf
from oracle import matrices as om
from oracle import method as mt
import synth


CASES = [
    (om.KIND_2D5, (7, 5), 0.5, True),
    (om.KIND_2D5, (7, 5), 0.5, False),
    (om.KIND_2D5, (1, 9), 0.3, False),
    (om.KIND_2D5, (3, 4), 0.7, True),
    (om.KIND_2D13_SQ, (6, 5), 0.2, False),
    (om.KIND_2D13_SQ, (6, 5), 0.2, True),
    (om.KIND_3D7, (4, 3, 5), 0.9, False),
    (om.KIND_3D7, (4, 3, 5), 0.9, True),
]


@pytest.mark.parametrize("kind,dims,k2,per", CASES)
def test_tiny_logdet_three_ways(kind, dims, k2, per):
    Q = om.precision(kind, dims, k2, periodic=per)
    sign, ld_np = np.linalg.slogdet(Q.toarray())
    assert sign > 0
    ld_chol = mt.exact_logdet_band(Q)
    ld_cf = cf.logdet(kind, dims, k2, per)
    assert abs(ld_chol - ld_np) <= 1e-11 * max(1.0, abs(ld_np))
    assert abs(ld_cf - ld_np) <= 1e-11 * max(1.0, abs(ld_np))


@pytest.mark.parametrize("kind,dims,k2,per", [
    (om.KIND_2D5, (64, 64), 0.5, True),
    (om.KIND_2D5, (96, 80), 0.01, False),
    (om.KIND_2D13_SQ, (48, 40), 0.05, False),
    (om.KIND_3D7, (12, 10, 9), 0.2, False),
])
def test_band_cholesky_vs_closed_form(kind, dims, k2, per):
    Q = om.precision(kind, dims, k2, periodic=per)
    ld_chol = mt.exact_logdet_band(Q)
    ld_cf = cf.logdet(kind, dims, k2, per)
    assert abs(ld_chol - ld_cf) <= 1e-10 * abs(ld_cf)


def test_scale_and_square_identities():
    dims = (20, 17)
    Q1 = om.precision(om.KIND_2D5, dims, 0.3)
    Q2 = om.precision(om.KIND_2D13_SQ, dims, 0.3)
    Qs = om.precision(om.KIND_2D5, dims, 0.3, scale=2.5)
    n = 20 * 17
    l1 = mt.exact_logdet_band(Q1)
    assert abs(mt.exact_logdet_band(Q2) - 2 * l1) <= 1e-10 * abs(l1)
    assert abs(mt.exact_logdet_band(Qs) - (l1 + n * np.log(2.5))) <= 1e-10 * abs(l1)


def test_not_spd_detected():
    Q = om.precision(om.KIND_2D5, (6, 6), 0.5) - 3.0 * sp.identity(36)
    with pytest.raises(mt.NotSPD):
        mt.exact_logdet_band(Q.tocsr())


def test_selected_inverse_vs_dense_and_closed_form():
    dims = (9, 7)
    Q = om.precision(om.KIND_2D13_SQ, dims, 0.4)
    Z, b = mt.selected_inverse(Q)
    Qi = np.linalg.inv(Q.toarray())
    n = Q.shape[0]
    Zb = Z.reshape(n, b + 1)
    for j in range(n):
        for o in range(b + 1):
            i = j + o
            if i < n:
                assert abs(Zb[j, o] - Qi[i, j]) <= 1e-12 * abs(Qi).max()
    tr = mt.trace_inv_times(Z, b, sp.identity(n))
    assert abs(tr - cf.trace_inv(om.KIND_2D13_SQ, dims, 0.4, False)) <= 1e-11 * tr


def test_selected_inverse_gradients_match_finite_differences():
    """tr(Q^-1 dQ/d eta) == d log det / d eta for kappa^2, tau (mask), scale."""
    dims = (24, 20)
    n = 480
    mask = synth.obs_mask(4, n, 0.1)
    k2, tau = 0.1, 4.0

    def ld(k2_, tau_, s_):
        return mt.exact_logdet_band(om.precision(om.KIND_2D5, dims, k2_, tau=tau_, mask=mask,
                                                 scale=s_))

    Q = om.precision(om.KIND_2D5, dims, k2, tau=tau, mask=mask)
    Z, b = mt.selected_inverse(Q)
    g_k2 = mt.trace_inv_times(Z, b, sp.identity(n))
    g_tau = mt.trace_inv_times(Z, b, sp.diags(mask.astype(float)))
    g_s = mt.trace_inv_times(Z, b, Q)   # dQ/ds = Q at s = 1
    h = 1e-5
    fd_k2 = (ld(k2 + h, tau, 1) - ld(k2 - h, tau, 1)) / (2 * h)
    fd_tau = (ld(k2, tau + h, 1) - ld(k2, tau - h, 1)) / (2 * h)
    assert abs(g_k2 - fd_k2) <= 1e-6 * abs(fd_k2)
    assert abs(g_tau - fd_tau) <= 1e-6 * abs(fd_tau)
    assert abs(g_s - n) <= 1e-9 * n


def test_dst_probing_equals_dense_eigh():
    """u_k^T v via orthonormal DST/FFT == dense eigendecomposition, both boundaries."""
    from oracle import probing
    for kind, dims, per in [(om.KIND_2D5, (8, 6), False), (om.KIND_2D5, (8, 6), True),
                            (om.KIND_2D13_SQ, (7, 9), False), (om.KIND_3D7, (4, 5, 3), False)]:
        Q = om.precision(kind, dims, 0.3, periodic=per)
        col = probing.colour_greedy(Q, 2)
        for f in (np.log, lambda x: 1.0 / x):
            a = cf.probed_value(kind, dims, 0.3, per, col, f)
            b = mt.probed_dense(Q, col, f)
            assert abs(a - b) <= 1e-11 * max(1.0, abs(b))


def test_circulant_symbol_route_matches_spectral():
    from oracle import probing
    dims = (16, 12)
    Q = om.precision(om.KIND_2D5, dims, 0.5, periodic=True)
    col = probing.colour_greedy(Q, 3)
    a = cf.circulant_probed_log(dims, 0.5, col)
    b = cf.probed_value(om.KIND_2D5, dims, 0.5, True, col, np.log)
    assert abs(a - b) <= 1e-10 * abs(b)
