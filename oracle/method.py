"""Oracle: the log-determinant method end to end, and exact references (test infrastructure).

  exact_logdet_band    log det Q = 2 sum log L_jj from a banded Cholesky in
                       natural order (Sec. 2, the traditional route, without
                       reordering).
  selected_inverse     (Q^{-1})_{ij} inside the band of L (Takahashi), for the
                       exact gradient tr(Q^{-1} dQ/d eta).
  probed_dense         sum_c v_c^T f(Q) v_c by a dense eigendecomposition
                       (tiny cases).
  probed_rational_band sum_c Re sum_l alpha_l v_c^T (Q - sigma_l I)^{-1} v_c by
                       exact complex-symmetric banded LDL^T solves: the
                       method's target with no Krylov error.
  probed_rational_splu the same target with each shifted system solved by a
                       sparse LU factorisation (SuperLU, minimum-degree
                       ordering): grids whose natural-order band is too wide
                       for the banded solver (512^2 2D, 32^3 3D).
  spectral_bounds      the enclosing interval [m, M] used for the quadrature.
  logdet_method        the method in the paper's order: probing vectors from
                       the colouring (Sec. 2.1) -> rational nodes (Eq.
                       "eq_rat_app") -> CG-M per probing vector (Sec. 2.1) ->
                       sum of v_c^T f_N(Q) v_c; optional gradient terms
                       (E v_c)^T Q^{-1} v_c from the seed solution; optionally
                       only a chosen subset of the colours (full-size grids,
                       where every probing vector is an independent CG-M run).

Reading of the spectral bounds (the paper only says extremal-eigenvalue
estimates are needed): for Q = scale * (diag(kappa2) - Lap + tau diag(mask)),
Weyl's inequalities with the exact extreme eigenvalues of -Lap give
    m = scale * (min kappa2 + sum_d mu_min(N_d)),
    M = scale * (max kappa2 + tau * [mask nonempty] + sum_d mu_max(N_d)),
mu_min = 2 - 2cos(pi/(N+1)), mu_max = 2 + 2cos(pi/(N+1)) (Dirichlet);
mu_min = 0, mu_max = max_k 2 - 2cos(2 pi k / N) (periodic).  The Matern square
uses (.)^2 of the 5-point bounds.  M is raised to at least 1.01 m so the
conformal map is never degenerate.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import _native
from .cgm import cgm
from .hht import log_nodes
from .matrices import bandwidth, to_lower_band

KIND_CSR, KIND_2D5, KIND_2D13_SQ, KIND_3D7 = 0, 1, 2, 3


class NotSPD(RuntimeError):
    pass


def exact_logdet_band(Q: sp.csr_matrix) -> float:
    n = Q.shape[0]
    b = bandwidth(Q)
    A = to_lower_band(Q, b)
    lib = _native.lib()
    st = lib.or_chol_band(n, b, _native.ptr(A))
    if st != 0:
        raise NotSPD("non-positive pivot at column %d" % (st - 1))
    return float(lib.or_logdet_from_chol(n, b, _native.ptr(A)))


def selected_inverse(Q: sp.csr_matrix):
    """(Z_band, b): (Q^{-1})_{ij} for j <= i <= j+b, band storage as to_lower_band."""
    n = Q.shape[0]
    b = bandwidth(Q)
    A = to_lower_band(Q, b)
    lib = _native.lib()
    st = lib.or_chol_band(n, b, _native.ptr(A))
    if st != 0:
        raise NotSPD("non-positive pivot at column %d" % (st - 1))
    Z = np.zeros_like(A)
    lib.or_takahashi_diag(n, b, _native.ptr(A), _native.ptr(Z))
    return Z, b


def trace_inv_times(Z: np.ndarray, b: int, E: sp.spmatrix) -> float:
    """tr(Q^{-1} E) for symmetric E whose pattern lies inside the band."""
    E = E.tocoo()
    n = E.shape[0]
    Zb = Z.reshape(n, b + 1)
    i, j = np.maximum(E.row, E.col), np.minimum(E.row, E.col)
    if np.any(i - j > b):
        raise ValueError("E wider than the band of L")
    return float(np.sum(Zb[j, i - j] * E.data))


def probed_dense(Q, colour: np.ndarray, f) -> float:
    Qd = Q.toarray() if sp.issparse(Q) else np.asarray(Q)
    lam, U = np.linalg.eigh(Qd)
    if lam.min() <= 0:
        raise NotSPD("eigenvalue <= 0")
    F = (U * f(lam)) @ U.T
    colour = np.asarray(colour)
    total = 0.0
    for c in range(int(colour.max()) + 1):
        idx = np.nonzero(colour == c)[0]
        total += float(F[np.ix_(idx, idx)].sum())
    return total


def probed_rational_band(Q: sp.csr_matrix, colour: np.ndarray, sigma, alpha,
                         per_colour: bool = False):
    """sum_c Re sum_l alpha_l v_c^T (Q - sigma_l I)^{-1} v_c, exact solves."""
    n = Q.shape[0]
    b = bandwidth(Q)
    colour = np.asarray(colour)
    C = int(colour.max()) + 1
    V = np.zeros((C, n))
    V[colour, np.arange(n)] = 1.0
    V = np.ascontiguousarray(V)
    lib = _native.lib()
    base = to_lower_band(Q, b).astype(np.complex128)
    diag_idx = np.arange(n) * (b + 1)
    terms = np.zeros(C)
    q = np.zeros(C, complex)
    work = np.zeros(n, complex)
    for s, al in zip(sigma, alpha):
        A = base.copy()
        A[diag_idx] -= s
        st = lib.or_ldlt_band_z(n, b, _native.ptr(A))
        if st != 0:
            raise RuntimeError("zero pivot in shifted LDL^T")
        lib.or_fwd_quadform_z(n, b, _native.ptr(A), C, _native.ptr(V), _native.ptr(q),
                              _native.ptr(work))
        terms += np.real(al * q)
    return terms if per_colour else float(terms.sum())


def probed_rational_splu(Q: sp.csr_matrix, colour: np.ndarray, sigma, alpha,
                         per_colour: bool = False):
    """sum_c Re sum_l alpha_l v_c^T (Q - sigma_l I)^{-1} v_c with exact sparse solves.

    Each shifted matrix Q - sigma_l I (complex symmetric) is factorised once by
    SuperLU with a minimum-degree ordering of its symmetric pattern, and all
    probing vectors are solved against it; v^T x is the bilinear form (no
    conjugate), as in the Cauchy integral of Eq. "eq_rat_app".
    """
    n = Q.shape[0]
    colour = np.asarray(colour)
    C = int(colour.max()) + 1
    V = np.zeros((n, C), dtype=np.complex128)
    V[np.arange(n), colour] = 1.0
    I = sp.identity(n, dtype=np.complex128, format="csc")
    Qc = Q.astype(np.complex128).tocsc()
    terms = np.zeros(C)
    for s, al in zip(sigma, alpha):
        lu = spla.splu((Qc - s * I).tocsc(), permc_spec="MMD_AT_PLUS_A",
                       options={"SymmetricMode": True})
        X = lu.solve(V)
        q = np.sum(V * X, axis=0)
        terms += np.real(al * q)
    return terms if per_colour else float(terms.sum())


def lap_extremes_1d(N: int, periodic: bool):
    if periodic:
        k = np.arange(N)
        mu = 2.0 - 2.0 * np.cos(2.0 * np.pi * k / N)
        return 0.0, float(mu.max())
    return (2.0 - 2.0 * np.cos(np.pi / (N + 1)), 2.0 + 2.0 * np.cos(np.pi / (N + 1)))


def spectral_bounds(kind: int, dims, kappa2, periodic: bool = False, tau: float = 0.0,
                    mask=None, scale: float = 1.0):
    k2 = np.asarray(kappa2, dtype=np.float64)
    mu_lo = sum(lap_extremes_1d(int(d), periodic)[0] for d in dims)
    mu_hi = sum(lap_extremes_1d(int(d), periodic)[1] for d in dims)
    lo = float(k2.min()) + mu_lo
    hi = float(k2.max()) + mu_hi
    if mask is not None and tau != 0.0 and np.any(np.asarray(mask) != 0):
        hi += tau
    if kind == KIND_2D13_SQ:
        lo, hi = lo * lo, hi * hi
    lo, hi = scale * lo, scale * hi
    hi = max(hi, 1.01 * lo)
    return lo, hi


def logdet_method(Q: sp.csr_matrix, colour: np.ndarray, lmin: float, lmax: float,
                  n_shifts: int, tol: float, maxiter: int = 100000, grad_mats=(),
                  per_colour: bool = False, colours=None):
    """Probing x rational approximation x CG-M, in the paper's order.

    Returns dict(logdet, grads, terms (per colour), iters (per colour)).
    grad_mats: list of E_eta = dQ/d eta; gradient estimate sum_c (E v_c)^T x0_c.
    colours: run only these probing vectors (the others' terms stay NaN and the sums
    cover the chosen ones); None runs all of them.
    """
    sigma, alpha = log_nodes(lmin, lmax, n_shifts)
    colour = np.asarray(colour)
    C = int(colour.max()) + 1
    n = Q.shape[0]
    run = range(C) if colours is None else [int(c) for c in colours]
    terms = np.full(C, np.nan) if colours is not None else np.zeros(C)
    gterms = np.full((len(grad_mats), C), np.nan) if colours is not None else np.zeros((len(grad_mats), C))
    seeds = np.full(C, np.nan) if colours is not None else np.zeros(C)
    iters = np.zeros(C, dtype=np.int64)
    mv = Q.dot
    for c in run:
        v = (colour == c).astype(np.float64)
        res = cgm(mv, v, -sigma, tol, maxiter)
        terms[c] = float(np.real(np.sum(alpha * res["pi"])))
        seeds[c] = float(v @ res["x0"])
        iters[c] = res["iters"]
        for g, E in enumerate(grad_mats):
            gterms[g, c] = float((E @ v) @ res["x0"])
    out = dict(logdet=float(np.nansum(terms)), grads=np.nansum(gterms, axis=1), iters=iters,
               sigma=sigma, alpha=alpha)
    if per_colour:
        out["terms"] = terms
        out["gterms"] = gterms
        out["seeds"] = seeds
    return out


# ---------------------------------------------------------------- likelihood (Sec. 1, 3)
def gaussian_loglik(Q: sp.csr_matrix, Y: np.ndarray) -> float:
    """sum over the columns y of Y of log N(y | 0, Q^{-1}) = 1/2 log det Q - 1/2 y^T Q y
    - n/2 log(2 pi), with log det Q by the band Cholesky (the directly observed field
    of Sec. 3)."""
    Y = np.asarray(Y)
    if Y.ndim == 1:
        Y = Y[:, None]
    n, s = Y.shape
    ld = exact_logdet_band(Q)
    quad = float(np.sum(Y * (Q @ Y)))
    return 0.5 * s * ld - 0.5 * quad - 0.5 * s * n * np.log(2.0 * np.pi)
