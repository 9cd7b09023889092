"""Oracle: closed forms for constant-coefficient grid precisions (test infrastructure).

For Q = kappa^2 I - Lap on a rectangle (Dirichlet truncation) or torus
(periodic), the eigenvectors are tensor products of 1D sine / Fourier modes
and the eigenvalues are
    Dirichlet: lambda = kappa^2 + sum_d (2 - 2 cos(pi k_d / (N_d + 1))),  k_d = 1..N_d
    periodic:  lambda = kappa^2 + sum_d (2 - 2 cos(2 pi k_d / N_d)),    k_d = 0..N_d-1
and the Matern square Q1^2 has eigenvalues lambda^2 with the same vectors.

From these, with the identity log det Q = tr log Q = sum log lambda_i
(Sec. 2.1, Eq. "eq_logdet_ident"):
  * exact log det and tr Q^{-1};
  * the exact probed value  sum_c v_c^T f(Q) v_c = sum_c sum_k f(lambda_k) |u_k^T v_c|^2
    for any colouring and any scalar function f (log for the probing error,
    the rational f_N for the method's target), with u_k^T v_c obtained by an
    orthonormal DST-I / FFT of the indicator grid (Sec. 2.1: probing vectors).
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft

KIND_2D5, KIND_2D13_SQ, KIND_3D7 = 1, 2, 3


def lap_eigs_1d(n: int, periodic: bool) -> np.ndarray:
    if periodic:
        k = np.arange(n)
        return 2.0 - 2.0 * np.cos(2.0 * np.pi * k / n)
    k = np.arange(1, n + 1)
    return 2.0 - 2.0 * np.cos(np.pi * k / (n + 1))


def eig_grid(kind: int, dims, kappa2: float, periodic: bool, scale: float = 1.0) -> np.ndarray:
    """Eigenvalues on the spectral grid, array shaped reversed(dims) (x fastest last)."""
    dims = [int(d) for d in dims]
    mu = np.zeros([1] * len(dims))
    for ax, nd in enumerate(dims):
        shape = [1] * len(dims)
        shape[len(dims) - 1 - ax] = nd
        mu = mu + lap_eigs_1d(nd, periodic).reshape(shape)
    lam1 = kappa2 + mu
    lam = lam1 ** 2 if kind == KIND_2D13_SQ else lam1
    return scale * lam


def logdet(kind, dims, kappa2, periodic, scale=1.0) -> float:
    lam = eig_grid(kind, dims, kappa2, periodic, scale)
    return float(np.sum(np.log(lam)))


def trace_inv(kind, dims, kappa2, periodic, scale=1.0) -> float:
    return float(np.sum(1.0 / eig_grid(kind, dims, kappa2, periodic, scale)))


def extreme_eigs(kind, dims, kappa2, periodic, scale=1.0):
    lam = eig_grid(kind, dims, kappa2, periodic, scale)
    return float(lam.min()), float(lam.max())


def spectral_coeffs(grid_vals: np.ndarray, periodic: bool) -> np.ndarray:
    """|u_k^T v|^2 for every eigenvector u_k, v given on the grid (reversed dims)."""
    if periodic:
        c = sfft.fftn(grid_vals, norm="ortho")
        return np.abs(c) ** 2
    c = sfft.dstn(grid_vals, type=1, norm="ortho")
    return c * c


def probed_value(kind, dims, kappa2, periodic, colour: np.ndarray, f, scale=1.0,
                 per_colour: bool = False, colours=None):
    """sum_c v_c^T f(Q) v_c with v_c = indicator(colour == c).

    f maps an eigenvalue array to values (real).  Returns the total, or the
    per-colour array when per_colour=True.  `colours` restricts the classes
    evaluated (the others are left at zero), for sampled checks of large grids.
    """
    dims = [int(d) for d in dims]
    shape = tuple(reversed(dims))
    lam = eig_grid(kind, dims, kappa2, periodic, scale)
    flam = f(lam)
    col = np.asarray(colour).reshape(shape)
    ncol = int(col.max()) + 1 if col.size else 0
    out = np.zeros(ncol)
    for c in (range(ncol) if colours is None else colours):
        v = (col == c).astype(np.float64)
        out[c] = float(np.sum(flam * spectral_coeffs(v, periodic)))
    return out if per_colour else float(out.sum())


def circulant_probed_log(dims, kappa2, colour: np.ndarray) -> float:
    """Periodic grids only: log Q is circulant with symbol l(delta) =
    (1/n) sum_k log(lambda_k) e^{2 pi i k.delta/N}; the probed value is
    sum_i sum_{j: colour(j)=colour(i)} l(j - i).  Independent route to
    probed_value(..., f=log) for the periodic 5-point model."""
    dims = [int(d) for d in dims]
    shape = tuple(reversed(dims))
    lam = eig_grid(KIND_2D5 if len(dims) == 2 else KIND_3D7, dims, kappa2, True)
    ell = np.real(sfft.ifftn(np.log(lam)))      # l(delta), indexed by delta mod N
    col = np.asarray(colour).reshape(shape)
    total = 0.0
    ncol = int(col.max()) + 1
    for c in range(ncol):
        v = (col == c).astype(np.float64)
        # sum_{i,j in class} l(j-i) = sum_delta l(delta) * autocorr_v(delta)
        V = sfft.fftn(v)
        auto = np.real(sfft.ifftn(V * np.conj(V)))
        total += float(np.sum(ell * auto))
    return total


def log_column(kind, dims, kappa2, periodic, j: int, scale=1.0) -> np.ndarray:
    """y = log(Q) e_j exactly, by the eigenbasis: y = U diag(log lambda) U^T e_j with U
    the orthonormal DST-I (Dirichlet) or DFT (periodic) basis of the grid."""
    dims = [int(d) for d in dims]
    shape = tuple(reversed(dims))
    lam = eig_grid(kind, dims, kappa2, periodic, scale)
    e = np.zeros(int(np.prod(dims)))
    e[j] = 1.0
    e = e.reshape(shape)
    if periodic:
        y = sfft.ifftn(np.log(lam) * sfft.fftn(e, norm="ortho"), norm="ortho").real
    else:
        y = sfft.idstn(np.log(lam) * sfft.dstn(e, type=1, norm="ortho"), type=1, norm="ortho")
    return y.reshape(-1)


def quadratic_forms(kind, dims, kappa2, periodic, Z: np.ndarray, f=np.log, scale=1.0) -> np.ndarray:
    """z_k^T f(Q) z_k for each column z_k of Z (n x s): sum_i f(lambda_i) |u_i^T z_k|^2."""
    dims = [int(d) for d in dims]
    shape = tuple(reversed(dims))
    flam = f(eig_grid(kind, dims, kappa2, periodic, scale))
    Z = np.asarray(Z)
    return np.array([float(np.sum(flam * spectral_coeffs(Z[:, k].reshape(shape), periodic)))
                     for k in range(Z.shape[1])])


def apply_function(kind, dims, kappa2, periodic, V: np.ndarray, f, scale=1.0) -> np.ndarray:
    """f(Q) V exactly for the columns of V (n x s): U diag(f(lambda)) U^T V with U the
    orthonormal DST-I (Dirichlet) or DFT (periodic) basis of the grid."""
    dims = [int(d) for d in dims]
    shape = tuple(reversed(dims))
    flam = f(eig_grid(kind, dims, kappa2, periodic, scale))
    V = np.asarray(V, dtype=np.float64)
    out = np.empty_like(V)
    for k in range(V.shape[1]):
        v = V[:, k].reshape(shape)
        if periodic:
            y = sfft.ifftn(flam * sfft.fftn(v, norm="ortho"), norm="ortho").real
        else:
            y = sfft.idstn(flam * sfft.dstn(v, type=1, norm="ortho"), type=1, norm="ortho")
        out[:, k] = y.reshape(-1)
    return out
