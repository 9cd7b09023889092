"""Maximum-likelihood fit of GMRF hyperparameters with the probed log det (Sec. 3).

Model (Sec. 3, with kappa^2 for the paper's kappa and the prior scale s for its
precision factor): a field observed directly, y ~ N(0, Q^{-1}), with
    Q = s * Q0(kappa^2),   Q0 = kappa^2 I - Lap (5- or 7-point)  or  (kappa^2 I - Lap)^2,
on a regular grid.  For samples y_1..y_S the log-likelihood, constants dropped, is
    l = S/2 log det Q - 1/2 sum_k y_k^T Q y_k,
with log det Q and d log det Q / d(kappa^2, s) from the probed estimate of a context
(ld_logdet_grad; the colouring distance sets the accuracy, Table 1's subject) and the
quadratic forms from operator applications on the device (ld_apply).  The parameters
are optimised in log space, eta = (log kappa^2, log s), by a modified Newton iteration:
the Hessian is formed by central differences of the gradient, its eigenvalues are
clamped negative (an ascent direction whatever the curvature), the step is limited to
a trust region in log space and halved until the objective increases.

sample() draws the synthetic fields: x = Q^{-1/2} z for standard normal z given by the
caller (ld_invsqrt_mv).
"""
from __future__ import annotations

import numpy as np

from . import (LD_FP64, LD_P_KAPPA2, LD_P_SCALE, LD_STENCIL_2D13_SQ, LD_STENCIL_2D5, grid_matrix,
               ld_apply, ld_create, ld_invsqrt_mv, ld_logdet_grad, ld_set_params, options)


def sample(kind, dims, kappa2, scale, z, periodic=False, n_shifts=24, tol=1e-10):
    """Fields x = Q^{-1/2} z ~ N(0, Q^{-1}) for the columns of z (n x S)."""
    ctx = ld_create(grid_matrix(kind, dims, kappa2, periodic=periodic, scale=scale), 1, n_shifts, tol,
                    options(precision=LD_FP64))
    x, _ = ld_invsqrt_mv(ctx, z)
    return x


class Likelihood:
    """l(eta) and its gradient for eta = (log kappa^2, log s) on fixed samples Y (n x S)."""

    def __init__(self, kind, dims, Y, distance, periodic=False, n_shifts=20, tol=1e-9, precision=LD_FP64):
        self.kind, self.dims, self.periodic = kind, tuple(dims), periodic
        self.Y = np.ascontiguousarray(Y, dtype=np.float64)
        if self.Y.ndim == 1:
            self.Y = self.Y[:, None]
        self.S = self.Y.shape[1]
        self.ctx = ld_create(grid_matrix(kind, self.dims, 1.0, periodic=periodic), distance, n_shifts, tol,
                             options(precision=precision))
        # the 13-point square needs Q1 y = (kappa^2 I - Lap) y for dQ/dkappa^2 = 2 s Q1
        self.q1 = None
        if kind == LD_STENCIL_2D13_SQ:
            self.q1 = ld_create(grid_matrix(LD_STENCIL_2D5, self.dims, 1.0, periodic=periodic), 1, 8, 1e-6,
                                options(precision=LD_FP64))
        self.evaluations = 0

    def __call__(self, eta):
        k2, s = float(np.exp(eta[0])), float(np.exp(eta[1]))
        ld_set_params(self.ctx, k2, 0.0, s)
        logdet, g, _ = ld_logdet_grad(self.ctx, [LD_P_KAPPA2, LD_P_SCALE])
        QY = ld_apply(self.ctx, self.Y)
        quad = float(np.sum(self.Y * QY))
        if self.q1 is None:
            dquad_k2 = s * float(np.sum(self.Y * self.Y))          # dQ/dkappa^2 = s I
        else:
            ld_set_params(self.q1, k2, 0.0, 1.0)
            dquad_k2 = 2.0 * s * float(np.sum(self.Y * ld_apply(self.q1, self.Y)))
        dquad_s = quad / s                                          # dQ/ds = Q / s
        val = 0.5 * self.S * logdet - 0.5 * quad
        grad = np.array([k2 * (0.5 * self.S * g[0] - 0.5 * dquad_k2),
                         s * (0.5 * self.S * g[1] - 0.5 * dquad_s)])
        self.evaluations += 1
        return val, grad


def fit(lik: Likelihood, kappa2_0, scale_0, max_iter=40, h=1e-3, gtol=1e-7, max_step=1.0):
    """Modified Newton ascent of lik from (kappa2_0, scale_0), steps at most max_step in
    each log parameter; returns a dict with the estimates, the log-likelihood, the
    iteration count and the path."""
    eta = np.log([kappa2_0, scale_0]).astype(np.float64)
    val, g = lik(eta)
    path = [(float(np.exp(eta[0])), float(np.exp(eta[1])), val)]
    it = 0
    for it in range(1, max_iter + 1):
        H = np.empty((2, 2))
        for i in range(2):
            e = np.zeros(2)
            e[i] = h
            H[:, i] = (lik(eta + e)[1] - lik(eta - e)[1]) / (2 * h)
        H = 0.5 * (H + H.T)
        lam, U = np.linalg.eigh(H)
        floor = 1e-3 * max(1e-12, float(np.abs(lam).max()))
        lam = np.minimum(lam, -floor)
        step = -(U @ ((U.T @ g) / lam))
        big = float(np.abs(step).max())
        if big > max_step:                      # trust region in log space
            step *= max_step / big
        improved = False
        for _ in range(30):
            cand_val, cand_g = lik(eta + step)
            if cand_val >= val:
                improved = True
                break
            step *= 0.5
        if not improved:
            break
        eta, val, g = eta + step, cand_val, cand_g
        path.append((float(np.exp(eta[0])), float(np.exp(eta[1])), val))
        if np.abs(g).max() <= gtol * (1.0 + abs(val)) or np.abs(step).max() < 1e-9:
            break
    return {"kappa2": float(np.exp(eta[0])), "scale": float(np.exp(eta[1])), "loglik": val,
            "iterations": it, "evaluations": lik.evaluations, "path": path}


def fit_schedule(kind, dims, Y, distances=(2, 4, 8), kappa2_0=1.0, scale_0=1.0, periodic=False,
                 **kw):
    """Sec. 3's schedule: cheap small-distance colourings for the first iterations, larger
    ones for the last; each fit starts from the previous estimates.  Returns the list of
    (distance, fit result)."""
    out = []
    k2, s = kappa2_0, scale_0
    for d in distances:
        res = fit(Likelihood(kind, dims, Y, d, periodic=periodic), k2, s, **kw)
        out.append((d, res))
        k2, s = res["kappa2"], res["scale"]
    return out
