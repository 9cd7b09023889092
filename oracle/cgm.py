"""Oracle: multi-shift conjugate gradients (CG-M / COCG-M), plain numpy.

Sec. 2.1: the shifted systems (Q - sigma_l I) x = v share the Krylov space
K_k(Q, v) = K_k(Q - sigma_l I, v), so every shifted iterate follows from the
real seed CG on Q x = v with no extra matrix-vector products (Jegerlehner's
CG-M); complex shifts use the bilinear form x^T y (COCG-M).

Written here for systems (A + s I) x = v with s = -sigma.  With the seed CG
scalars alpha_k, beta_k (alpha_{-1} = 1, beta_{-1} = 0, zeta_{-1} = zeta_0 = 1)
the shifted residuals are r^s_k = zeta_k r_k with
    zeta_{k+1} = zeta_k zeta_{k-1} alpha_{k-1} /
                 ( alpha_{k-1} zeta_{k-1} (1 + s alpha_k)
                   + alpha_k beta_{k-1} (zeta_{k-1} - zeta_k) ),
    alpha^s_k = alpha_k zeta_{k+1} / zeta_k,
    beta^s_k  = beta_k (zeta_{k+1} / zeta_k)^2,
    x^s_{k+1} = x^s_k + alpha^s_k p^s_k,
    p^s_{k+1} = zeta_{k+1} r_{k+1} + beta^s_k p^s_k.
Projected form (only v^T x^s is needed for v^T f_N(Q) v):
    pi_{k+1}  = pi_k + alpha^s_k phi_k,           pi_0 = 0      (pi = v^T x^s)
    phi_{k+1} = zeta_{k+1} v^T r_{k+1} + beta^s_k phi_k,  phi_0 = v^T v (phi = v^T p^s).
A shifted system is converged when |zeta_k| ||r_k|| <= tol ||v|| (its own
relative residual); it is then frozen.  The seed is converged when
||r_k|| <= tol ||v||.  Iteration stops when the seed and every shift are
converged, or at maxiter.
"""
from __future__ import annotations

import numpy as np


class NotSPD(RuntimeError):
    pass


def cgm(matvec, v: np.ndarray, s: np.ndarray, tol: float, maxiter: int,
        keep_vectors: bool = False):
    """Run CG-M for (A + s_l I) x = v for all l, plus the seed s = 0.

    Returns dict with:
      pi     : complex (L,)  v^T x^{s_l}   (projected recurrence)
      x0     : real (n,)     seed solution A^{-1} v
      xs     : complex (L, n) shifted solutions (keep_vectors only)
      iters  : iterations taken
      alphas, betas : seed CG scalars
      converged : bool
    """
    v = np.asarray(v, dtype=np.float64)
    s = np.asarray(s, dtype=np.complex128)
    L = s.size
    n = v.size
    vnorm = float(np.sqrt(v @ v))
    out = dict(pi=np.zeros(L, complex), x0=np.zeros(n), iters=0, alphas=[], betas=[],
               converged=True)
    if vnorm == 0.0:
        if keep_vectors:
            out["xs"] = np.zeros((L, n), complex)
        return out
    r = v.copy()
    p = v.copy()
    x0 = np.zeros(n)
    rho = float(r @ r)
    zeta_prev = np.ones(L, complex)
    zeta = np.ones(L, complex)
    alpha_prev, beta_prev = 1.0, 0.0
    pi = np.zeros(L, complex)
    phi = np.full(L, float(v @ v), complex)
    active = np.ones(L, bool)
    seed_active = True
    if keep_vectors:
        xs = np.zeros((L, n), complex)
        ps = np.tile(v.astype(complex), (L, 1))
    k = 0
    while k < maxiter:
        w = matvec(p)
        pw = float(p @ w)
        if not pw > 0.0:
            raise NotSPD("p^T A p <= 0 at iteration %d" % k)
        alpha = rho / pw
        x0 += alpha * p
        r_new = r - alpha * w
        rho_new = float(r_new @ r_new)
        beta = rho_new / rho
        vr = float(v @ r_new)
        a = active
        zeta_next = np.where(a, zeta * zeta_prev * alpha_prev /
                             (alpha_prev * zeta_prev * (1.0 + s * alpha)
                              + alpha * beta_prev * (zeta_prev - zeta)), zeta)
        ratio = np.where(a, zeta_next / np.where(a, zeta, 1.0), 1.0)
        alpha_s = alpha * ratio
        beta_s = beta * ratio * ratio
        pi = np.where(a, pi + alpha_s * phi, pi)
        if keep_vectors:
            xs[a] += alpha_s[a, None] * ps[a]
            ps[a] = zeta_next[a, None] * r_new[None, :] + beta_s[a, None] * ps[a]
        phi = np.where(a, zeta_next * vr + beta_s * phi, phi)
        zeta_prev = np.where(a, zeta, zeta_prev)
        zeta = zeta_next
        out["alphas"].append(alpha)
        out["betas"].append(beta)
        alpha_prev, beta_prev = alpha, beta
        p = r_new + beta * p
        r = r_new
        rho = rho_new
        k += 1
        rn = np.sqrt(rho_new)
        active = active & (np.abs(zeta) * rn > tol * vnorm)
        seed_active = rn > tol * vnorm
        if not seed_active and not active.any():
            break
    out.update(pi=pi, x0=x0, iters=k, converged=not (seed_active or active.any()))
    if keep_vectors:
        out["xs"] = xs
    return out
