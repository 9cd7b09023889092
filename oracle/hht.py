"""Oracle: rational approximation of log from a conformally mapped contour integral.

The paper (Sec. 2.1, Eq. "eq_rat_app") evaluates log(Q) v through Cauchy's
integral over a contour enclosing the spectrum and avoiding (-inf, 0], using
the Hale-Higham-Trefethen midpoint rule, giving
    log(Q) v  ~  f_N(Q) v = sum_l alpha_l (Q - sigma_l I)^{-1} v.
The paper gives neither nodes nor weights; this module writes them out from
that construction (the square-root variant, whose error rate
exp(-2 pi^2 N / (log(M/m) + 6)) carries the "+6" the paper prints):

  1. substitute z = w^2:  log A = (1/2 pi i) oint 4 w log(w) (w^2 I - A)^{-1} dw,
     the w-contour enclosing [a, b] = [sqrt(m), sqrt(M)] in Re w > 0;
  2. the rectangle [-K, K] x [0, K'] maps onto the upper half w-plane by
     u = sn(t | k^2), w = sqrt(ab) (1/k + u) / (1/k - u), with
     k = (r - 1)/(r + 1), r = sqrt(b/a); the bottom edge lands on [a, b];
  3. midpoint rule on the line Im t = K'/2:  t_j = -K + (j - 1/2) h + i K'/2,
     h = 2K/N, j = 1..N; the lower half of the contour is the complex
     conjugate, so for real A and v
        log(A) v ~ Re sum_j alpha_j (A - sigma_j I)^{-1} v,
        sigma_j = w_j^2,  alpha_j = -(4 i h / pi) w_j log(w_j) w'(t_j),
        w'(t) = sqrt(ab) (2/k) cn dn / (1/k - sn)^2.

Complete elliptic integrals and real-argument Jacobi functions come from
scipy.special (parameter m = k^2); the complex argument uses the addition
formulas of Abramowitz & Stegun 16.21.
"""
from __future__ import annotations

import numpy as np
from scipy import special


def jacobi_complex(x: np.ndarray, y: float, m: float):
    """sn, cn, dn at x + i y (A&S 16.21.1-16.21.4), parameter m."""
    s, c, d, _ = special.ellipj(x, m)
    s1, c1, d1, _ = special.ellipj(np.full_like(x, y), 1.0 - m)
    den = c1 * c1 + m * s * s * s1 * s1
    sn = (s * d1 + 1j * c * d * s1 * c1) / den
    cn = (c * c1 - 1j * s * d * s1 * d1) / den
    dn = (d * c1 * d1 - 1j * m * s * c * s1) / den
    return sn, cn, dn


def log_nodes(lmin: float, lmax: float, N: int):
    """(sigma, alpha), each complex of length N, for log on [lmin, lmax]."""
    if not (0 < lmin <= lmax) or N < 1:
        raise ValueError("need 0 < lmin <= lmax and N >= 1")
    a, b = np.sqrt(lmin), np.sqrt(lmax)
    r = np.sqrt(b / a)
    k = (r - 1.0) / (r + 1.0)
    if k <= 0.0:
        raise ValueError("degenerate interval: lmin == lmax")
    m = k * k
    K = special.ellipk(m)
    Kp = special.ellipk(1.0 - m)
    h = 2.0 * K / N
    x = -K + (np.arange(1, N + 1) - 0.5) * h
    sn, cn, dn = jacobi_complex(x, Kp / 2.0, m)
    g = np.sqrt(a * b)
    w = g * (1.0 / k + sn) / (1.0 / k - sn)
    dw = g * (2.0 / k) * cn * dn / (1.0 / k - sn) ** 2
    sigma = w * w
    alpha = -(4j * h / np.pi) * w * np.log(w) * dw
    return sigma, alpha


def f_N(lam: np.ndarray, sigma: np.ndarray, alpha: np.ndarray) -> np.ndarray:
    """Scalar rational approximant Re sum_l alpha_l / (lambda - sigma_l)."""
    lam = np.asarray(lam, dtype=np.float64)
    out = np.zeros(lam.shape)
    for s, al in zip(sigma, alpha):
        out += np.real(al / (lam - s))
    return out


def certificate(lmin: float, lmax: float, sigma, alpha, samples: int = 4001) -> float:
    """max |f_N(lambda) - log(lambda)| over log-spaced samples of [lmin, lmax]."""
    lam = np.exp(np.linspace(np.log(lmin), np.log(lmax), samples))
    return float(np.max(np.abs(f_N(lam, sigma, alpha) - np.log(lam))))


def rate_bound(lmin: float, lmax: float, N: int) -> float:
    """exp(-2 pi^2 N / (log(M/m) + 6)), the square-root method's rate."""
    return float(np.exp(-2.0 * np.pi ** 2 * N / (np.log(lmax / lmin) + 6.0)))


# ---------------------------------------------------------------- inverse square root
# Same contour and quadrature with f(z) = z^{-1/2}: after z = w^2 the integrand
# f(w^2) 2w (w^2 I - A)^{-1} = 2 (w^2 I - A)^{-1} (principal branch, Re w > 0), so
#   A^{-1/2} v ~ Re sum_j beta_j (A - sigma_j I)^{-1} v,  beta_j = -(2 i h / pi) w'(t_j),
# with the nodes sigma_j of log_nodes.  Used to draw x = Q^{-1/2} z ~ N(0, Q^{-1}).

def invsqrt_nodes(lmin: float, lmax: float, N: int):
    """(sigma, beta) for z^{-1/2} on [lmin, lmax] (same sigma as log_nodes)."""
    if not (0 < lmin <= lmax) or N < 1:
        raise ValueError("need 0 < lmin <= lmax and N >= 1")
    a, b = np.sqrt(lmin), np.sqrt(lmax)
    r = np.sqrt(b / a)
    k = (r - 1.0) / (r + 1.0)
    if k <= 0.0:
        raise ValueError("degenerate interval: lmin == lmax")
    m = k * k
    K = special.ellipk(m)
    Kp = special.ellipk(1.0 - m)
    h = 2.0 * K / N
    x = -K + (np.arange(1, N + 1) - 0.5) * h
    sn, cn, dn = jacobi_complex(x, Kp / 2.0, m)
    g = np.sqrt(a * b)
    w = g * (1.0 / k + sn) / (1.0 / k - sn)
    dw = g * (2.0 / k) * cn * dn / (1.0 / k - sn) ** 2
    return w * w, -(2j * h / np.pi) * dw


def invsqrt_certificate(lmin: float, lmax: float, sigma, beta, samples: int = 4001) -> float:
    """max |f_N(lambda) sqrt(lambda) - 1| (relative error) over [lmin, lmax]."""
    lam = np.exp(np.linspace(np.log(lmin), np.log(lmax), samples))
    return float(np.max(np.abs(f_N(lam, sigma, beta) * np.sqrt(lam) - 1.0)))
