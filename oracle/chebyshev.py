"""Chebyshev polynomial preconditioner (paper Sec. 3 and Sec. 4).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Notation follows Sec. 3: the spectral interval [alpha, beta], theta =
(beta+alpha)/2, delta = (beta-alpha)/2, sigma = theta/delta, sigma_k =
T_k(sigma), rho_k = sigma_k/sigma_{k+1}.

Modified parameter (Sec. 4, "the optimal parameters are not optimal"): theta
is multiplied by a scale s (1.01 in Sec. 4, 1.001 in Sec. 5).  Reading used
here (the only one of the readings tried that reproduces Table 3's right
half to every printed digit): theta' = s*theta, delta unchanged, sigma =
theta'/delta.  The resulting p_k is the exact Chebyshev polynomial of the
shifted interval [theta'-delta, theta'+delta].
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class ChebParams:
    theta: float   # theta' = s (alpha+beta)/2
    delta: float   # (beta-alpha)/2
    sigma: float   # theta'/delta


def cheb_params(alpha: float, beta: float, s: float = 1.0) -> ChebParams:
    """theta, delta, sigma of Sec. 3 with theta scaled by s (Sec. 4)."""
    if not (0.0 < alpha < beta):
        raise ValueError("need 0 < alpha < beta")
    theta = s * (beta + alpha) / 2.0
    delta = (beta - alpha) / 2.0
    return ChebParams(theta=theta, delta=delta, sigma=theta / delta)


def rho_sequence(sigma: float, m: int) -> np.ndarray:
    """rho_0 = 1/sigma, rho_k = 1/(2 sigma - rho_{k-1}) (Sec. 3, Eq. rhocheb)."""
    rho = np.empty(m + 1)
    rho[0] = 1.0 / sigma
    for k in range(1, m + 1):
        rho[k] = 1.0 / (2.0 * sigma - rho[k - 1])
    return rho


def p_k_recurrence(x, prm: ChebParams, m: int):
    """Scalar p_m(x) by the three-term recursion for {p_k} in Sec. 3.

    p_{-1} = 0, p_0 = 1/theta,
    p_k = rho_k (2 sigma (1 - x/theta) p_{k-1} - rho_{k-1} p_{k-2} + 2/delta).
    Works elementwise on arrays.
    """
    x = np.asarray(x, dtype=np.float64)
    rho = rho_sequence(prm.sigma, m)
    p_prev = np.zeros_like(x)              # p_{-1}
    p_cur = np.full_like(x, 1.0 / prm.theta)  # p_0
    for k in range(1, m + 1):
        p_next = rho[k] * (2.0 * prm.sigma * (1.0 - x / prm.theta) * p_cur
                           - rho[k - 1] * p_prev + 2.0 / prm.delta)
        p_prev, p_cur = p_cur, p_next
    return p_cur


def _cheb_T(n: int, t):
    """First-kind Chebyshev polynomial T_n(t) by its three-term recursion (Eq. 3term)."""
    t = np.asarray(t, dtype=np.float64)
    if n == 0:
        return np.ones_like(t)
    t_prev, t_cur = np.ones_like(t), t.copy()
    for _ in range(1, n):
        t_prev, t_cur = t_cur, 2.0 * t * t_cur - t_prev
    return t_cur


def p_k_closed_form(x, prm: ChebParams, m: int):
    """p_m(x) = (1 - q_{m+1}(x))/x with q_{m+1}(x) = T_{m+1}(sigma - x/delta)/T_{m+1}(sigma).

    Sec. 3, Eq. cheb / Eq. qT (the minimax solution of Eq. maxmin), written
    on the (possibly shifted) interval of ``prm``.  Valid for x != 0.
    """
    x = np.asarray(x, dtype=np.float64)
    q = _cheb_T(m + 1, prm.sigma - x / prm.delta) / _cheb_T(m + 1, np.float64(prm.sigma))
    return (1.0 - q) / x


def cheb_apply(matvec, r: np.ndarray, prm: ChebParams, m: int) -> np.ndarray:
    """z = p_m(A) r by Algorithm 2 (Sec. 3), m matrix-vector products, no dots.

    Index reading: the loop body uses rho_k and rho_{k-1}, as the p_k
    recursion it is derived from requires (and as the k = 1 line does with
    rho_1); the printed rho_{k+1}, rho_k does not reproduce Table 3.
    """
    rho = rho_sequence(prm.sigma, m)
    x_old = r / prm.theta
    if m == 0:
        return x_old
    x = (2.0 * rho[1] / prm.delta) * (2.0 * r - matvec(r) / prm.theta)
    for k in range(2, m + 1):
        z = (2.0 / prm.delta) * (r - matvec(x))
        x_new = rho[k] * (2.0 * prm.sigma * x - rho[k - 1] * x_old + z)
        x_old, x = x, x_new
    return x
