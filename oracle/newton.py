"""Newton-based polynomial preconditioner (paper Sec. 2, Algorithm 1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).
"""
from __future__ import annotations

import numpy as np


def newton_zetas(alpha0: float, beta0: float, nlev: int) -> np.ndarray:
    """zeta_0..zeta_nlev of Algorithm 1, step 3 (Eq. zetaNewt).

    zeta_0 = 2/(alpha_0+beta_0), zeta_1 = 2/(1 + 2 alpha_0 zeta_0 - (alpha_0 zeta_0)^2),
    zeta_i = 2/(1 + 2 zeta_{i-1} - zeta_{i-1}^2) for i >= 2.

    The modified parameter of Sec. 4 enters through the interval: with theta
    scaled by s the caller passes alpha_0 = s theta - delta and beta_0 =
    s theta + delta (the interval of the scaled Chebyshev polynomial).
    """
    z = np.empty(nlev + 1)
    z[0] = 2.0 / (alpha0 + beta0)
    if nlev >= 1:
        a = alpha0 * z[0]
        z[1] = 2.0 / (1.0 + 2.0 * a - a * a)
    for i in range(2, nlev + 1):
        z[i] = 2.0 / (1.0 + 2.0 * z[i - 1] - z[i - 1] ** 2)
    return z


def newton_apply(matvec, u: np.ndarray, zetas: np.ndarray, level: int) -> np.ndarray:
    """P_level u by the recursion of Algorithm 1, step 5 (Eq. recursive).

    P_0 u = zeta_0 u,  P_{j+1} u = zeta_{j+1} (2 P_j u - P_j A P_j u).
    Uses 2^level - 1 matrix-vector products.
    """
    if level == 0:
        return zetas[0] * u
    pu = newton_apply(matvec, u, zetas, level - 1)
    papu = newton_apply(matvec, matvec(pu), zetas, level - 1)
    return zetas[level] * (2.0 * pu - papu)


def hotelling_dense(A: np.ndarray, zetas: np.ndarray, nlev: int) -> np.ndarray:
    """Dense P_nlev from the scaled Hotelling iteration (Sec. 2, Eq. newrec).

    P_0 = zeta_0 I and P_{j+1} = zeta_{j+1} (2 P_j - P_j A P_j); this is
    Eq. newrec with each level's scale applied to the new iterate, which is
    the matrix form of the scalar recursion Eq. recpolr, r_{2^j-1}(A) = P_j.
    """
    n = A.shape[0]
    P = zetas[0] * np.eye(n)
    for j in range(nlev):
        P = zetas[j + 1] * (2.0 * P - P @ A @ P)
    return P
