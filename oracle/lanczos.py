"""Extreme-eigenvalue estimates for the interval [alpha, beta].

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper (Sec. 5.1) estimates beta_0 with a few power iterations and
alpha_0 with an unpreconditioned DACG run to 1e-2; Algorithm 1 step 1 and
Algorithm 2 only require an interval containing the spectrum.  The workloads
with no closed-form spectrum take their interval from a short Lanczos run
(without reorthogonalisation) instead, with a safeguarded upper end, because
an underestimated beta makes P_k(A) indefinite (|T_{k+1}| grows outside the
interval).
"""
from __future__ import annotations

import numpy as np


def lanczos_bounds(matvec, v0: np.ndarray, steps: int, gershgorin: float | None = None,
                   keep_basis: bool = False):
    """Lanczos estimate of [lambda_min, lambda_max] with a safe upper end.

    Recurrence (no reorthogonalisation), v_1 = v0/||v0||, beta_0 = 0:
        w = A v_j - beta_{j-1} v_{j-1};  a_j = (w, v_j);  w = w - a_j v_j;
        b_j = ||w||;  v_{j+1} = w / b_j.
    The Ritz values are the eigenvalues of the tridiagonal T = tridiag(b, a, b).
    Upper end: max(ritz_max + |b_m s_m|, 1.01 ritz_max), where s_m is the last
    component of the top Ritz vector (the residual bound for that pair); if a
    Gershgorin bound is supplied and lies in [ritz_max, that value) it is used
    instead.  Lower end: ritz_min (an overestimate, which is safe: eigenvalues
    below alpha are mapped into (0, 1)).

    Returns (lower, upper, info) with info = dict(alpha=a, beta=b, ritz=theta,
    ritz_vectors=S, resid=|b_m s_m|); with keep_basis the Lanczos vectors
    v_1..v_m are kept as the columns of info["basis"] (n x m), so that a caller
    can form the top Ritz vector y = V s and check the residual bound
    ||A y - theta y|| = |b_m s_m| against the matrix itself.
    """
    v = v0 / np.linalg.norm(v0)
    v_prev = np.zeros_like(v)
    b_prev = 0.0
    a_list, b_list = [], []
    basis = []
    for _ in range(steps):
        if keep_basis:
            basis.append(v.copy())
        w = matvec(v) - b_prev * v_prev
        a = float(np.dot(w, v))
        w = w - a * v
        b = float(np.linalg.norm(w))
        a_list.append(a)
        b_list.append(b)
        if b == 0.0:
            break
        v_prev, v = v, w / b
        b_prev = b
    m = len(a_list)
    T = np.diag(a_list) + np.diag(b_list[:m - 1], 1) + np.diag(b_list[:m - 1], -1)
    theta, S = np.linalg.eigh(T)
    rmin, rmax = float(theta[0]), float(theta[-1])
    resid = abs(b_list[m - 1] * S[m - 1, -1])
    upper = max(rmax + resid, 1.01 * rmax)
    if gershgorin is not None and rmax <= gershgorin < upper:
        upper = float(gershgorin)
    info = dict(alpha=np.array(a_list), beta=np.array(b_list), ritz=theta, ritz_vectors=S, resid=resid)
    if keep_basis:
        info["basis"] = np.stack(basis, axis=1)
    return rmin, upper, info


def power_method(matvec, v0: np.ndarray, iters: int) -> float:
    """Rayleigh quotient after ``iters`` power iterations (Sec. 5.1's beta_0 estimate).

    The paper prints no values from its runs; pinned by closed forms in the
    tests: for a diagonal matrix the estimate after m iterations equals
    sum l^(2m-1) v0^2 / sum l^(2m-2) v0^2 exactly, and on the 64 x 64
    Laplacian it rises towards 8 sin^2(64 pi / 130) from below.
    """
    v = v0 / np.linalg.norm(v0)
    lam = 0.0
    for _ in range(iters):
        w = matvec(v)
        lam = float(np.dot(v, w))
        v = w / np.linalg.norm(w)
    return lam
