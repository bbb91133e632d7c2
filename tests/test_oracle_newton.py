"""Pins for oracle/newton.py: Theorem 3.1 (Newton == Chebyshev), the Hotelling
error bound and Theorem 2.1's interval map, checked on tiny dense matrices
against an eigendecomposition built here (not by the oracle)."""
import numpy as np
import pytest

import oracle as O


def spd(n, lo, hi, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.sort(np.concatenate([[lo, hi], rng.uniform(lo, hi, n - 2)]))
    return (Q * lam) @ Q.T, lam, Q


def cheb_poly_dense(A_lam, Q, alpha, beta, m):
    """p_m(A) from the eigendecomposition, p_m from T_{m+1} = cosh/cos closed form."""
    theta, delta = (alpha + beta) / 2, (beta - alpha) / 2
    sigma = theta / delta
    t = sigma - A_lam / delta
    T = np.where(np.abs(t) <= 1, np.cos((m + 1) * np.arccos(np.clip(t, -1, 1))),
                 np.cosh((m + 1) * np.arccosh(np.maximum(np.abs(t), 1))))
    q = T / np.cosh((m + 1) * np.arccosh(sigma))
    p = (1 - q) / A_lam
    return (Q * p) @ Q.T


@pytest.mark.parametrize("nlev", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("s", [1.0, 1.01])
def test_theorem31_newton_equals_chebyshev(nlev, s):
    A, lam, Q = spd(30, 0.01, 1.9, seed=nlev)
    alpha, beta = lam[0], lam[-1]
    prm = O.cheb_params(alpha, beta, s)
    # the scaled-theta polynomial is the Chebyshev one of the shifted interval
    a0, b0 = prm.theta - prm.delta, prm.theta + prm.delta
    z = O.newton_zetas(a0, b0, nlev)
    P_newton = O.hotelling_dense(A, z, nlev)
    m = 2 ** nlev - 1
    P_ref = cheb_poly_dense(lam, Q, a0, b0, m)
    assert np.max(np.abs(P_newton - P_ref)) <= 1e-11 * np.max(np.abs(P_ref))
    # Algorithm 1's recursive vector apply and Algorithm 2 agree column by column
    P_rec = np.column_stack([O.newton_apply(lambda u: A @ u, e, z, nlev) for e in np.eye(30)])
    P_alg2 = np.column_stack([O.cheb_apply(lambda u: A @ u, e, prm, m) for e in np.eye(30)])
    assert np.max(np.abs(P_rec - P_ref)) <= 1e-11 * np.max(np.abs(P_ref))
    assert np.max(np.abs(P_alg2 - P_ref)) <= 1e-11 * np.max(np.abs(P_ref))


def test_zeta_equals_chi():
    """zeta_j = 2 sigma_{2^{j-1}}^2 / sigma_{2^j}, sigma_k = T_k(sigma) (Thm 3.1)."""
    alpha, beta = 0.003, 1.7
    sigma = (alpha + beta) / (beta - alpha)
    z = O.newton_zetas(alpha, beta, 6)
    Tk = lambda k: np.cosh(k * np.arccosh(sigma))  # noqa: E731
    for j in range(1, 7):
        chi = 2 * Tk(2 ** (j - 1)) ** 2 / Tk(2 ** j)
        assert abs(z[j] - chi) <= 1e-13 * chi
    assert abs(z[0] - 2 / (alpha + beta)) < 1e-15


def test_hotelling_error_bound():
    """Unscaled Newton: ||I - P_j A|| <= ||I - P_0 A||^(2^j) (Sec. 2)."""
    A, lam, _ = spd(20, 0.2, 1.5, seed=3)
    c = 1.0
    r0 = np.linalg.norm(np.eye(20) - c * A, 2)
    for j in range(5):
        z = np.array([c] + [1.0] * j)
        P = O.hotelling_dense(A, z, j)
        e = np.linalg.norm(np.eye(20) - P @ A, 2)
        assert e <= r0 ** (2 ** j) * (1 + 1e-10) + 1e-14


def test_theorem21_interval_map():
    """Eigenvalues of P_0 A in [a, 2 - a] map into [2a - a^2, 1] after one step."""
    A, lam, _ = spd(25, 0.1, 1.9, seed=4)
    P1 = O.hotelling_dense(A, np.array([1.0, 1.0]), 1)
    mu = np.linalg.eigvalsh(0.5 * (P1 @ A + A @ P1))
    a = 0.1
    assert mu.min() >= 2 * a - a * a - 1e-12 and mu.max() <= 1 + 1e-12


@pytest.mark.parametrize("nlev", [0, 1, 2, 3, 4])
def test_newton_matvec_count(nlev):
    calls = [0]

    def mv(u):
        calls[0] += 1
        return 2.0 * u

    O.newton_apply(mv, np.ones(3), O.newton_zetas(0.5, 3.0, nlev), nlev)
    assert calls[0] == 2 ** nlev - 1
