"""Pins for oracle/chebyshev.py and oracle/spectrum.py.

Each test checks the oracle against something fixed outside it: the values
printed in Table 3, the textbook closed form of T_n (cos/cosh, not the
three-term recursion the oracle uses), exact eigenpairs of diagonal and
Laplacian matrices, and the Chebyshev minimax bound of Eq. cheb.
"""
import os

import numpy as np
import pytest

import oracle as O
import workloads as W
from conftest import GOLDEN


def T_closed(n, t):
    """Textbook T_n: cos(n arccos t) on [-1, 1], sign-adjusted cosh outside."""
    t = np.asarray(t, dtype=np.float64)
    out = np.empty_like(t)
    inside = np.abs(t) <= 1.0
    out[inside] = np.cos(n * np.arccos(t[inside]))
    big = ~inside
    out[big] = np.sign(t[big]) ** n * np.cosh(n * np.arccosh(np.abs(t[big])))
    return out


def p_closed(x, alpha, beta, s, m):
    """p_m on the interval [alpha, beta] shifted by (s-1)theta, via T_closed."""
    theta = s * (alpha + beta) / 2
    delta = (beta - alpha) / 2
    sigma = theta / delta
    q = T_closed(m + 1, sigma - np.asarray(x) / delta) / T_closed(m + 1, np.array([sigma]))[0]
    return (1 - q) / np.asarray(x)


def _table3_rows():
    rows = []
    with open(os.path.join(GOLDEN, "table3.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            s, m, it, mx, mn, l, k = line.split()
            rows.append((float(s), int(m), int(it), mx, mn, int(l), k))
    return rows


def _printed_tol(txt):
    """Half a unit in the last printed digit of a number printed as ``txt``."""
    if "e" in txt:
        mant, ex = txt.split("e")
        dec = len(mant.split(".")[1])
        return 0.5 * 10.0 ** (int(ex) - dec)
    dec = len(txt.split(".")[1])
    return 0.5 * 10.0 ** (-dec)


def _lap78_scaled_eigs():
    # eigenvalues of the 78^2 5-point Laplacian (diagonal 4) divided by 4:
    # the diagonally scaled matrix of Sec. 4
    i = np.arange(1, 79)
    l1 = 4 * np.sin(i * np.pi / (2 * 79)) ** 2
    return (l1[:, None] + l1[None, :]).ravel() / 4.0


@pytest.mark.parametrize("row", _table3_rows(), ids=lambda r: f"s{r[0]}-m{r[1]}")
def test_table3_spectrum(row):
    s, m, _, mx, mn, l, k = row
    lam = _lap78_scaled_eigs()
    prm = O.cheb_params(lam.min(), lam.max(), s)
    st = O.preconditioned_spectrum_stats(lam, prm, m)
    assert abs(st["mu_max"] - float(mx)) <= _printed_tol(mx)
    assert abs(st["mu_min"] - float(mn)) <= _printed_tol(mn)
    assert st["l"] == l
    assert abs(st["kappa"] - float(k)) <= _printed_tol(k)


def test_table3_scaling_is_diag_over_4():
    A = W.laplacian_2d_5pt(78, 78)
    v, dis = O.jacobi_scale_csr(A.rowptr, A.col, A.val, A.n)
    assert np.allclose(dis, 0.5)
    assert np.array_equal(v, A.val / 4.0)


@pytest.mark.parametrize("alpha,beta,s,m", [(0.01, 2.0, 1.0, 7), (1e-3, 1.0, 1.001, 20),
                                             (0.3, 6.5, 1.01, 40), (2.0, 3.0, 1.0, 0),
                                             (0.05, 1.9, 1.0, 1), (1e-4, 2.0, 1.001, 60)])
def test_recurrence_matches_closed_form(alpha, beta, s, m):
    prm = O.cheb_params(alpha, beta, s)
    x = np.concatenate([np.linspace(alpha, beta, 201), [0.5 * alpha, 1.05 * beta]])
    ref = p_closed(x, alpha, beta, s, m)
    got = O.p_k_recurrence(x, prm, m)
    assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-9
    got2 = O.p_k_closed_form(x, prm, m)
    assert np.max(np.abs(got2 - ref) / np.abs(ref)) < 1e-9


def test_rho_is_ratio_of_T():
    sigma = 1.37
    rho = O.rho_sequence(sigma, 30)
    k = np.arange(31)
    sig_k = T_closed(0, np.full(31, sigma)) * 0 + np.cosh(k * np.arccosh(sigma))
    sig_k1 = np.cosh((k + 1) * np.arccosh(sigma))
    assert np.allclose(rho, sig_k / sig_k1, rtol=1e-13)


@pytest.mark.parametrize("m", [0, 1, 2, 3, 8, 20, 40])
def test_cheb_apply_diagonal_matrix(m):
    rng = np.random.default_rng(5)
    lam = np.sort(rng.uniform(0.02, 1.8, 64))
    v = rng.uniform(-1, 1, 64)
    alpha, beta, s = lam[0], lam[-1], 1.001
    z = O.cheb_apply(lambda u: lam * u, v, O.cheb_params(alpha, beta, s), m)
    ref = p_closed(lam, alpha, beta, s, m) * v
    assert np.max(np.abs(z - ref)) <= 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("m", [3, 10])
def test_cheb_apply_laplacian_eigenvector(m):
    n = 50
    A = W.laplacian_1d(n)
    mv = O.csr_matvec(A.rowptr, A.col, A.val, n)
    j = np.arange(1, n + 1)
    lam_min, lam_max = 4 * np.sin(np.pi / (2 * (n + 1))) ** 2, 4 * np.sin(n * np.pi / (2 * (n + 1))) ** 2
    prm = O.cheb_params(lam_min, lam_max, 1.0)
    for i in (1, 7, 25, 50):
        v = np.sin(i * j * np.pi / (n + 1))
        lam_i = 4 * np.sin(i * np.pi / (2 * (n + 1))) ** 2
        z = O.cheb_apply(mv, v, prm, m)
        ref = p_closed(np.array([lam_i]), lam_min, lam_max, 1.0, m)[0] * v
        assert np.max(np.abs(z - ref)) <= 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("m", [1, 4, 8, 15])
def test_chebyshev_bound_on_laplacian(m):
    """Spectrum of P_m(A)A lies in 1 +- 1/T_{m+1}(sigma); the bottom end is attained."""
    n = 40
    A = W.laplacian_1d(n).to_scipy().toarray()
    lam_min, lam_max = 4 * np.sin(np.pi / (2 * (n + 1))) ** 2, 4 * np.sin(n * np.pi / (2 * (n + 1))) ** 2
    prm = O.cheb_params(lam_min, lam_max, 1.0)
    P = np.column_stack([O.cheb_apply(lambda u: A @ u, e, prm, m) for e in np.eye(n)])
    mu = np.linalg.eigvalsh(0.5 * (P @ A + (P @ A).T))
    eps = 1.0 / np.cosh((m + 1) * np.arccosh(prm.sigma))
    assert mu.min() >= 1 - eps - 1e-12 and mu.max() <= 1 + eps + 1e-12
    assert abs(mu.min() - (1 - eps)) < 1e-10


def test_m0_and_m1_forms():
    rng = np.random.default_rng(1)
    lam = rng.uniform(0.1, 2.0, 30)
    r = rng.uniform(-1, 1, 30)
    prm = O.cheb_params(0.1, 2.0, 1.0)
    z0 = O.cheb_apply(lambda u: lam * u, r, prm, 0)
    assert np.allclose(z0, r / 1.05, rtol=1e-15)
    # p_1(x) = c (2 - x/theta) with T_2(t) = 2 t^2 - 1 giving the coefficient
    z1 = O.cheb_apply(lambda u: lam * u, r, prm, 1)
    ref = p_closed(lam, 0.1, 2.0, 1.0, 1) * r
    assert np.allclose(z1, ref, rtol=1e-13)


def test_bad_interval_rejected():
    with pytest.raises(ValueError):
        O.cheb_params(1.0, 0.5)
    with pytest.raises(ValueError):
        O.cheb_params(0.0, 0.5)
