"""Lap1600 (Sec. 5.1, Table 4) at a reduced grid: the 5-point Laplacian on
N^2 interior points of the unit square, Jacobi scaled, x* = ones, b = A x*,
x0 = 0, exact bounds of the scaled operator, s = 1.001, tol 1e-8, degrees
m = 2^nlev - 1 = 0 ... 63.  The GPU's iteration counts must equal the
oracle's within +-1 for every degree, in the Chebyshev form and in the
Newton form (the same polynomial, Theorem 3.1), its operation counts must be
Table 4's (A x v = (m+1) iter, ddot = 3 iter), and the trend of Table 4 must
hold: iterations fall with m while the products stay within a band."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from nchelpers import csr_to_gpu, need_gpu, rel_err, to_dev

pytestmark = pytest.mark.gpu

N = 200
DEGREES = (0, 1, 3, 7, 15, 31, 63)


@pytest.fixture(scope="module")
def system():
    torch = need_gpu()
    import paper_2008_01440_gb300 as nc
    A = W.laplacian_2d_5pt(N, N)
    M0 = csr_to_gpu(torch, nc, A)
    M = nc.nc_matrix_jacobi(M0)
    lo, hi = (v / 4.0 for v in W.laplacian_2d_bounds(N, N))
    ones = torch.ones(A.n, dtype=torch.float64, device="cuda")
    b = torch.empty(A.n, dtype=torch.float64, device="cuda")
    nc.nc_matvec(M0, ones, b)
    # the oracle on the same problem
    val, dis = O.jacobi_scale_csr(A.rowptr, A.col, A.val, A.n)
    mv = O.csr_matvec(A.rowptr, A.col, val, A.n)
    bo = dis * O.csr_matvec(A.rowptr, A.col, A.val, A.n)(np.ones(A.n))
    prm = O.cheb_params(lo, hi, 1.001)
    oracle = {m: O.pcg(mv, bo, lambda r, m=m: O.cheb_apply(mv, r, prm, m), m=m, tol=1e-8, maxit=20000)
              for m in DEGREES}
    return torch, nc, A, M, lo, hi, b, oracle, dis


@pytest.mark.parametrize("m", DEGREES)
@pytest.mark.parametrize("form", ["chebyshev", "newton"])
def test_lap_iterations_match_oracle(system, m, form):
    torch, nc, A, M, lo, hi, b, oracle, dis = system
    if form == "newton" and m == 0:
        pytest.skip("the Newton form of degree 0 is the Chebyshev one (P = zeta_0 I)")
    S = nc.pcg_setup(M, lo, hi, m, 1.001, x0_is_zero=True, poly=form)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    r = nc.pcg_solve(S, b, x, 1e-8, 20000)
    ro = oracle[m]
    assert r["status"] == 0 and ro.status == 0
    assert abs(r["iters"] - ro.iters) <= 1, (r["iters"], ro.iters)
    assert r["n_spmv"] == (m + 1) * r["iters"] and r["n_dot"] == 3 * r["iters"]
    xh = x.cpu().numpy()
    assert rel_err(xh, np.ones(A.n)) <= 1e-4
    assert rel_err(xh, dis * ro.x) <= (hi / lo) * 1e-8


def test_lap_trend_of_table4(system):
    """Iterations fall strictly with m; the products (m+1) iter stay within
    a factor 2 of each other from m = 1 on (Table 4: 3536 ... 4416)."""
    torch, nc, A, M, lo, hi, b, oracle, dis = system
    its, prods = [], []
    for m in DEGREES:
        S = nc.pcg_setup(M, lo, hi, m, 1.001, x0_is_zero=True)
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        r = nc.pcg_solve(S, b, x, 1e-8, 20000)
        its.append(r["iters"])
        prods.append(r["n_spmv"])
    assert all(a > b_ for a, b_ in zip(its, its[1:])), its
    assert max(prods[1:]) <= 2 * min(prods[1:]), prods
