"""The one-cluster whole-solve kernel (nc_options.use_graph = 2) against the
float64 oracle and against the graph path.

Same bars as the graph path: PCG iteration count within +-1 of the oracle,
relative residual 1e-8, solution error bounded by kappa * tol.  The
persistent kernel sums its dot products in another order than the graph's
kernels, so the two paths agree to rounding, not bitwise; a repeated
persistent solve is bitwise identical (fixed reduction order).
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from nchelpers import csr_to_gpu, need_gpu, rel_err, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    import paper_2008_01440_gb300 as nc
    return torch, nc


def lap(nx, ny):
    return W.laplacian_2d_5pt(nx, ny), *W.laplacian_2d_bounds(nx, ny)


def oracle_solve(A, lo, hi, k, s, b, tol, maxit, x0=None, jacobi=False):
    if jacobi:
        val, dis = O.jacobi_scale_csr(A.rowptr, A.col, A.val, A.n)
    else:
        val, dis = A.val, np.ones(A.n)
    mv = O.csr_matvec(A.rowptr, A.col, val, A.n)
    prm = O.cheb_params(lo, hi, s)
    x0s = None if x0 is None else x0 / dis
    ro = O.pcg(mv, dis * b, lambda r: O.cheb_apply(mv, r, prm, k), m=k, x0=x0s, tol=tol, maxit=maxit)
    return ro, dis * ro.x


def persistent_solver(torch, nc, M, lo, hi, k, s, **opts):
    S = nc.pcg_setup(M, lo, hi, k, s, persistent=True, **opts)
    assert nc.pcg_get_info(S)["persistent"]
    return S


@pytest.mark.parametrize("k,s", [(0, 1.0), (1, 1.0), (2, 1.001), (8, 1.0), (8, 1.001), (15, 1.01), (31, 1.001)])
def test_persistent_laplacian64_matches_oracle(env, k, s):
    torch, nc = env
    A, lo, hi = lap(64, 64)
    b = W.rhs_from_solution(A, W.uniform_vector(A.n, seed=1))
    S = persistent_solver(torch, nc, csr_to_gpu(torch, nc, A), lo, hi, k, s)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    res = nc.pcg_solve(S, to_dev(torch, b), x, 1e-8, 5000)
    ro, xo = oracle_solve(A, lo, hi, k, s, b, 1e-8, 5000)
    assert res["status"] == 0 and ro.status == 0
    assert abs(res["iters"] - ro.iters) <= 1, (res["iters"], ro.iters)
    assert res["relres"] <= 1e-8 and res["true_relres"] <= 2e-8
    assert res["n_dot"] == 3 * res["iters"]
    assert res["n_spmv"] == (k + 1) * res["iters"]
    assert rel_err(x.cpu().numpy(), xo) <= (hi / lo) * 1e-8


@pytest.mark.parametrize("N,k", [(24, 10), (27, 20)])
def test_persistent_diffusion_jacobi(env, N, k):
    """Log-normal 3D diffusion, Jacobi scaled, 20-step Lanczos bounds: 16
    CTAs of 864 / 1248 rows, several rows per thread, n not a multiple of the
    32-row slice for N = 27."""
    torch, nc = env
    A = W.diffusion_3d_7pt_lognormal(N, seed=N)
    M = nc.nc_matrix_jacobi(csr_to_gpu(torch, nc, A))
    lo, hi, _, _ = nc.nc_bounds_lanczos(M, 20, to_dev(torch, W.uniform_vector(A.n, seed=99)))
    b = W.uniform_vector(A.n, seed=5)
    S = persistent_solver(torch, nc, M, lo, hi, k, 1.001)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    res = nc.pcg_solve(S, to_dev(torch, b), x, 1e-8, 5000)
    ro, xo = oracle_solve(A, lo, hi, k, 1.001, b, 1e-8, 5000, jacobi=True)
    assert res["status"] == 0 and ro.status == 0
    assert abs(res["iters"] - ro.iters) <= 1, (res["iters"], ro.iters)
    assert res["true_relres"] <= 1e-7
    assert rel_err(x.cpu().numpy(), xo) <= (hi / lo) * 1e-8


def test_persistent_largest_2d_and_fallback(env):
    """140^2 = 19600 rows fit one cluster (about 5 rows per thread); 420^2
    does not and keeps the graph path, with the same answer quality."""
    torch, nc = env
    for side, fits in ((140, True), (420, False)):
        A, lo, hi = lap(side, side)
        b = W.uniform_vector(A.n, seed=2)
        S = nc.pcg_setup(csr_to_gpu(torch, nc, A), lo, hi, 40, 1.001, persistent=True)
        assert nc.pcg_get_info(S)["persistent"] == fits
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        res = nc.pcg_solve(S, to_dev(torch, b), x, 1e-6, 2000)
        ro, xo = oracle_solve(A, lo, hi, 40, 1.001, b, 1e-6, 2000)
        assert res["status"] == 0 and ro.status == 0
        assert abs(res["iters"] - ro.iters) <= 1, (res["iters"], ro.iters)
        assert rel_err(x.cpu().numpy(), xo) <= (hi / lo) * 1e-6


def test_persistent_matches_graph_and_is_deterministic(env):
    torch, nc = env
    A, lo, hi = lap(64, 64)
    M = csr_to_gpu(torch, nc, A)
    b = to_dev(torch, W.uniform_vector(A.n, seed=3))
    Sg = nc.pcg_setup(M, lo, hi, 8, 1.001)
    assert not nc.pcg_get_info(Sg)["persistent"]
    xg = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    rg = nc.pcg_solve(Sg, b, xg, 1e-10, 1000)
    Sp = persistent_solver(torch, nc, M, lo, hi, 8, 1.001)
    xp = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    rp = nc.pcg_solve(Sp, b, xp, 1e-10, 1000)
    assert rg["status"] == rp["status"] == 0
    assert abs(rg["iters"] - rp["iters"]) <= 1
    assert rel_err(xp.cpu().numpy(), xg.cpu().numpy()) <= 1e-8
    xp2 = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    rp2 = nc.pcg_solve(Sp, b, xp2, 1e-10, 1000)
    assert rp2 == rp and torch.equal(xp2, xp)


def test_persistent_nonzero_initial_guess_and_host_buffers(env):
    torch, nc = env
    A, lo, hi = lap(64, 64)
    xs = W.uniform_vector(A.n, seed=1)
    b = W.rhs_from_solution(A, xs)
    x0 = 0.5 * W.uniform_vector(A.n, seed=6)
    S = persistent_solver(torch, nc, csr_to_gpu(torch, nc, A), lo, hi, 8, 1.001)
    x = to_dev(torch, x0)
    res = nc.pcg_solve(S, to_dev(torch, b), x, 1e-8, 1000)
    ro, xo = oracle_solve(A, lo, hi, 8, 1.001, b, 1e-8, 1000, x0=x0)
    assert res["status"] == 0 and abs(res["iters"] - ro.iters) <= 1
    assert rel_err(x.cpu().numpy(), xs) <= (hi / lo) * 1e-8
    xh = x0.copy()
    rh = nc.pcg_solve_host(S, b, xh, 1e-8, 1000)
    assert rh == res and np.array_equal(xh, x.cpu().numpy())


def test_persistent_edge_cases(env):
    torch, nc = env
    A, lo, hi = lap(64, 64)
    S = persistent_solver(torch, nc, csr_to_gpu(torch, nc, A), lo, hi, 8, 1.001)
    x = torch.ones(A.n, dtype=torch.float64, device="cuda")
    # zero right-hand side with x0 = 0: converged at once, x stays 0
    S0 = persistent_solver(torch, nc, csr_to_gpu(torch, nc, A), lo, hi, 8, 1.001, x0_is_zero=True)
    r0 = nc.pcg_solve(S0, torch.zeros(A.n, dtype=torch.float64, device="cuda"), x, 1e-8, 100)
    assert r0["status"] == 0 and r0["iters"] == 0 and not torch.any(x)
    # iteration limit: status MAXIT after exactly maxit iterations, k+1 products each
    b = to_dev(torch, W.uniform_vector(A.n, seed=4))
    x.zero_()
    r3 = nc.pcg_solve(S, b, x, 1e-14, 3)
    assert r3["status"] == nc.NC_ERR_MAXIT and r3["iters"] == 3 and r3["n_spmv"] == 9 * 3
    # maxit = 0: no iteration
    r4 = nc.pcg_solve(S, b, x, 1e-14, 0)
    assert r4["status"] == nc.NC_ERR_MAXIT and r4["iters"] == 0
    # non-finite right-hand side: breakdown reported, no hang
    bn = b.clone()
    bn[17] = float("nan")
    x.zero_()
    rn = nc.pcg_solve(S, bn, x, 1e-8, 100)
    assert rn["status"] == nc.NC_ERR_BREAKDOWN


@pytest.mark.parametrize("n", [1, 2, 31, 129])
def test_persistent_tiny(env, n):
    torch, nc = env
    A = W.laplacian_1d(n)
    lo = 4 * np.sin(np.pi / (2 * (n + 1))) ** 2
    hi = max(4 * np.sin(n * np.pi / (2 * (n + 1))) ** 2, 1.5 * lo)
    b = W.uniform_vector(n, seed=n)
    # SELL forced: AUTO keeps CSR where 32-row slices are mostly padding
    S = persistent_solver(torch, nc, csr_to_gpu(torch, nc, A), lo, hi, 4, 1.001, spmv_format="sell")
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    res = nc.pcg_solve(S, to_dev(torch, b), x, 1e-10, 500)
    ro, xo = oracle_solve(A, lo, hi, 4, 1.001, b, 1e-10, 500)
    assert res["status"] == 0 and abs(res["iters"] - ro.iters) <= 1
    assert rel_err(x.cpu().numpy(), xo) <= 1e-7


def test_persistent_falls_back_where_unsupported(env):
    """Mixed precision, residual replacement or the plain CSR layout keep the
    graph path; the result is that path's."""
    torch, nc = env
    A, lo, hi = lap(64, 64)
    M = csr_to_gpu(torch, nc, A)
    b = to_dev(torch, W.uniform_vector(A.n, seed=5))
    for opts in (dict(apply_dtype="f32", rr_period=20), dict(spmv_format="csr"), dict(rr_period=10)):
        S = nc.pcg_setup(M, lo, hi, 8, 1.001, persistent=True, **opts)
        assert not nc.pcg_get_info(S)["persistent"]
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        res = nc.pcg_solve(S, b, x, 1e-8, 1000)
        assert res["status"] == 0 and res["true_relres"] <= 1e-7
