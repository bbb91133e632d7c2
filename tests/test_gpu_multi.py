"""Several right-hand sides sharing the matrix (pcg_solve_multi).

Each column is an independent PCG recurrence: against the oracle's solve of
that column (iterations +-1, error bounded by kappa * tol) and against the
single-right-hand-side solver (same iterations +-1, solutions to rounding:
the dot products are summed in another order).  Columns stop at different
iterations and are frozen meanwhile; a zero column returns x = 0.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
import workloads as W
from conftest import GOLDEN
from nchelpers import csr_to_gpu, need_gpu, rel_err, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    import paper_2008_01440_gb300 as nc
    return torch, nc


def diffusion(torch, nc, N, seed):
    A = W.diffusion_3d_7pt_lognormal(N, seed=seed)
    M = nc.nc_matrix_jacobi(csr_to_gpu(torch, nc, A))
    val, dis = O.jacobi_scale_csr(A.rowptr, A.col, A.val, A.n)
    mv = O.csr_matvec(A.rowptr, A.col, val, A.n)
    lo, hi, _, _ = nc.nc_bounds_lanczos(M, 20, to_dev(torch, W.uniform_vector(A.n, seed=3)))
    return A, M, mv, dis, lo, hi


def block(torch, cols):
    return to_dev(torch, np.stack(cols))


@pytest.mark.parametrize("m", [1, 3, 8])
def test_multi_matches_oracle_and_single(env, m):
    torch, nc = env
    A, M, mv, dis, lo, hi = diffusion(torch, nc, 24, 11)
    k = 12
    cols = [W.uniform_vector(A.n, seed=100 + c) for c in range(m)]
    S = nc.pcg_setup(M, lo, hi, k, 1.001)
    X = torch.zeros(m, A.n, dtype=torch.float64, device="cuda")
    res = nc.pcg_solve_multi(S, block(torch, cols), X, 1e-8, 2000)
    prm = O.cheb_params(lo, hi, 1.001)
    for c in range(m):
        ro = O.pcg(mv, dis * cols[c], lambda r: O.cheb_apply(mv, r, prm, k), m=k, tol=1e-8, maxit=2000)
        assert res[c]["status"] == 0 and abs(res[c]["iters"] - ro.iters) <= 1, (c, res[c]["iters"], ro.iters)
        assert res[c]["n_dot"] == 3 * res[c]["iters"] and res[c]["n_spmv"] == (k + 1) * res[c]["iters"]
        assert res[c]["true_relres"] <= 2e-8
        assert rel_err(X[c].cpu().numpy(), dis * ro.x) <= (hi / lo) * 1e-8
        x1 = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        r1 = nc.pcg_solve(S, to_dev(torch, cols[c]), x1, 1e-8, 2000)
        assert abs(r1["iters"] - res[c]["iters"]) <= 1
        assert rel_err(X[c].cpu().numpy(), x1.cpu().numpy()) <= (hi / lo) * 1e-8


def test_multi_columns_stop_independently(env):
    """Columns needing 0, few and many iterations in one block; the frozen
    ones keep their own results, and graph and host loop agree."""
    torch, nc = env
    A = W.laplacian_2d_5pt(64, 64)
    lo, hi = W.laplacian_2d_bounds(64, 64)
    M = csr_to_gpu(torch, nc, A)
    mv = O.csr_matvec(A.rowptr, A.col, A.val, A.n)
    v1 = np.sin(np.pi * (np.arange(A.n) % 64 + 1) / 65) * np.sin(np.pi * (np.arange(A.n) // 64 + 1) / 65)
    cols = [np.zeros(A.n), mv(v1), W.uniform_vector(A.n, seed=7), 1e6 * W.uniform_vector(A.n, seed=8)]
    out = []
    for graph in (True, False):
        S = nc.pcg_setup(M, lo, hi, 8, 1.001, use_graph=graph)
        X = torch.zeros(len(cols), A.n, dtype=torch.float64, device="cuda")
        res = nc.pcg_solve_multi(S, block(torch, cols), X, 1e-8, 1000)
        out.append((res, X.clone()))
    (ra, Xa), (rb, Xb) = out
    assert ra == rb and torch.equal(Xa, Xb)
    assert ra[0]["iters"] == 0 and not torch.any(Xa[0])
    assert ra[1]["iters"] < ra[2]["iters"]          # an eigenvector converges at once
    prm = O.cheb_params(lo, hi, 1.001)
    for c in (1, 2, 3):
        ro = O.pcg(mv, cols[c], lambda r: O.cheb_apply(mv, r, prm, 8), m=8, tol=1e-8, maxit=1000)
        assert ra[c]["status"] == 0 and abs(ra[c]["iters"] - ro.iters) <= 1


@pytest.mark.parametrize("dt", ["f32", "bf16"])
def test_multi_mixed_precision(env, dt):
    torch, nc = env
    A, M, mv, dis, lo, hi = diffusion(torch, nc, 24, 5)
    cols = [W.uniform_vector(A.n, seed=200 + c) for c in range(4)]
    S = nc.pcg_setup(M, lo, hi, 10, 1.001, apply_dtype=dt)
    X = torch.zeros(4, A.n, dtype=torch.float64, device="cuda")
    res = nc.pcg_solve_multi(S, block(torch, cols), X, 1e-8, 2000)
    prm = O.cheb_params(lo, hi, 1.001)
    for c in range(4):
        ro = O.pcg(mv, dis * cols[c], lambda r: O.cheb_apply(mv, r, prm, 10), m=10, tol=1e-8, maxit=2000)
        assert res[c]["status"] == 0 and res[c]["true_relres"] <= 1e-7
        assert abs(res[c]["iters"] - ro.iters) <= max(2, int(0.1 * ro.iters))
        x1 = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        r1 = nc.pcg_solve(S, to_dev(torch, cols[c]), x1, 1e-8, 2000)
        assert abs(r1["iters"] - res[c]["iters"]) <= 1


def test_multi_fullsize_golden(env):
    """The 128^3 workload with four right-hand sides, the first being the
    one of the golden record: its iteration count within +-1."""
    torch, nc = env
    with open(os.path.join(GOLDEN, "c2_oracle.json")) as f:
        g = json.load(f)
    A = W.diffusion_3d_7pt_lognormal(128, seed=g["seed_matrix"])
    M = nc.nc_matrix_jacobi(csr_to_gpu(torch, nc, A))
    S = nc.pcg_setup(M, g["lmin"], g["lmax"], 20, g["theta_scale"], x0_is_zero=True)
    cols = [W.uniform_vector(A.n, seed=g["seed_rhs"])] + [W.uniform_vector(A.n, seed=300 + c) for c in range(3)]
    X = torch.zeros(4, A.n, dtype=torch.float64, device="cuda")
    res = nc.pcg_solve_multi(S, block(torch, cols), X, g["tol"], 5000)
    assert all(r["status"] == 0 and r["true_relres"] <= 2 * g["tol"] for r in res)
    assert abs(res[0]["iters"] - g["solves"]["20"]["iters"]) <= 1


def test_multi_argument_checks(env):
    torch, nc = env
    A = W.laplacian_2d_5pt(16, 16)
    lo, hi = W.laplacian_2d_bounds(16, 16)
    M = csr_to_gpu(torch, nc, A)
    B = torch.ones(2, A.n, dtype=torch.float64, device="cuda")
    X = torch.zeros_like(B)
    for opts in (dict(spmv_format="csr"), dict(rr_period=5), dict(poly="newton")):
        S = nc.pcg_setup(M, lo, hi, 7, 1.0, **opts)
        with pytest.raises(nc.NcError) as ei:
            nc.pcg_solve_multi(S, B, X, 1e-8, 100)
        assert ei.value.status == nc.NC_ERR_UNSUPPORTED
    S = nc.pcg_setup(M, lo, hi, 7, 1.0)
    B9 = torch.ones(9, A.n, dtype=torch.float64, device="cuda")
    with pytest.raises(nc.NcError) as ei:
        nc.pcg_solve_multi(S, B9, torch.zeros_like(B9), 1e-8, 100)
    assert ei.value.status == nc.NC_ERR_ARG
