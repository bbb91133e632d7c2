"""Full-size parity on the elasticity workload (Q1 hexahedra, 100^3 nodes x 3
dofs, n = 3,000,000, 3x3 blocks), in the configuration bench.py times.

The oracle's Lanczos bounds and its iteration counts for the configuration's
degrees k = 20 and 60 were written by tests/golden/make_c3_golden.py, which
calls only the oracle (about half an hour of CPU per degree); P_k(A)v is
recomputed here by the oracle on the full system (k block products, seconds).
"""
import json
import os

import numpy as np
import pytest

import oracle as O
import workloads as W
from conftest import GOLDEN
from nchelpers import elem_err, need_gpu, rel_err, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def system():
    torch = need_gpu()
    import paper_2008_01440_gb300 as nc
    with open(os.path.join(GOLDEN, "c3_oracle.json")) as f:
        g = json.load(f)
    A, b = W.elasticity_q1_bsr3(100, seed=g["seed_matrix"])
    assert A.n == g["n"] and A.nnzb == g["nnzb"]
    M0 = nc.nc_matrix_bsr3(to_dev(torch, A.browptr), to_dev(torch, A.bcol), to_dev(torch, A.val.reshape(-1)))
    M = nc.nc_matrix_jacobi(M0)
    return torch, nc, g, A, b, M


def test_c3_lanczos_bounds(system):
    torch, nc, g, A, b, M = system
    lo, hi, rmin, rmax = nc.nc_bounds_lanczos(M, 20, to_dev(torch, W.uniform_vector(A.n, seed=g["seed_v0"])))
    assert abs(lo - g["lmin"]) <= 1e-9 * g["lmin"]
    assert abs(hi - g["lmax"]) <= 1e-9 * g["lmax"]
    assert abs(rmax - g["ritz_max"]) <= 1e-9 * g["ritz_max"]


@pytest.mark.parametrize("k", [20, 60])
def test_c3_apply_parity(system, k):
    """z = P_k(A) v on the full Jacobi-scaled system, both block layouts."""
    torch, nc, g, A, b, M = system
    val, dis = O.jacobi_scale_bsr3(A.browptr, A.bcol, A.val, A.nb)
    mv = O.bsr3_matvec(A.browptr, A.bcol, val, A.nb)
    v = W.uniform_vector(A.n, seed=21)
    ref = O.cheb_apply(mv, v, O.cheb_params(g["lmin"], g["lmax"], g["theta_scale"]), k)
    for fmt in ("sell", "csr"):
        S = nc.pcg_setup(M, g["lmin"], g["lmax"], k, g["theta_scale"], spmv_format=fmt)
        z = torch.empty(A.n, dtype=torch.float64, device="cuda")
        nc.pcg_apply_poly(S, to_dev(torch, v), z)
        got = z.cpu().numpy()
        assert rel_err(got, ref) <= 1e-12 and elem_err(got, ref) <= 1e-12, fmt
        S.close()


@pytest.mark.parametrize("k", [20, 60])
def test_c3_solve_iterations(system, k):
    """float64 PCG with P_k: the oracle's iteration count within +-1."""
    torch, nc, g, A, b, M = system
    S = nc.pcg_setup(M, g["lmin"], g["lmax"], k, g["theta_scale"], x0_is_zero=True)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    res = nc.pcg_solve(S, to_dev(torch, b), x, g["tol"], 5000)
    ref = g["solves"][str(k)]
    assert res["status"] == 0
    assert abs(res["iters"] - ref["iters"]) <= 1, (res["iters"], ref["iters"])
    assert res["relres"] <= g["tol"] and res["true_relres"] <= 2 * g["tol"]
    assert res["n_spmv"] == (k + 1) * res["iters"] and res["n_dot"] == 3 * res["iters"]


@pytest.mark.parametrize("k", [20, 60])
def test_c3_mixed_precision_with_residual_replacement(system, k):
    """float32 P_k, float64 outer CG, r = b - A x in float64 every 50
    iterations (the benchmarked mixed configuration): reaches the tolerance
    by the true residual, within 10% of the oracle's iteration count."""
    torch, nc, g, A, b, M = system
    S = nc.pcg_setup(M, g["lmin"], g["lmax"], k, g["theta_scale"], apply_dtype="f32", rr_period=50,
                     x0_is_zero=True)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    res = nc.pcg_solve(S, to_dev(torch, b), x, g["tol"], 5000)
    ref = g["solves"][str(k)]["iters"]
    assert res["status"] == 0 and res["true_relres"] <= 2 * g["tol"]
    assert abs(res["iters"] - ref) <= max(2, int(0.1 * ref)), (res["iters"], ref)
    assert res["n_replace"] == (res["iters"] - 1) // 50
