"""Full-size parity on the 128^3 workload, in the configuration bench.py times.

The oracle's results for this system (Lanczos bounds, iteration counts for
k = 10, 20, 40) were written by tests/golden/make_c2_golden.py, which calls
only the oracle; P_k(A)v is recomputed here by the oracle on the full system
(about 20-40 scipy products, seconds).
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
    with open(os.path.join(GOLDEN, "c2_oracle.json")) as f:
        g = json.load(f)
    A = W.diffusion_3d_7pt_lognormal(128, seed=g["seed_matrix"])
    M0 = nc.nc_matrix_csr(to_dev(torch, A.rowptr), to_dev(torch, A.col), to_dev(torch, A.val))
    M = nc.nc_matrix_jacobi(M0)
    return torch, nc, g, A, M0, M


def test_fullsize_lanczos_bounds(system):
    torch, nc, g, A, M0, M = system
    lo, hi, rmin, rmax = nc.nc_bounds_lanczos(M, 20, to_dev(torch, W.uniform_vector(A.n, seed=g["seed_v0"])))
    assert abs(lo - g["lmin"]) <= 1e-9 * g["lmin"]
    assert abs(hi - g["lmax"]) <= 1e-9 * g["lmax"]


@pytest.mark.parametrize("k", [10, 20, 40])
def test_fullsize_solve_iterations(system, k):
    torch, nc, g, A, M0, M = system
    S = nc.pcg_setup(M, g["lmin"], g["lmax"], k, g["theta_scale"], x0_is_zero=True)
    assert nc.pcg_get_info(S)["spmv_format"] == "psell"
    b = to_dev(torch, W.uniform_vector(A.n, seed=g["seed_rhs"]))
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    res = nc.pcg_solve(S, b, x, g["tol"], 5000)
    ref = g["solves"][str(k)]
    assert res["status"] == 0
    assert abs(res["iters"] - ref["iters"]) <= 1, (res["iters"], ref["iters"])
    assert res["relres"] <= g["tol"] and res["true_relres"] <= 2 * g["tol"]


def test_fullsize_apply_parity(system):
    torch, nc, g, A, M0, M = system
    k = 20
    val, dis = O.jacobi_scale_csr(A.rowptr, A.col, A.val, A.n)
    mv = O.csr_matvec(A.rowptr, A.col, val, A.n)
    v = W.uniform_vector(A.n, seed=21)
    ref = O.cheb_apply(mv, v, O.cheb_params(g["lmin"], g["lmax"], g["theta_scale"]), k)
    for fmt in ("psell", "sell", "csr"):
        S = nc.pcg_setup(M, g["lmin"], g["lmax"], k, g["theta_scale"], spmv_format=fmt)
        assert nc.pcg_get_info(S)["spmv_format"] == fmt
        z = torch.empty(A.n, dtype=torch.float64, device="cuda")
        nc.pcg_apply_poly(S, to_dev(torch, v), z)
        got = z.cpu().numpy()
        assert rel_err(got, ref) <= 1e-12 and elem_err(got, ref) <= 1e-12, fmt


@pytest.mark.parametrize("dt", ["f32", "bf16"])
def test_fullsize_mixed_precision_reaches_tol(system, dt):
    """Reduced-precision P_k with a float64 outer CG still reaches 1e-8 on the
    full system; its iteration count stays within 10% of the FP64 oracle's."""
    torch, nc, g, A, M0, M = system
    k = 20
    S = nc.pcg_setup(M, g["lmin"], g["lmax"], k, g["theta_scale"], apply_dtype=dt, x0_is_zero=True)
    b = to_dev(torch, W.uniform_vector(A.n, seed=g["seed_rhs"]))
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    res = nc.pcg_solve(S, b, x, g["tol"], 5000)
    ref = g["solves"][str(k)]["iters"]
    assert res["status"] == 0 and res["true_relres"] <= 2 * g["tol"]
    assert abs(res["iters"] - ref) <= max(2, 0.1 * ref)
