"""GPU parity of the 3x3-block path (plain block CSR and BSELL-32) against the
oracle on the Q1-hex elasticity workload at reduced sizes."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from nchelpers import elem_err, need_gpu, rel_err, to_dev

pytestmark = pytest.mark.gpu

FORMATS = ["csr", "sell"]


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    import paper_2008_01440_gb300 as nc
    return torch, nc


def upload(torch, nc, A):
    return nc.nc_matrix_bsr3(to_dev(torch, A.browptr), to_dev(torch, A.bcol), to_dev(torch, A.val.reshape(-1)))


def scaled_oracle(A):
    val, dis = O.jacobi_scale_bsr3(A.browptr, A.bcol, A.val, A.nb)
    mv = O.bsr3_matvec(A.browptr, A.bcol, val, A.nb)
    brows = np.repeat(np.arange(A.nb), np.diff(A.browptr))
    rs = np.zeros(A.n)
    np.add.at(rs, (3 * brows[:, None] + np.arange(3)[None, :]).ravel(), np.abs(val).sum(axis=2).ravel())
    return mv, dis, float(rs.max())


@pytest.mark.parametrize("N", [3, 7, 12])
def test_bsr3_matvec_and_jacobi(env, N):
    torch, nc = env
    A, _ = W.elasticity_q1_bsr3(N, seed=N)
    M = upload(torch, nc, A)
    x = W.uniform_vector(A.n, seed=1)
    y = torch.empty(A.n, dtype=torch.float64, device="cuda")
    nc.nc_matvec(M, to_dev(torch, x), y)
    ref = O.bsr3_matvec(A.browptr, A.bcol, A.val, A.nb)(x)
    assert elem_err(y.cpu().numpy(), ref) <= 1e-13
    Ms = nc.nc_matrix_jacobi(M)
    nc.nc_matvec(Ms, to_dev(torch, x), y)
    mv, dis, g = scaled_oracle(A)
    assert elem_err(y.cpu().numpy(), mv(x)) <= 1e-13
    assert abs(nc.nc_gershgorin(Ms) - g) <= 1e-13 * g


@pytest.mark.parametrize("fmt", FORMATS)
@pytest.mark.parametrize("N,k", [(5, 1), (9, 8), (14, 20), (14, 60)])
def test_bsr3_apply_parity(env, N, k, fmt):
    torch, nc = env
    A, _ = W.elasticity_q1_bsr3(N, seed=2)
    M = nc.nc_matrix_jacobi(upload(torch, nc, A))
    mv, dis, g = scaled_oracle(A)
    v0 = W.uniform_vector(A.n, seed=3)
    lo, hi, _, _ = nc.nc_bounds_lanczos(M, 20, to_dev(torch, v0))
    lo_o, hi_o, _ = O.lanczos_bounds(mv, v0, 20, gershgorin=g)
    assert abs(lo - lo_o) <= 1e-8 * lo_o and abs(hi - hi_o) <= 1e-9 * hi_o
    S = nc.pcg_setup(M, lo, hi, k, 1.001, spmv_format=fmt)
    info = nc.pcg_get_info(S)
    assert info["spmv_format"] == fmt
    v = W.uniform_vector(A.n, seed=4)
    z = torch.empty(A.n, dtype=torch.float64, device="cuda")
    nc.pcg_apply_poly(S, to_dev(torch, v), z)
    ref = O.cheb_apply(mv, v, O.cheb_params(lo, hi, 1.001), k)
    got = z.cpu().numpy()
    assert rel_err(got, ref) <= 1e-12 and elem_err(got, ref) <= 1e-12


@pytest.mark.parametrize("fmt", FORMATS)
@pytest.mark.parametrize("k", [20, 60])
def test_bsr3_solve_parity(env, k, fmt):
    """Elasticity 16^3 nodes, Jacobi scaled, 20-step Lanczos bounds, s = 1.001:
    iterations within +-1 of the oracle."""
    torch, nc = env
    A, b = W.elasticity_q1_bsr3(16, seed=5)
    M = nc.nc_matrix_jacobi(upload(torch, nc, A))
    mv, dis, g = scaled_oracle(A)
    lo, hi, _ = O.lanczos_bounds(mv, W.uniform_vector(A.n, seed=3), 20, gershgorin=g)
    S = nc.pcg_setup(M, lo, hi, k, 1.001, spmv_format=fmt)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    res = nc.pcg_solve(S, to_dev(torch, b), x, 1e-8, 5000)
    ro = O.pcg(mv, dis * b, lambda r: O.cheb_apply(mv, r, O.cheb_params(lo, hi, 1.001), k), m=k, tol=1e-8,
               maxit=5000)
    assert res["status"] == 0 and ro.status == 0
    assert abs(res["iters"] - ro.iters) <= 1, (res["iters"], ro.iters)
    assert res["true_relres"] <= 2e-8


@pytest.mark.parametrize("dt", ["f32", "bf16"])
def test_bsr3_mixed_precision_with_replacement(env, dt):
    """FP32 / BF16 apply with FP64 residual replacement every 50 iterations
    (the elasticity configuration): converges to 1e-8, iterations close to
    the FP64 oracle's."""
    torch, nc = env
    A, b = W.elasticity_q1_bsr3(16, seed=5)
    M = nc.nc_matrix_jacobi(upload(torch, nc, A))
    mv, dis, g = scaled_oracle(A)
    lo, hi, _ = O.lanczos_bounds(mv, W.uniform_vector(A.n, seed=3), 20, gershgorin=g)
    S = nc.pcg_setup(M, lo, hi, 20, 1.001, apply_dtype=dt, rr_period=50)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    res = nc.pcg_solve(S, to_dev(torch, b), x, 1e-8, 5000)
    ro = O.pcg(mv, dis * b, lambda r: O.cheb_apply(mv, r, O.cheb_params(lo, hi, 1.001), 20), m=20, tol=1e-8)
    assert res["status"] == 0 and res["true_relres"] <= 2e-8
    assert abs(res["iters"] - ro.iters) <= max(3, 0.15 * ro.iters)
