"""The two-level variant (Sec. 6, conclusions) with a block-Jacobi first
level on the elasticity operator: the scaled operator W^T A W (through its
products) against the oracle's, Lanczos bounds, PCG iteration counts and the
solution of the original system against the oracle, a nonzero initial guess,
and the non-SPD diagonal block refused."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from nchelpers import elem_err, need_gpu, rel_err, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    import paper_2008_01440_gb300 as nc
    return torch, nc


def handles(torch, nc, A):
    M0 = nc.nc_matrix_bsr3(to_dev(torch, A.browptr), to_dev(torch, A.bcol), to_dev(torch, A.val.reshape(-1)))
    return M0, nc.nc_matrix_block_jacobi(M0)


def oracle_two_level(A):
    val, Wb, Lb = O.block_jacobi_factor_bsr3(A.browptr, A.bcol, A.val, A.nb)
    return O.bsr3_matvec(A.browptr, A.bcol, val, A.nb), Wb, Lb


def test_scaled_operator_parity(env):
    torch, nc = env
    A, _ = W.elasticity_q1_bsr3(8, seed=5)
    M0, Mb = handles(torch, nc, A)
    mv, _, _ = oracle_two_level(A)
    v = W.uniform_vector(A.n, seed=1)
    y = torch.empty(A.n, dtype=torch.float64, device="cuda")
    nc.nc_matvec(Mb, to_dev(torch, v), y)
    ref = mv(v)
    assert elem_err(y.cpu().numpy(), ref) <= 1e-13


@pytest.mark.parametrize("fmt", ["sell", "csr"])
def test_two_level_solve_matches_oracle(env, fmt):
    torch, nc = env
    A, b = W.elasticity_q1_bsr3(12, seed=7)
    M0, Mb = handles(torch, nc, A)
    mv, Wb, Lb = oracle_two_level(A)
    v0 = W.uniform_vector(A.n, seed=3)
    lo, hi, _, _ = nc.nc_bounds_lanczos(Mb, 20, to_dev(torch, v0))
    val, _, _ = O.block_jacobi_factor_bsr3(A.browptr, A.bcol, A.val, A.nb)
    brows = np.repeat(np.arange(A.nb), np.diff(A.browptr))
    rs = np.zeros(A.n)
    np.add.at(rs, (3 * brows[:, None] + np.arange(3)[None, :]).ravel(), np.abs(val).sum(axis=2).ravel())
    lo_o, hi_o, _ = O.lanczos_bounds(mv, v0, 20, gershgorin=float(rs.max()))
    assert abs(lo - lo_o) <= 1e-9 * lo_o and abs(hi - hi_o) <= 1e-9 * hi_o
    k = 20
    S = nc.pcg_setup(Mb, lo, hi, k, 1.001, spmv_format=fmt)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    res = nc.pcg_solve(S, to_dev(torch, b), x, 1e-8, 2000)
    bs = np.einsum("bki,bk->bi", Wb, b.reshape(-1, 3)).ravel()              # W^T b
    ro = O.pcg(mv, bs, lambda r: O.cheb_apply(mv, r, O.cheb_params(lo_o, hi_o, 1.001), k), m=k, tol=1e-8,
               maxit=2000)
    xo = np.einsum("bij,bj->bi", Wb, ro.x.reshape(-1, 3)).ravel()           # x = W y
    assert res["status"] == 0 and ro.status == 0
    assert abs(res["iters"] - ro.iters) <= 1, (res["iters"], ro.iters)
    assert res["true_relres"] <= 2e-8
    assert rel_err(x.cpu().numpy(), xo) <= (hi / lo) * 1e-8
    # the original system: A x = b
    Ao = O.bsr3_matvec(A.browptr, A.bcol, A.val, A.nb)
    assert np.linalg.norm(Ao(x.cpu().numpy()) - b) <= 1e-6 * np.linalg.norm(b)


def test_two_level_initial_guess_and_host_buffers(env):
    torch, nc = env
    A, b = W.elasticity_q1_bsr3(8, seed=9)
    M0, Mb = handles(torch, nc, A)
    lo, hi, _, _ = nc.nc_bounds_lanczos(Mb, 20, to_dev(torch, W.uniform_vector(A.n, seed=3)))
    S = nc.pcg_setup(Mb, lo, hi, 10, 1.001)
    xs = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    nc.pcg_solve(S, to_dev(torch, b), xs, 1e-12, 2000)
    # start from a perturbed solution: fewer iterations, same answer
    x0 = xs.cpu().numpy() + 1e-6 * W.uniform_vector(A.n, seed=4)
    xg = to_dev(torch, x0)
    r0 = nc.pcg_solve(S, to_dev(torch, b), xg, 1e-12, 2000)
    assert r0["status"] == 0
    assert rel_err(xg.cpu().numpy(), xs.cpu().numpy()) <= 1e-8
    xh = x0.copy()
    rh = nc.pcg_solve_host(S, b, xh, 1e-12, 2000)
    assert rh == r0 and np.array_equal(xh, xg.cpu().numpy())


def test_two_level_rejects_bad_input(env):
    torch, nc = env
    A, _ = W.elasticity_q1_bsr3(4, seed=2)
    val = A.val.copy()
    brows = np.repeat(np.arange(A.nb), np.diff(A.browptr))
    val[np.nonzero(brows == A.bcol)[0][0]] = -np.eye(3)
    M0 = nc.nc_matrix_bsr3(to_dev(torch, A.browptr), to_dev(torch, A.bcol), to_dev(torch, val.reshape(-1)))
    with pytest.raises(nc.NcError) as ei:
        nc.nc_matrix_block_jacobi(M0)
    assert ei.value.status == nc.NC_ERR_ARG
    Mj = nc.nc_matrix_jacobi(nc.nc_matrix_bsr3(to_dev(torch, A.browptr), to_dev(torch, A.bcol),
                                               to_dev(torch, A.val.reshape(-1))))
    with pytest.raises(nc.NcError):
        nc.nc_matrix_block_jacobi(Mj)                                    # already scaled
