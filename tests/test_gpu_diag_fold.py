"""Constant diagonal left out of the offset-pattern layout: when every row's
a_ii is the same (the Jacobi-scaled matrix, whose scaled diagonal is exactly
1, or a constant-coefficient operator), the layout stores no diagonal slot
and the steps apply it through their u coefficient, y = (ca + cd d) u + ...
+ cd (A - d I) u -- one product and one stored value fewer per row.

Checked against the FP64 oracle (apply element-wise, solves +-1 iteration),
against the same solver with the diagonal stored (keep_diagonal), in the
multi-right-hand-side block and in engine slots, and that a varying
diagonal is never folded."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from nchelpers import csr_to_gpu, elem_err, need_gpu, rel_err, to_dev

pytestmark = pytest.mark.gpu

TOL_APPLY = 1e-12


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    import paper_2008_01440_gb300 as nc
    return torch, nc


def _scaled_system(torch, nc, N, seed):
    A = W.diffusion_3d_7pt_lognormal(N, seed=seed)
    val, dis = O.jacobi_scale_csr(A.rowptr, A.col, A.val, A.n)
    M = nc.nc_matrix_jacobi(csr_to_gpu(torch, nc, A))
    lo, hi, _, _ = nc.nc_bounds_lanczos(M, 20, to_dev(torch, W.uniform_vector(A.n, seed=99)))
    return A, val, dis, M, lo, hi


@pytest.mark.parametrize("dt", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("k", [1, 2, 3, 10, 31])
def test_folded_apply_matches_oracle(env, dt, k):
    torch, nc = env
    A, val, dis, M, lo, hi = _scaled_system(torch, nc, 23, 5)
    S = nc.pcg_setup(M, lo, hi, k, 1.001, spmv_format="psell", apply_dtype=dt)
    info = nc.pcg_get_info(S)
    assert info["spmv_format"] == "psell" and info["diag_folded"] == 1
    assert info["diag_value"] == 1.0 - info["shift"]
    assert info["padding"] < 1.0   # the diagonal is not stored
    v = W.uniform_vector(A.n, seed=k)
    z = torch.empty(A.n, dtype=torch.float64, device="cuda")
    nc.pcg_apply_poly(S, to_dev(torch, v), z)
    mv = O.csr_matvec(A.rowptr, A.col, val, A.n)
    ref = O.cheb_apply(mv, v, O.cheb_params(lo, hi, 1.001), k)
    got = z.cpu().numpy()
    tol = {"f64": TOL_APPLY, "f32": 2e-5, "bf16": 5e-2}[dt]
    assert rel_err(got, ref) <= tol
    if dt == "f64":
        assert elem_err(got, ref) <= TOL_APPLY
    # the same solver with the diagonal stored
    Sk = nc.pcg_setup(M, lo, hi, k, 1.001, spmv_format="psell", apply_dtype=dt, keep_diagonal=True)
    assert nc.pcg_get_info(Sk)["diag_folded"] == 0
    zk = torch.empty_like(z)
    nc.pcg_apply_poly(Sk, to_dev(torch, v), zk)
    assert rel_err(got, zk.cpu().numpy()) <= (1e-13 if dt == "f64" else tol)


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_folded_solve_matches_oracle(env, dt):
    torch, nc = env
    A, val, dis, M, lo, hi = _scaled_system(torch, nc, 26, 8)
    b = W.uniform_vector(A.n, seed=3)
    mv = O.csr_matvec(A.rowptr, A.col, val, A.n)
    ro = O.pcg(mv, dis * b, lambda r: O.cheb_apply(mv, r, O.cheb_params(lo, hi, 1.001), 10), m=10, tol=1e-8,
               maxit=5000)
    S = nc.pcg_setup(M, lo, hi, 10, 1.001, spmv_format="psell", apply_dtype=dt, x0_is_zero=True)
    assert nc.pcg_get_info(S)["diag_folded"] == 1
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    r = nc.pcg_solve(S, to_dev(torch, b), x, 1e-8, 5000)
    assert r["status"] == 0 and r["true_relres"] <= 2e-8
    assert abs(r["iters"] - ro.iters) <= (1 if dt == "f64" else 3)
    assert rel_err(x.cpu().numpy(), dis * ro.x) <= (hi / lo) * 1e-8
    # several right-hand sides in one block
    B = np.stack([W.uniform_vector(A.n, seed=40 + c) for c in range(3)])
    X = torch.zeros(3, A.n, dtype=torch.float64, device="cuda")
    res = nc.pcg_solve_multi(S, to_dev(torch, B), X, 1e-8, 5000)
    for c in range(3):
        roc = O.pcg(mv, dis * B[c], lambda r: O.cheb_apply(mv, r, O.cheb_params(lo, hi, 1.001), 10), m=10,
                    tol=1e-8, maxit=5000)
        assert res[c]["status"] == 0 and abs(res[c]["iters"] - roc.iters) <= (1 if dt == "f64" else 3)
        assert rel_err(X[c].cpu().numpy(), dis * roc.x) <= (hi / lo) * 1e-8
    # and as engine slots (a group of the three)
    eng = nc.pcg_batch_create(3, 3 * A.n, 32, f64_apply=(dt == "f64"))
    slots = nc.pcg_batch_add_solver_multi(eng, S, to_dev(torch, B))
    assert nc.pcg_batch_run(eng, 1e-8, 5000) == 0
    for c, sl in enumerate(slots):
        done, rs = nc.pcg_batch_status(eng, sl)
        assert done and rs["status"] == 0 and abs(rs["iters"] - res[c]["iters"]) <= 1
        xe = torch.empty(A.n, dtype=torch.float64, device="cuda")
        nc.pcg_batch_collect(eng, sl, xe)
        torch.cuda.synchronize()
        assert rel_err(xe.cpu().numpy(), X[c].cpu().numpy()) <= (hi / lo) * 1e-8
    eng.close()


def test_fold_needs_a_constant_diagonal(env):
    """The unscaled log-normal operator (a varying diagonal) keeps its
    diagonal; the 2D Laplacian (4 on every row) folds 4 - theta'; its
    apply matches the oracle element-wise."""
    torch, nc = env
    A = W.diffusion_3d_7pt_lognormal(16, seed=2)
    S = nc.pcg_setup(csr_to_gpu(torch, nc, A), 0.1, 2.0, 4, 1.0, spmv_format="psell")
    assert nc.pcg_get_info(S)["diag_folded"] == 0
    L = W.laplacian_2d_5pt(37, 29)
    lo, hi = W.laplacian_2d_bounds(37, 29)
    S = nc.pcg_setup(csr_to_gpu(torch, nc, L), lo, hi, 8, 1.0, spmv_format="psell")
    info = nc.pcg_get_info(S)
    assert info["diag_folded"] == 1 and info["diag_value"] == 4.0 - info["shift"]
    v = W.uniform_vector(L.n, seed=1)
    z = torch.empty(L.n, dtype=torch.float64, device="cuda")
    nc.pcg_apply_poly(S, to_dev(torch, v), z)
    ref = O.cheb_apply(O.csr_matvec(L.rowptr, L.col, L.val, L.n), v, O.cheb_params(lo, hi, 1.0), 8)
    assert elem_err(z.cpu().numpy(), ref) <= TOL_APPLY
