"""GPU parity of the CSR path through the C ABI against the FP64 oracle.

Tolerances: P_k(A)v in float64 must match the oracle to 1e-12 relative, both
norm-wise and element by element (relative to max|ref|); PCG must reach the
same iteration count within +-1 and the 1e-8 relative residual.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from nchelpers import csr_to_gpu, elem_err, gershgorin_np, need_gpu, rel_err, to_dev

pytestmark = pytest.mark.gpu

TOL_APPLY = 1e-12


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    import paper_2008_01440_gb300 as nc
    return torch, nc


def scaled(A):
    val, dis = O.jacobi_scale_csr(A.rowptr, A.col, A.val, A.n)
    return W.CSR(A.n, A.rowptr, A.col, val), dis


def lap64():
    A = W.laplacian_2d_5pt(64, 64)
    lo, hi = W.laplacian_2d_bounds(64, 64)
    return A, lo, hi


def test_matvec_and_jacobi_parity(env):
    torch, nc = env
    A = W.diffusion_3d_7pt_lognormal(20, seed=3)
    M = csr_to_gpu(torch, nc, A)
    x = W.uniform_vector(A.n, seed=1)
    y = torch.empty(A.n, dtype=torch.float64, device="cuda")
    nc.nc_matvec(M, to_dev(torch, x), y)
    ref = O.csr_matvec(A.rowptr, A.col, A.val, A.n)(x)
    assert elem_err(y.cpu().numpy(), ref) < 1e-14
    Ms = nc.nc_matrix_jacobi(M)
    nc.nc_matvec(Ms, to_dev(torch, x), y)
    As, _ = scaled(A)
    ref = O.csr_matvec(As.rowptr, As.col, As.val, A.n)(x)
    assert elem_err(y.cpu().numpy(), ref) < 1e-14
    g = nc.nc_gershgorin(Ms)
    assert g == gershgorin_np(As.rowptr, As.col, As.val, A.n) or abs(g - gershgorin_np(As.rowptr, As.col, As.val, A.n)) < 1e-14


FORMATS = ["csr", "sell", "psell"]


@pytest.mark.parametrize("fmt", FORMATS)
@pytest.mark.parametrize("k,s", [(0, 1.0), (1, 1.0), (2, 1.001), (3, 1.0), (8, 1.0), (8, 1.001), (31, 1.001)])
def test_apply_poly_laplacian64(env, k, s, fmt):
    torch, nc = env
    A, lo, hi = lap64()
    M = csr_to_gpu(torch, nc, A)
    S = nc.pcg_setup(M, lo, hi, k, s, spmv_format=fmt)
    assert nc.pcg_get_info(S)["spmv_format"] == fmt
    v = W.uniform_vector(A.n, seed=k + 10)
    z = torch.empty(A.n, dtype=torch.float64, device="cuda")
    nc.pcg_apply_poly(S, to_dev(torch, v), z)
    ref = O.cheb_apply(O.csr_matvec(A.rowptr, A.col, A.val, A.n), v, O.cheb_params(lo, hi, s), k)
    got = z.cpu().numpy()
    assert rel_err(got, ref) <= TOL_APPLY and elem_err(got, ref) <= TOL_APPLY


@pytest.mark.parametrize("fmt", FORMATS)
@pytest.mark.parametrize("N,k", [(24, 10), (24, 20), (24, 40), (31, 20)])
def test_apply_poly_diffusion_lanczos_bounds(env, N, k, fmt):
    torch, nc = env
    A = W.diffusion_3d_7pt_lognormal(N, seed=N)
    As, _ = scaled(A)
    M = nc.nc_matrix_jacobi(csr_to_gpu(torch, nc, A))
    v0 = W.uniform_vector(A.n, seed=99)
    lo, hi, rmin, rmax = nc.nc_bounds_lanczos(M, 20, to_dev(torch, v0))
    mv = O.csr_matvec(As.rowptr, As.col, As.val, A.n)
    g = gershgorin_np(As.rowptr, As.col, As.val, A.n)
    lo_o, hi_o, info = O.lanczos_bounds(mv, v0, 20, gershgorin=g)
    assert abs(lo - lo_o) <= 1e-9 * lo_o and abs(hi - hi_o) <= 1e-9 * hi_o
    S = nc.pcg_setup(M, lo, hi, k, 1.001, spmv_format=fmt)
    v = W.uniform_vector(A.n, seed=7)
    z = torch.empty(A.n, dtype=torch.float64, device="cuda")
    nc.pcg_apply_poly(S, to_dev(torch, v), z)
    ref = O.cheb_apply(mv, v, O.cheb_params(lo, hi, 1.001), k)
    got = z.cpu().numpy()
    assert rel_err(got, ref) <= TOL_APPLY and elem_err(got, ref) <= TOL_APPLY


def test_auto_layout_choice(env):
    """AUTO picks the offset-pattern layout for a grid operator (small
    padding, few distinct offset sets), SELL-32 when forced or in the cluster
    solve, and CSR for a matrix with one dense row (padding far above 1.5)."""
    torch, nc = env
    A = W.diffusion_3d_7pt_lognormal(20, seed=1)
    S = nc.pcg_setup(csr_to_gpu(torch, nc, A), 0.1, 2.0, 4, 1.0)
    info = nc.pcg_get_info(S)
    assert info["spmv_format"] == "psell" and 1.0 <= info["padding"] < 1.2
    # interior, and one set per combination of missing faces: at most 3^2 x 2
    assert 1 <= info["patterns"] <= 18
    # the sliced layouts store the shifted operator A - theta' I (every row has a diagonal)
    assert info["shift"] == info["theta"] == 1.0 * (0.1 + 2.0) / 2
    info = nc.pcg_get_info(nc.pcg_setup(csr_to_gpu(torch, nc, A), 0.1, 2.0, 4, 1.0, spmv_format="sell"))
    assert info["spmv_format"] == "sell" and info["patterns"] == 0 and 1.0 <= info["padding"] < 1.2
    n = 2000
    rows = [np.array([i]) for i in range(n)]
    rows[7] = np.arange(n)
    rowptr = np.zeros(n + 1, dtype=np.int32)
    rowptr[1:] = np.cumsum([len(r) for r in rows])
    B = W.CSR(n, rowptr, np.concatenate(rows).astype(np.int32), np.ones(rowptr[-1]))
    S2 = nc.pcg_setup(csr_to_gpu(torch, nc, B), 0.1, 2.0, 4, 1.0)
    assert nc.pcg_get_info(S2)["spmv_format"] == "csr"


@pytest.mark.parametrize("fmt", FORMATS)
def test_apply_poly_ragged_rows_and_long_rows(env, fmt):
    """Empty rows, a row longer than one shared-memory chunk, n not a multiple
    of the 256-row tile: exercises every branch of the row kernel."""
    torch, nc = env
    rng = np.random.default_rng(4)
    n = 1000 + 37
    rows = []
    for i in range(n):
        if i % 97 == 5:
            rows.append(np.array([], dtype=np.int64))
        elif i == 300:
            rows.append(np.arange(n))                 # dense row (> 2048 nnz? n=1037: no)
        else:
            rows.append(np.unique(rng.integers(0, n, size=rng.integers(1, 12))))
    # one very long row across several chunks
    big = 3 * 2048 + 11
    n2 = big + 5
    rows2 = [np.unique(rng.integers(0, n2, size=4)) for _ in range(n2)]
    rows2[n2 - 3] = np.arange(n2)
    for rr, nn in ((rows, n), (rows2, n2)):
        rowptr = np.zeros(nn + 1, dtype=np.int32)
        rowptr[1:] = np.cumsum([len(r) for r in rr])
        col = np.concatenate([np.sort(r) for r in rr]).astype(np.int32)
        val = rng.uniform(-1, 1, col.size)
        Ac = W.CSR(nn, rowptr, col, val)
        M = csr_to_gpu(torch, nc, Ac)
        S = nc.pcg_setup(M, 0.5, 3.0, 5, 1.0, spmv_format=fmt)
        # rows without a stored diagonal: no shifted operator
        assert nc.pcg_get_info(S)["shift"] == 0.0
        v = rng.uniform(-1, 1, nn)
        z = torch.empty(nn, dtype=torch.float64, device="cuda")
        nc.pcg_apply_poly(S, to_dev(torch, v), z)
        ref = O.cheb_apply(O.csr_matvec(rowptr, col, val, nn), v, O.cheb_params(0.5, 3.0, 1.0), 5)
        assert rel_err(z.cpu().numpy(), ref) <= TOL_APPLY


@pytest.mark.parametrize("fmt", FORMATS)
@pytest.mark.parametrize("n", [1, 2, 31, 33, 255, 256, 257])
def test_apply_poly_tiny(env, n, fmt):
    torch, nc = env
    A = W.laplacian_1d(n)
    lo = 4 * np.sin(np.pi / (2 * (n + 1))) ** 2
    hi = 4 * np.sin(n * np.pi / (2 * (n + 1))) ** 2
    if hi <= lo:
        hi = lo * 1.5
    M = csr_to_gpu(torch, nc, A)
    S = nc.pcg_setup(M, lo, hi, 6, 1.001, spmv_format=fmt)
    v = W.uniform_vector(n, seed=n)
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    nc.pcg_apply_poly(S, to_dev(torch, v), z)
    ref = O.cheb_apply(O.csr_matvec(A.rowptr, A.col, A.val, n), v, O.cheb_params(lo, hi, 1.001), 6)
    assert rel_err(z.cpu().numpy(), ref) <= TOL_APPLY


def _solve_both(torch, nc, A, lo, hi, k, s, b, jacobi, tol=1e-8, maxit=5000, **opts):
    M0 = csr_to_gpu(torch, nc, A)
    M = nc.nc_matrix_jacobi(M0) if jacobi else M0
    S = nc.pcg_setup(M, lo, hi, k, s, **opts)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    res = nc.pcg_solve(S, to_dev(torch, b), x, tol, maxit)
    if jacobi:
        As, dis = scaled(A)
        mv = O.csr_matvec(As.rowptr, As.col, As.val, A.n)
        bo = dis * b
    else:
        mv = O.csr_matvec(A.rowptr, A.col, A.val, A.n)
        bo = b
    prm = O.cheb_params(lo, hi, s)
    ro = O.pcg(mv, bo, lambda r: O.cheb_apply(mv, r, prm, k), m=k, tol=tol, maxit=maxit)
    xo = dis * ro.x if jacobi else ro.x
    return res, ro, x.cpu().numpy(), xo


@pytest.mark.parametrize("fmt", FORMATS)
@pytest.mark.parametrize("k,s", [(8, 1.0), (8, 1.001), (0, 1.0), (15, 1.01)])
def test_solve_laplacian64(env, k, s, fmt):
    """The 64x64 5-point Laplacian with b = A x*, x* ~ U[-1,1], exact bounds."""
    torch, nc = env
    A, lo, hi = lap64()
    b = W.rhs_from_solution(A, W.uniform_vector(A.n, seed=1))
    res, ro, x, xo = _solve_both(torch, nc, A, lo, hi, k, s, b, jacobi=False, spmv_format=fmt)
    assert res["status"] == 0 and ro.status == 0
    assert abs(res["iters"] - ro.iters) <= 1, (res["iters"], ro.iters)
    assert res["relres"] <= 1e-8 and res["true_relres"] <= 2e-8
    assert res["n_dot"] == 3 * res["iters"]
    assert res["n_spmv"] == (k + 1) * res["iters"]
    kappa = hi / lo
    assert rel_err(x, xo) <= kappa * 1e-8


@pytest.mark.parametrize("fmt", FORMATS)
@pytest.mark.parametrize("k", [10, 20, 40])
def test_solve_diffusion_reduced(env, k, fmt):
    """Variable-coefficient 3D diffusion (log-normal, sigma=1) at 32^3, Jacobi
    scaled, 20-step Lanczos bounds, s = 1.001."""
    torch, nc = env
    A = W.diffusion_3d_7pt_lognormal(32, seed=11)
    As, _ = scaled(A)
    g = gershgorin_np(As.rowptr, As.col, As.val, A.n)
    lo, hi, _ = O.lanczos_bounds(O.csr_matvec(As.rowptr, As.col, As.val, A.n), W.uniform_vector(A.n, seed=3), 20,
                                 gershgorin=g)
    b = W.uniform_vector(A.n, seed=5)
    res, ro, x, xo = _solve_both(torch, nc, A, lo, hi, k, 1.001, b, jacobi=True, spmv_format=fmt)
    assert res["status"] == 0 and ro.status == 0
    assert abs(res["iters"] - ro.iters) <= 1, (res["iters"], ro.iters)
    assert res["relres"] <= 1e-8 and res["true_relres"] <= 1e-7


def test_graph_and_host_loop_identical(env):
    torch, nc = env
    A, lo, hi = lap64()
    b = to_dev(torch, W.uniform_vector(A.n, seed=3))
    M = csr_to_gpu(torch, nc, A)
    out = []
    for g in (True, False):
        S = nc.pcg_setup(M, lo, hi, 8, 1.001, use_graph=g)
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        r = nc.pcg_solve(S, b, x, 1e-8, 1000)
        out.append((r, x.clone()))
        # second solve on the same solver reuses the graph and gives the same answer
        x2 = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        r2 = nc.pcg_solve(S, b, x2, 1e-8, 1000)
        assert r2 == r and torch.equal(x2, x)
    assert out[0][0] == out[1][0]
    assert torch.equal(out[0][1], out[1][1])


def test_solve_host_buffers_identical(env):
    torch, nc = env
    A, lo, hi = lap64()
    bh = W.uniform_vector(A.n, seed=8)
    M = csr_to_gpu(torch, nc, A)
    S = nc.pcg_setup(M, lo, hi, 8, 1.0, x0_is_zero=True)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    r1 = nc.pcg_solve(S, to_dev(torch, bh), x, 1e-8, 1000)
    xh = np.zeros(A.n)
    r2 = nc.pcg_solve_host(S, bh, xh, 1e-8, 1000)
    assert r1 == r2 and np.array_equal(xh, x.cpu().numpy())


def test_nonzero_initial_guess(env):
    torch, nc = env
    A, lo, hi = lap64()
    xs = W.uniform_vector(A.n, seed=1)
    b = W.rhs_from_solution(A, xs)
    M = csr_to_gpu(torch, nc, A)
    S = nc.pcg_setup(M, lo, hi, 8, 1.0)
    x = to_dev(torch, xs + 1e-3 * W.uniform_vector(A.n, seed=2))
    res = nc.pcg_solve(S, to_dev(torch, b), x, 1e-8, 1000)
    ro = O.pcg(O.csr_matvec(A.rowptr, A.col, A.val, A.n), b,
               lambda r: O.cheb_apply(O.csr_matvec(A.rowptr, A.col, A.val, A.n), r, O.cheb_params(lo, hi, 1.0), 8),
               m=8, x0=xs + 1e-3 * W.uniform_vector(A.n, seed=2), tol=1e-8)
    assert res["status"] == 0 and abs(res["iters"] - ro.iters) <= 1


def test_edge_cases(env):
    torch, nc = env
    A, lo, hi = lap64()
    M = csr_to_gpu(torch, nc, A)
    S = nc.pcg_setup(M, lo, hi, 8, 1.0)
    # b = 0 -> x = 0 in zero iterations, even from a nonzero guess
    x = torch.ones(A.n, dtype=torch.float64, device="cuda")
    res = nc.pcg_solve(S, torch.zeros(A.n, dtype=torch.float64, device="cuda"), x, 1e-8, 100)
    assert res["status"] == 0 and res["iters"] == 0 and torch.count_nonzero(x) == 0
    # maxit
    b = to_dev(torch, W.uniform_vector(A.n, seed=1))
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    res = nc.pcg_solve(S, b, x, 1e-14, 3)
    assert res["status"] == nc.NC_ERR_MAXIT and res["iters"] == 3
    res = nc.pcg_solve(S, b, x, 1e-8, 0)
    assert res["status"] == nc.NC_ERR_MAXIT and res["iters"] == 0
    # beta far too small: P_k(A) indefinite (odd k) -> reported, no hang
    Sbad = nc.pcg_setup(M, lo, hi / 8, 11, 1.0)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    res = nc.pcg_solve(Sbad, b, x, 1e-10, 200)
    assert res["status"] == nc.NC_ERR_INDEFINITE
    # bad arguments are rejected before any work
    with pytest.raises(nc.NcError):
        nc.pcg_setup(M, hi, lo, 8, 1.0)
    with pytest.raises(nc.NcError):
        nc.pcg_setup(M, lo, hi, -1, 1.0)
    # empty system
    E = nc.nc_matrix_csr(torch.zeros(1, dtype=torch.int32, device="cuda"),
                         torch.zeros(0, dtype=torch.int32, device="cuda"),
                         torch.zeros(0, dtype=torch.float64, device="cuda"))
    SE = nc.pcg_setup(E, 1.0, 2.0, 4, 1.0)
    e = torch.zeros(0, dtype=torch.float64, device="cuda")
    assert nc.pcg_solve(SE, e, e.clone(), 1e-8, 10)["iters"] == 0


@pytest.mark.parametrize("fmt", FORMATS)
@pytest.mark.parametrize("dt,tol_apply", [("f32", 1e-5), ("bf16", 3e-2)])
def test_mixed_precision_apply_and_solve(env, dt, tol_apply, fmt):
    """F32 / BF16 matrix inside P_k with a float64 outer CG: the apply is
    reported against the FP64 oracle and the solve still reaches 1e-8."""
    torch, nc = env
    A = W.diffusion_3d_7pt_lognormal(32, seed=11)
    As, _ = scaled(A)
    mv = O.csr_matvec(As.rowptr, As.col, As.val, A.n)
    lo, hi, _ = O.lanczos_bounds(mv, W.uniform_vector(A.n, seed=3), 20,
                                 gershgorin=gershgorin_np(As.rowptr, As.col, As.val, A.n))
    M = nc.nc_matrix_jacobi(csr_to_gpu(torch, nc, A))
    S = nc.pcg_setup(M, lo, hi, 20, 1.001, apply_dtype=dt, spmv_format=fmt)
    v = W.uniform_vector(A.n, seed=7)
    z = torch.empty(A.n, dtype=torch.float64, device="cuda")
    nc.pcg_apply_poly(S, to_dev(torch, v), z)
    ref = O.cheb_apply(mv, v, O.cheb_params(lo, hi, 1.001), 20)
    assert rel_err(z.cpu().numpy(), ref) <= tol_apply
    b = W.uniform_vector(A.n, seed=5)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    res = nc.pcg_solve(S, to_dev(torch, b), x, 1e-8, 2000)
    assert res["status"] == 0 and res["relres"] <= 1e-8 and res["true_relres"] <= 1e-7


@pytest.mark.parametrize("dt,period", [("f64", 5), ("f32", 5), ("f32", 50), ("bf16", 7)])
def test_residual_replacement(env, dt, period):
    """FP64 residual replacement every `period` iterations (the mixed-precision
    safeguard): same iteration count as the FP64 oracle with the same
    replacement schedule (within +-1 for f64, 10% for reduced precision)."""
    torch, nc = env
    A = W.diffusion_3d_7pt_lognormal(32, seed=11)
    As, dis = scaled(A)
    mv = O.csr_matvec(As.rowptr, As.col, As.val, A.n)
    lo, hi, _ = O.lanczos_bounds(mv, W.uniform_vector(A.n, seed=3), 20,
                                 gershgorin=gershgorin_np(As.rowptr, As.col, As.val, A.n))
    b = W.uniform_vector(A.n, seed=5)
    k = 10
    res, ro, x, xo = _solve_both(torch, nc, A, lo, hi, k, 1.001, b, jacobi=True, apply_dtype=dt, rr_period=period)
    ro2 = O.pcg(mv, dis * b, lambda r: O.cheb_apply(mv, r, O.cheb_params(lo, hi, 1.001), k), m=k, tol=1e-8,
                rr_period=period)
    assert res["status"] == 0 and res["true_relres"] <= 2e-8
    tol_it = 1 if dt == "f64" else max(2, 0.1 * ro2.iters)
    assert abs(res["iters"] - ro2.iters) <= tol_it
    assert res["n_replace"] == (res["iters"] - 1) // period


def test_autotune_layout(env):
    """TUNE measures both layouts on the matrix and keeps the faster; the
    result of the apply is the same either way."""
    torch, nc = env
    A = W.diffusion_3d_7pt_lognormal(48, seed=2)
    M = nc.nc_matrix_jacobi(csr_to_gpu(torch, nc, A))
    lo, hi = 0.01, 2.0
    S = nc.pcg_setup(M, lo, hi, 10, 1.001, spmv_format="tune")
    info = nc.pcg_get_info(S)
    assert info["tune_us_plain"] > 0 and info["tune_us_sliced"] > 0
    faster = "sell" if info["tune_us_sliced"] <= info["tune_us_plain"] else "csr"
    assert info["spmv_format"] == faster
    S2 = nc.pcg_setup(M, lo, hi, 10, 1.001, spmv_format="csr" if faster == "sell" else "sell")
    v = to_dev(torch, W.uniform_vector(A.n, seed=1))
    z1 = torch.empty(A.n, dtype=torch.float64, device="cuda")
    z2 = torch.empty(A.n, dtype=torch.float64, device="cuda")
    nc.pcg_apply_poly(S, v, z1)
    nc.pcg_apply_poly(S2, v, z2)
    assert rel_err(z1.cpu().numpy(), z2.cpu().numpy()) <= 1e-13
    # with a dense row the sliced layout is skipped (padding > 4x): no timing of it
    n = 3000
    rows = [np.array([i]) for i in range(n)]
    rows[5] = np.arange(n)
    rowptr = np.zeros(n + 1, dtype=np.int32)
    rowptr[1:] = np.cumsum([len(r) for r in rows])
    B = W.CSR(n, rowptr, np.concatenate(rows).astype(np.int32), np.ones(rowptr[-1]))
    S3 = nc.pcg_setup(csr_to_gpu(torch, nc, B), 0.1, 2.0, 4, 1.0, spmv_format="tune")
    assert nc.pcg_get_info(S3)["spmv_format"] == "csr"


def test_power_method_bound_matches_oracle(env):
    """Sec. 5.1's beta_0 estimate: the GPU power method against the oracle's
    (same start vector and iteration count), below the exact lambda_max of the
    2D Laplacian and approaching it."""
    torch, nc = env
    A, lo, hi = lap64()
    M = csr_to_gpu(torch, nc, A)
    v0 = W.uniform_vector(A.n, seed=4)
    mv = O.csr_matvec(A.rowptr, A.col, A.val, A.n)
    for iters in (1, 5, 40):
        lam = nc.nc_bounds_power(M, iters, to_dev(torch, v0))
        ref = O.power_method(mv, v0, iters)
        assert abs(lam - ref) <= 1e-12 * ref
        assert lam <= hi * (1 + 1e-12)
    assert nc.nc_bounds_power(M, 400, to_dev(torch, v0)) >= 0.99 * hi
    # scaled diffusion operator: below the Lanczos upper end
    Ad = W.diffusion_3d_7pt_lognormal(20, seed=2)
    Md = nc.nc_matrix_jacobi(csr_to_gpu(torch, nc, Ad))
    _, hi_l, _, rmax = nc.nc_bounds_lanczos(Md, 20, to_dev(torch, W.uniform_vector(Ad.n, seed=3)))
    lam = nc.nc_bounds_power(Md, 30, to_dev(torch, W.uniform_vector(Ad.n, seed=3)))
    assert lam <= hi_l and lam >= 0.8 * rmax
    with pytest.raises(nc.NcError):
        nc.nc_bounds_power(M, 0, to_dev(torch, v0))
