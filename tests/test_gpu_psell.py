"""The offset-pattern sliced layout (NC_FORMAT_PSELL): slices store no column
indices, only which distinct set of offsets col - row they use.

With its diagonal stored (keep_diagonal) its products must equal the plain
sliced layout's exactly: both run the same fma chain per row in column
order, and a slot a row lacks holds a 0, whose fma leaves the sum unchanged.
A constant diagonal left out of the layout (the default) changes only the
rounding: those results are checked against the oracle and the stored form.  Both are checked against the oracle as well,
together with the conditions under which the solver falls back to SELL-32
(columns not increasing, more than 64 offsets in a slice, too many distinct
sets), a row without a diagonal (no shifted operator), grid faces whose
padded slots point outside the matrix (clamped gathers of weight 0), mixed
precision and several right-hand sides."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from nchelpers import csr_to_gpu, elem_err, need_gpu, rel_err, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    import paper_2008_01440_gb300 as nc
    return torch, nc


def apply(torch, nc, M, n, lo, hi, k, s, v, **opts):
    S = nc.pcg_setup(M, lo, hi, k, s, **opts)
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    nc.pcg_apply_poly(S, to_dev(torch, v), z)
    return nc.pcg_get_info(S), z.cpu().numpy()


def csr_from_rows(n, rows, vals):
    rowptr = np.zeros(n + 1, dtype=np.int32)
    rowptr[1:] = np.cumsum([len(r) for r in rows])
    return W.CSR(n, rowptr, np.concatenate(rows).astype(np.int32), np.concatenate(vals).astype(np.float64))


@pytest.mark.parametrize("grid", [(7, 9), (45, 37), (64, 64)])
@pytest.mark.parametrize("k,s", [(1, 1.0), (8, 1.001), (31, 1.001)])
def test_laplacian_equals_sell_and_oracle(env, grid, k, s):
    """n = 63 and 1665 leave a ragged last slice; the faces' rows lack the
    offsets -nx, +nx, -1, +1 of their slices (padded slots, clamped gathers)."""
    torch, nc = env
    nx, ny = grid
    A = W.laplacian_2d_5pt(nx, ny)
    lo, hi = W.laplacian_2d_bounds(nx, ny)
    M = csr_to_gpu(torch, nc, A)
    v = W.uniform_vector(A.n, seed=k)
    ip, zp = apply(torch, nc, M, A.n, lo, hi, k, s, v, spmv_format="psell", keep_diagonal=True)
    isl, zs = apply(torch, nc, M, A.n, lo, hi, k, s, v, spmv_format="sell")
    assert ip["spmv_format"] == "psell" and isl["spmv_format"] == "sell" and ip["diag_folded"] == 0
    assert 1 <= ip["patterns"] <= 9 and ip["padding"] < 1.5
    assert np.array_equal(zp, zs)
    ref = O.cheb_apply(O.csr_matvec(A.rowptr, A.col, A.val, A.n), v, O.cheb_params(lo, hi, s), k)
    assert rel_err(zp, ref) <= 1e-12 and elem_err(zp, ref) <= 1e-12
    # the Laplacian's constant diagonal (4) left out of the layout
    iff, zf = apply(torch, nc, M, A.n, lo, hi, k, s, v, spmv_format="psell")
    assert iff["diag_folded"] == 1 and iff["diag_value"] == 4.0 - iff["shift"] and iff["padding"] < 1.0
    assert rel_err(zf, ref) <= 1e-12 and elem_err(zf, ref) <= 1e-12


@pytest.mark.parametrize("N", [21, 32])
@pytest.mark.parametrize("dt", ["f64", "f32", "bf16"])
def test_diffusion_solve_equals_sell(env, N, dt):
    torch, nc = env
    A = W.diffusion_3d_7pt_lognormal(N, seed=N)
    M = nc.nc_matrix_jacobi(csr_to_gpu(torch, nc, A))
    lo, hi, _, _ = nc.nc_bounds_lanczos(M, 20, to_dev(torch, W.uniform_vector(A.n, seed=3)))
    b = to_dev(torch, W.uniform_vector(A.n, seed=5))
    out = {}
    for fmt, keep in (("psell", True), ("sell", False), ("psell", False)):
        S = nc.pcg_setup(M, lo, hi, 10, 1.001, apply_dtype=dt, spmv_format=fmt, keep_diagonal=keep)
        assert nc.pcg_get_info(S)["spmv_format"] == fmt
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        out[fmt, keep] = (nc.pcg_solve(S, b, x, 1e-8, 2000), x.cpu().numpy())
    (rp, xp), (rs, xs) = out["psell", True], out["sell", False]
    assert rp["status"] == 0 and rp["true_relres"] <= 2e-8
    assert rp["iters"] == rs["iters"] and np.array_equal(xp, xs)
    # the scaled diagonal (exactly 1) left out: the same iterations +-1, the solution within reach
    rf, xf = out["psell", False]
    assert rf["status"] == 0 and abs(rf["iters"] - rp["iters"]) <= 1
    assert rel_err(xf, xp) <= (hi / lo) * 1e-8
    # and against the oracle's PCG (float64 only: the others report error against it)
    if dt == "f64":
        val, dis = O.jacobi_scale_csr(A.rowptr, A.col, A.val, A.n)
        mv = O.csr_matvec(A.rowptr, A.col, val, A.n)
        prm = O.cheb_params(lo, hi, 1.001)
        bo = dis * W.uniform_vector(A.n, seed=5)
        ro = O.pcg(mv, bo, lambda r: O.cheb_apply(mv, r, prm, 10), m=10, tol=1e-8, maxit=2000)
        assert abs(rp["iters"] - ro.iters) <= 1 and abs(rf["iters"] - ro.iters) <= 1
        assert rel_err(xp, dis * ro.x) <= (hi / lo) * 1e-8 and rel_err(xf, dis * ro.x) <= (hi / lo) * 1e-8


def test_falls_back_when_columns_do_not_increase(env):
    torch, nc = env
    A = W.laplacian_2d_5pt(40, 40)
    rows, vals = [], []
    for i in range(A.n):
        a, b = A.rowptr[i], A.rowptr[i + 1]
        rows.append(A.col[a:b][::-1])
        vals.append(A.val[a:b][::-1])
    B = csr_from_rows(A.n, rows, vals)
    lo, hi = W.laplacian_2d_bounds(40, 40)
    v = W.uniform_vector(A.n, seed=2)
    info, z = apply(torch, nc, csr_to_gpu(torch, nc, B), A.n, lo, hi, 8, 1.001, v, spmv_format="psell")
    assert info["spmv_format"] == "sell" and info["patterns"] == 0
    ref = O.cheb_apply(O.csr_matvec(A.rowptr, A.col, A.val, A.n), v, O.cheb_params(lo, hi, 1.001), 8)
    assert rel_err(z, ref) <= 1e-12


def test_falls_back_on_unstructured_columns(env):
    """Random columns: far more than 64 distinct offsets per slice."""
    torch, nc = env
    rng = np.random.default_rng(8)
    n = 3000
    rows, vals = [], []
    for i in range(n):
        c = np.unique(np.concatenate([[i], rng.integers(0, n, 6)]))
        rows.append(c)
        vals.append(np.where(c == i, 8.0, -0.5))
    B = csr_from_rows(n, rows, vals)
    M = csr_to_gpu(torch, nc, B)
    v = W.uniform_vector(n, seed=4)
    ref = O.cheb_apply(O.csr_matvec(B.rowptr, B.col, B.val, n), v, O.cheb_params(5.0, 11.0, 1.0), 6)
    for fmt, expect in (("psell", "sell"), ("auto", "sell")):
        info, z = apply(torch, nc, M, n, 5.0, 11.0, 6, 1.0, v, spmv_format=fmt)
        assert info["spmv_format"] == expect
        assert rel_err(z, ref) <= 1e-12


def test_falls_back_when_the_sets_do_not_repeat(env):
    """Three offsets per slice, but a different set in every slice: the
    distinct sets exceed the 16384-offset table.  (The diagonal varies, so
    it stays in the layout: folded out, two offsets per slice would fit.)"""
    torch, nc = env
    n = 1 << 18
    rows, vals = [], []
    for i in range(n):
        d = 1 + (i >> 5)
        c = [j for j in (i - d, i, i + d) if 0 <= j < n]
        rows.append(np.array(c))
        vals.append(np.array([4.0 + 0.25 * (i % 3) if j == i else -1.0 for j in c]))
    B = csr_from_rows(n, rows, vals)
    M = csr_to_gpu(torch, nc, B)
    v = W.uniform_vector(n, seed=6)
    info, z = apply(torch, nc, M, n, 2.0, 6.0, 4, 1.0, v, spmv_format="psell")
    assert info["spmv_format"] == "sell"
    ref = O.cheb_apply(O.csr_matvec(B.rowptr, B.col, B.val, n), v, O.cheb_params(2.0, 6.0, 1.0), 4)
    assert rel_err(z, ref) <= 1e-12


def test_row_without_diagonal_stores_a_itself(env):
    torch, nc = env
    A = W.laplacian_2d_5pt(33, 30)
    rows, vals = [], []
    for i in range(A.n):
        a, b = A.rowptr[i], A.rowptr[i + 1]
        keep = A.col[a:b] != i if i == 500 else np.ones(b - a, bool)
        rows.append(A.col[a:b][keep])
        vals.append(A.val[a:b][keep])
    B = csr_from_rows(A.n, rows, vals)
    v = W.uniform_vector(A.n, seed=9)
    info, z = apply(torch, nc, csr_to_gpu(torch, nc, B), A.n, 0.5, 8.0, 6, 1.0, v, spmv_format="psell")
    assert info["spmv_format"] == "psell" and info["shift"] == 0.0
    ref = O.cheb_apply(O.csr_matvec(B.rowptr, B.col, B.val, A.n), v, O.cheb_params(0.5, 8.0, 1.0), 6)
    assert rel_err(z, ref) <= 1e-12 and elem_err(z, ref) <= 1e-12


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_multi_rhs_equals_sell(env, dt):
    torch, nc = env
    A = W.diffusion_3d_7pt_lognormal(21, seed=2)
    M = nc.nc_matrix_jacobi(csr_to_gpu(torch, nc, A))
    lo, hi, _, _ = nc.nc_bounds_lanczos(M, 20, to_dev(torch, W.uniform_vector(A.n, seed=3)))
    B = torch.stack([to_dev(torch, W.uniform_vector(A.n, seed=40 + c)) for c in range(5)])
    out = {}
    for fmt in ("psell", "sell"):
        S = nc.pcg_setup(M, lo, hi, 12, 1.001, apply_dtype=dt, spmv_format=fmt, keep_diagonal=True)
        assert nc.pcg_get_info(S)["spmv_format"] == fmt
        X = torch.zeros_like(B)
        out[fmt] = (nc.pcg_solve_multi(S, B, X, 1e-8, 2000), X.cpu().numpy())
    (rp, xp), (rs, xs) = out["psell"], out["sell"]
    assert [r["iters"] for r in rp] == [r["iters"] for r in rs]
    assert all(r["status"] == 0 and r["true_relres"] <= 2e-8 for r in rp)
    assert np.array_equal(xp, xs)


def test_cluster_solve_keeps_plain_sell(env):
    torch, nc = env
    A = W.laplacian_2d_5pt(64, 64)
    lo, hi = W.laplacian_2d_bounds(64, 64)
    S = nc.pcg_setup(csr_to_gpu(torch, nc, A), lo, hi, 8, 1.001, persistent=True)
    info = nc.pcg_get_info(S)
    assert info["spmv_format"] == "sell" and info["persistent"] == 1
