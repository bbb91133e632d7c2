"""The staged step kernel (NC_STEP_STAGED) and the step-kernel tuner.

The staged variant computes each row exactly as the direct kernel does (the
same fma chain in slot order, the same epilogue), with the tile's matrix
slices and its rows of r and x_{k-2} read from shared memory after bulk
asynchronous copies.  So P_k(A)v, which has no reductions, must be
bit-identical between the variants for every value type, every stage count
and CTAs-per-SM setting, ragged and tiny n (partial last tile: vectors from
global memory), and vectors that are not 16-byte aligned (no vector
staging).  Solves (whose dot products reduce over another grid) must match
the oracle and the direct variant's iteration count.  The tuner must list
what it measured and keep results at the oracle's tolerance."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from nchelpers import csr_to_gpu, elem_err, need_gpu, rel_err, to_dev

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "bf16": 3e-2}


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    import paper_2008_01440_gb300 as nc
    return torch, nc


def _apply(torch, nc, M, n, lo, hi, k, s, v_dev, **opts):
    S = nc.pcg_setup(M, lo, hi, k, s, **opts)
    z = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    nc.pcg_apply_poly(S, v_dev, z)
    info = nc.pcg_get_info(S)
    assert info["faults"] == 0
    return info, z.cpu().numpy()


@pytest.mark.parametrize("grid", [(5, 5, 5), (17, 9, 13), (40, 40, 40), (64, 64, 33)])
@pytest.mark.parametrize("dt", ["f64", "f32", "bf16"])
def test_staged_equals_direct_and_oracle(env, grid, dt):
    """n = 125 (one partial tile), 1989 (ragged tail), 64000 and 135168
    (several waves of tiles) on the scaled log-normal diffusion operator."""
    torch, nc = env
    nx, ny, nz = grid
    A = W.diffusion_3d_7pt_lognormal(nx, seed=nx + ny) if nx == ny == nz else None
    if A is None:
        st = W.stencil7_aniso(nx, ny, nz, 1.0, 0.5, 0.25)
        A = W.stencil7_to_csr(st)
    M = nc.nc_matrix_jacobi(csr_to_gpu(torch, nc, A))
    lo, hi, _, _ = nc.nc_bounds_lanczos(M, 20, to_dev(torch, W.uniform_vector(A.n, seed=3)))
    v = W.uniform_vector(A.n, seed=7)
    vd = to_dev(torch, v)
    k = 10
    idir, zd = _apply(torch, nc, M, A.n, lo, hi, k, 1.001, vd, apply_dtype=dt, spmv_format="psell",
                      step_kernel="direct")
    assert idir["spmv_format"] == "psell" and idir["step_kernel"] == "direct"
    i2, z2 = _apply(torch, nc, M, A.n, lo, hi, k, 1.001, vd, apply_dtype=dt, spmv_format="psell",
                    step_kernel="direct", step_rows_per_thread=2)
    assert i2["step_rows_per_thread"] == 2 and np.array_equal(z2, zd)
    for stages, ctas, rpt, order in ((2, 1, 1, 0), (3, 2, 1, 1), (4, 6, 1, 0), (2, 4, 2, 0), (3, 8, 2, 1),
                                     (2, 6, 1, 1)):
        ist, zs = _apply(torch, nc, M, A.n, lo, hi, k, 1.001, vd, apply_dtype=dt, spmv_format="psell",
                         step_kernel="staged", step_stages=stages, step_ctas_per_sm=ctas,
                         step_rows_per_thread=rpt, step_tile_order=order)
        assert ist["step_kernel"] == "staged" and ist["step_stages"] == stages
        assert ist["step_rows_per_thread"] == rpt and ist["step_tile_order"] == order
        assert np.array_equal(zs, zd), (dt, stages, ctas, rpt, order)
    val, dis = O.jacobi_scale_csr(A.rowptr, A.col, A.val, A.n)
    mv = O.csr_matvec(A.rowptr, A.col, val, A.n)
    ref = O.cheb_apply(mv, v, O.cheb_params(lo, hi, 1.001), k)
    assert rel_err(zd, ref) <= TOL[dt] and elem_err(zd, ref) <= TOL[dt]


@pytest.mark.parametrize("k", [1, 2, 3, 8, 31])
def test_staged_unaligned_vector_and_degrees(env, k):
    """v starts 8 bytes past a 16-byte boundary: the float64 apply reads r
    and its first step's u from v itself, so no vector can be staged; the
    matrix slices still are."""
    torch, nc = env
    A = W.laplacian_2d_5pt(300, 211)   # n = 63300: 248 tiles, the last partial
    lo, hi = W.laplacian_2d_bounds(300, 211)
    M = csr_to_gpu(torch, nc, A)
    v = W.uniform_vector(A.n, seed=k)
    big = torch.zeros(A.n + 1, dtype=torch.float64, device="cuda")
    big[1:] = to_dev(torch, v)
    vd = big[1:]
    assert vd.data_ptr() % 16 == 8
    _, zd = _apply(torch, nc, M, A.n, lo, hi, k, 1.001, vd, spmv_format="psell", step_kernel="direct")
    for rpt in (1, 2):
        _, zs = _apply(torch, nc, M, A.n, lo, hi, k, 1.001, vd, spmv_format="psell", step_kernel="staged",
                       step_rows_per_thread=rpt, step_tile_order=rpt - 1)
        assert np.array_equal(zs, zd), rpt
    ref = O.cheb_apply(O.csr_matvec(A.rowptr, A.col, A.val, A.n), v, O.cheb_params(lo, hi, 1.001), k)
    assert rel_err(zs, ref) <= 1e-12 and elem_err(zs, ref) <= 1e-12


@pytest.mark.parametrize("n", [1, 2, 31, 33, 255, 256, 257, 4097])
def test_staged_tiny_and_ragged(env, n):
    torch, nc = env
    A = W.laplacian_1d(n)
    lo = 4.0 * np.sin(np.pi / (2.0 * (n + 1))) ** 2
    hi = 4.0 * np.sin(n * np.pi / (2.0 * (n + 1))) ** 2
    if n == 1:
        lo, hi = 1.9, 2.1
    M = csr_to_gpu(torch, nc, A)
    v = W.uniform_vector(n, seed=n)
    vd = to_dev(torch, v)
    _, zd = _apply(torch, nc, M, n, lo, hi, 6, 1.001, vd, spmv_format="psell", step_kernel="direct")
    _, z2 = _apply(torch, nc, M, n, lo, hi, 6, 1.001, vd, spmv_format="psell", step_kernel="direct",
                   step_rows_per_thread=2)
    assert np.array_equal(z2, zd)
    for rpt in (1, 2):
        for order in (0, 1):
            _, zs = _apply(torch, nc, M, n, lo, hi, 6, 1.001, vd, spmv_format="psell", step_kernel="staged",
                           step_rows_per_thread=rpt, step_tile_order=order)
            assert np.array_equal(zs, zd), (rpt, order)
    ref = O.cheb_apply(O.csr_matvec(A.rowptr, A.col, A.val, A.n), v, O.cheb_params(lo, hi, 1.001), 6)
    assert rel_err(zs, ref) <= 1e-12


@pytest.mark.parametrize("dt", ["f64", "f32", "bf16"])
def test_staged_solve_matches_direct_and_oracle(env, dt):
    """The dot-product steps (last Chebyshev step with (r, z), q = A p with
    (p, q)) also run staged: same iteration count as the direct variant,
    true residual at the tolerance, and in float64 the oracle's count +-1."""
    torch, nc = env
    N = 48
    A = W.diffusion_3d_7pt_lognormal(N, seed=N)
    M = nc.nc_matrix_jacobi(csr_to_gpu(torch, nc, A))
    lo, hi, _, _ = nc.nc_bounds_lanczos(M, 20, to_dev(torch, W.uniform_vector(A.n, seed=3)))
    b = to_dev(torch, W.uniform_vector(A.n, seed=5))
    out = {}
    for var in ("direct", "staged", "split"):
        S = nc.pcg_setup(M, lo, hi, 10, 1.001, apply_dtype=dt, spmv_format="psell", step_kernel=var,
                         rr_period=50 if dt != "f64" else 0, step_rows_per_thread=2 if dt == "bf16" else 0,
                         step_tile_order=1 if dt == "f32" else 0)
        info = nc.pcg_get_info(S)
        # split: direct plain steps, the dot-product steps as the plain step and a separate dot product
        assert info["step_kernel"] == ("direct" if var == "split" else var) and info["dot_step_kernel"] == var
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        r = nc.pcg_solve(S, b, x, 1e-8, 2000)
        assert nc.pcg_get_info(S)["faults"] == 0
        out[var] = (r, x.cpu().numpy())
    (rd, xd) = out["direct"]
    for var in ("staged", "split"):
        rs, xs = out[var]
        assert rs["status"] == 0 and rs["true_relres"] <= 2e-8
        assert abs(rs["iters"] - rd["iters"]) <= 1
        assert rel_err(xs, xd) <= 1e-6
    rs, xs = out["staged"]
    if dt == "f64":
        val, dis = O.jacobi_scale_csr(A.rowptr, A.col, A.val, A.n)
        mv = O.csr_matvec(A.rowptr, A.col, val, A.n)
        prm = O.cheb_params(lo, hi, 1.001)
        bo = dis * W.uniform_vector(A.n, seed=5)
        ro = O.pcg(mv, bo, lambda r: O.cheb_apply(mv, r, prm, 10), m=10, tol=1e-8, maxit=2000)
        assert abs(rs["iters"] - ro.iters) <= 1
        assert rel_err(xs, dis * ro.x) <= (hi / lo) * 1e-8


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_tuner_lists_candidates_and_keeps_parity(env, dt):
    torch, nc = env
    N = 64
    A = W.diffusion_3d_7pt_lognormal(N, seed=2)
    M = nc.nc_matrix_jacobi(csr_to_gpu(torch, nc, A))
    lo, hi, _, _ = nc.nc_bounds_lanczos(M, 20, to_dev(torch, W.uniform_vector(A.n, seed=3)))
    S = nc.pcg_setup(M, lo, hi, 10, 1.001, apply_dtype=dt, step_kernel="tune")
    info = nc.pcg_get_info(S)
    cands = nc.pcg_tune_candidates(S)
    assert info["tune_candidates"] == len(cands) >= 4
    assert info["num_sms"] >= 1
    kinds = {c["op"] for c in cands}
    assert {"step", "last_step_dot"} <= kinds and (("q_dot" in kinds) == (dt != "f64"))
    for kind in kinds:
        chosen = [c for c in cands if c["op"] == kind and c["chosen"]]
        assert len(chosen) == 1
        best = min(c["us"] for c in cands if c["op"] == kind)
        assert chosen[0]["us"] == best and best > 0
    plain = [c for c in cands if c["op"] == "step" and c["chosen"]][0]
    assert info["step_kernel"] == plain["step_kernel"]
    assert {c["step_kernel"] for c in cands if c["op"] == "step"} == {"direct", "staged"}
    # the dot-product steps also try the plain step plus a separate dot product
    assert {c["step_kernel"] for c in cands if c["op"] != "step"} == {"direct", "staged", "split"}
    v = W.uniform_vector(A.n, seed=9)
    z = torch.empty(A.n, dtype=torch.float64, device="cuda")
    nc.pcg_apply_poly(S, to_dev(torch, v), z)
    val, dis = O.jacobi_scale_csr(A.rowptr, A.col, A.val, A.n)
    ref = O.cheb_apply(O.csr_matvec(A.rowptr, A.col, val, A.n), v, O.cheb_params(lo, hi, 1.001), 10)
    got = z.cpu().numpy()
    assert rel_err(got, ref) <= TOL[dt] and elem_err(got, ref) <= TOL[dt]
    b = to_dev(torch, W.uniform_vector(A.n, seed=5))
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    r = nc.pcg_solve(S, b, x, 1e-8, 2000)
    assert r["status"] == 0 and r["true_relres"] <= 2e-8


def test_direct_options_are_kept(env):
    """Fixed direct choices (prefetch distance, dot-step CTAs) are reported as
    given and change nothing in the result."""
    torch, nc = env
    A = W.laplacian_2d_5pt(120, 90)
    lo, hi = W.laplacian_2d_bounds(120, 90)
    M = csr_to_gpu(torch, nc, A)
    vd = to_dev(torch, W.uniform_vector(A.n, seed=1))
    i0, z0 = _apply(torch, nc, M, A.n, lo, hi, 8, 1.001, vd, apply_dtype="f32", step_kernel="direct")
    i1, z1 = _apply(torch, nc, M, A.n, lo, hi, 8, 1.001, vd, apply_dtype="f32", step_kernel="direct",
                    prefetch_tiles=-1, red_ctas_per_sm=4)
    assert i1["prefetch_tiles"] == 0 and i1["red_ctas_per_sm"] == 4
    assert i0["prefetch_tiles"] == 2 * i0["num_sms"] and i0["tune_candidates"] == 0
    assert np.array_equal(z0, z1)


def _banded(n, offsets):
    """Symmetric banded matrix: 10 on the diagonal, -1 at +-o for o in
    offsets (diagonally dominant, spectrum inside Gershgorin's [4, 16])."""
    rows, vals = [], []
    offs = sorted({0} | set(offsets) | {-o for o in offsets})
    for i in range(n):
        c = np.array([i + o for o in offs if 0 <= i + o < n], dtype=np.int32)
        rows.append(c)
        vals.append(np.where(c == i, 10.0, -1.0))
    rowptr = np.zeros(n + 1, dtype=np.int32)
    rowptr[1:] = np.cumsum([len(r) for r in rows])
    return W.CSR(n, rowptr, np.concatenate(rows), np.concatenate(vals))


@pytest.mark.parametrize("offsets,n", [((1, 2, 500), 50001), ((1000, 3000, 7000), 40000), ((1, 64, 4096), 70001)])
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_staged_gather_windows_and_fallback(env, offsets, n, dt):
    """Banded operators whose offsets are near (0, +-1, +-2, +-500), far
    (+-1000, +-3000, +-7000: every slot gathers a separate stretch of
    x_{k-1}) or mixed (0, +-1, +-64, +-4096): the staged kernel's result is
    the direct kernel's, bit for bit, for both row counts per thread, and
    n % 4 != 0 leaves a ragged last tile."""
    torch, nc = env
    A = _banded(n, offsets)
    M = csr_to_gpu(torch, nc, A)
    v = W.uniform_vector(n, seed=3)
    vd = to_dev(torch, v)
    info, zd = _apply(torch, nc, M, n, 4.0, 16.0, 7, 1.001, vd, apply_dtype=dt, spmv_format="psell",
                      step_kernel="direct")
    assert info["spmv_format"] == "psell"
    _, z2 = _apply(torch, nc, M, n, 4.0, 16.0, 7, 1.001, vd, apply_dtype=dt, spmv_format="psell",
                   step_kernel="direct", step_rows_per_thread=2)
    assert np.array_equal(z2, zd)
    for rpt in (1, 2):
        _, zs = _apply(torch, nc, M, n, 4.0, 16.0, 7, 1.001, vd, apply_dtype=dt, spmv_format="psell",
                       step_kernel="staged", step_rows_per_thread=rpt)
        assert np.array_equal(zs, zd), rpt
    ref = O.cheb_apply(O.csr_matvec(A.rowptr, A.col, A.val, n), v, O.cheb_params(4.0, 16.0, 1.001), 7)
    assert rel_err(zd, ref) <= TOL[dt] and elem_err(zd, ref) <= TOL[dt]


def test_tune_cache_reproduces_the_choice(env, tmp_path, monkeypatch):
    """With NC_TUNE_CACHE set, the first solver on an operator measures and
    appends its choices; a second solver on the same operator reads them
    (nothing measured), runs the same kernels, and gives the same bits."""
    torch, nc = env
    A = W.diffusion_3d_7pt_lognormal(48, seed=5)
    M = nc.nc_matrix_jacobi(csr_to_gpu(torch, nc, A))
    lo, hi, _, _ = nc.nc_bounds_lanczos(M, 20, to_dev(torch, W.uniform_vector(A.n, seed=3)))
    path = tmp_path / "tune.cache"
    monkeypatch.setenv("NC_TUNE_CACHE", str(path))
    vd = to_dev(torch, W.uniform_vector(A.n, seed=9))
    i1, z1 = _apply(torch, nc, M, A.n, lo, hi, 10, 1.001, vd, apply_dtype="f32", step_kernel="tune")
    assert i1["tune_candidates"] > 0 and i1["tune_from_cache"] == 0
    lines = path.read_text().splitlines()
    assert len(lines) == 1 and lines[0].startswith(f"ncpcg-tune-v1 n={A.n} ")
    i2, z2 = _apply(torch, nc, M, A.n, lo, hi, 10, 1.001, vd, apply_dtype="f32", step_kernel="tune")
    assert i2["tune_candidates"] == 0 and i2["tune_from_cache"] == 1
    keys = ("step_kernel", "dot_step_kernel", "step_stages", "step_ctas_per_sm", "step_rows_per_thread",
            "dot_step_stages", "dot_step_ctas_per_sm", "prefetch_tiles", "red_ctas_per_sm")
    assert {k: i1[k] for k in keys} == {k: i2[k] for k in keys}
    assert np.array_equal(z1, z2)
    assert len(path.read_text().splitlines()) == 1
    # another precision is another signature: measured and appended
    i3, _ = _apply(torch, nc, M, A.n, lo, hi, 10, 1.001, vd, apply_dtype="f64", step_kernel="tune")
    assert i3["tune_from_cache"] == 0 and len(path.read_text().splitlines()) == 2
