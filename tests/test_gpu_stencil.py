"""GPU parity of the matrix-free 7-point stencil path against the oracle.

The oracle's stencil product is written from the definition on a zero-padded
grid; exact spectral bounds come from the closed form of workloads.
"""
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


SHAPES = [(1, 1, 1), (2, 1, 1), (5, 3, 2), (31, 9, 7), (33, 17, 5), (16, 16, 16), (40, 3, 70), (64, 64, 64),
          (130, 7, 9)]


def _stencil(shape, seed):
    rng = np.random.default_rng(seed)
    wx, wy, wz = rng.uniform(0.01, 1.0, 3)
    return W.stencil7_aniso(*shape, wx, wy, wz)


@pytest.mark.parametrize("shape", SHAPES)
def test_stencil_matvec_parity(env, shape):
    torch, nc = env
    st = _stencil(shape, 1)
    M = nc.nc_matrix_stencil7(st.nx, st.ny, st.nz, st.c0, st.cx, st.cy, st.cz)
    x = W.uniform_vector(st.n, seed=2)
    y = torch.empty(st.n, dtype=torch.float64, device="cuda")
    nc.nc_matvec(M, to_dev(torch, x), y)
    ref = O.stencil7_matvec(st.nx, st.ny, st.nz, st.c0, st.cx, st.cy, st.cz)(x)
    assert elem_err(y.cpu().numpy(), ref) <= 1e-14


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("k,s", [(0, 1.0), (1, 1.0), (5, 1.001), (31, 1.001)])
def test_stencil_apply_parity(env, shape, k, s):
    torch, nc = env
    st = _stencil(shape, 3)
    M = nc.nc_matrix_stencil7(st.nx, st.ny, st.nz, st.c0, st.cx, st.cy, st.cz)
    lo, hi = W.stencil7_bounds(st)
    if hi <= lo:
        lo, hi = 0.5 * lo, lo
    S = nc.pcg_setup(M, lo, hi, k, s)
    v = W.uniform_vector(st.n, seed=4)
    z = torch.empty(st.n, dtype=torch.float64, device="cuda")
    nc.pcg_apply_poly(S, to_dev(torch, v), z)
    ref = O.cheb_apply(O.stencil7_matvec(st.nx, st.ny, st.nz, st.c0, st.cx, st.cy, st.cz), v,
                       O.cheb_params(lo, hi, s), k)
    got = z.cpu().numpy()
    assert rel_err(got, ref) <= 1e-12 and elem_err(got, ref) <= 1e-12


@pytest.mark.parametrize("shape,k", [((24, 24, 24), 8), ((48, 20, 33), 20), ((16, 16, 16), 31), ((71, 71, 71), 31)])
def test_stencil_solve_parity(env, shape, k):
    """Jacobi-scaled anisotropic stencil, exact bounds of the scaled operator,
    s = 1.001: iteration count within +-1 of the oracle, residual 1e-8."""
    torch, nc = env
    st = _stencil(shape, 5)
    M = nc.nc_matrix_jacobi(nc.nc_matrix_stencil7(st.nx, st.ny, st.nz, st.c0, st.cx, st.cy, st.cz))
    sc = W.Stencil7(st.nx, st.ny, st.nz, *O.jacobi_scale_stencil7(st.c0, st.cx, st.cy, st.cz))
    lo, hi = W.stencil7_bounds(sc)
    S = nc.pcg_setup(M, lo, hi, k, 1.001)
    b = W.uniform_vector(st.n, seed=6)
    x = torch.zeros(st.n, dtype=torch.float64, device="cuda")
    res = nc.pcg_solve(S, to_dev(torch, b), x, 1e-8, 3000)
    mv = O.stencil7_matvec(sc.nx, sc.ny, sc.nz, sc.c0, sc.cx, sc.cy, sc.cz)
    dis = 1.0 / np.sqrt(st.c0)
    ro = O.pcg(mv, dis * b, lambda r: O.cheb_apply(mv, r, O.cheb_params(lo, hi, 1.001), k), m=k, tol=1e-8,
               maxit=3000)
    assert res["status"] == 0 and ro.status == 0
    assert abs(res["iters"] - ro.iters) <= 1, (res["iters"], ro.iters)
    assert res["relres"] <= 1e-8 and res["true_relres"] <= 2e-8
    xo = dis * ro.x
    assert rel_err(x.cpu().numpy(), xo) <= (hi / lo) * 1e-8


def test_stencil_matches_assembled_csr(env):
    """The same operator as a stencil handle and as CSR gives the same solve."""
    torch, nc = env
    st = _stencil((20, 30, 25), 7)
    C = W.stencil7_to_csr(st)
    lo, hi = W.stencil7_bounds(st)
    b = to_dev(torch, W.uniform_vector(st.n, seed=8))
    out = []
    for M in (nc.nc_matrix_stencil7(st.nx, st.ny, st.nz, st.c0, st.cx, st.cy, st.cz),
              nc.nc_matrix_csr(to_dev(torch, C.rowptr), to_dev(torch, C.col), to_dev(torch, C.val))):
        S = nc.pcg_setup(M, lo, hi, 12, 1.001)
        x = torch.zeros(st.n, dtype=torch.float64, device="cuda")
        out.append((nc.pcg_solve(S, b, x, 1e-9, 2000), x.cpu().numpy()))
    assert abs(out[0][0]["iters"] - out[1][0]["iters"]) <= 1
    assert rel_err(out[0][1], out[1][1]) <= 1e-6


@pytest.mark.parametrize("dt", ["f32"])
def test_stencil_mixed_precision(env, dt):
    torch, nc = env
    st = _stencil((64, 64, 64), 9)
    M = nc.nc_matrix_jacobi(nc.nc_matrix_stencil7(st.nx, st.ny, st.nz, st.c0, st.cx, st.cy, st.cz))
    sc = W.Stencil7(st.nx, st.ny, st.nz, *O.jacobi_scale_stencil7(st.c0, st.cx, st.cy, st.cz))
    lo, hi = W.stencil7_bounds(sc)
    S = nc.pcg_setup(M, lo, hi, 31, 1.001, apply_dtype=dt, rr_period=50)
    v = W.uniform_vector(st.n, seed=1)
    z = torch.empty(st.n, dtype=torch.float64, device="cuda")
    nc.pcg_apply_poly(S, to_dev(torch, v), z)
    mv = O.stencil7_matvec(sc.nx, sc.ny, sc.nz, sc.c0, sc.cx, sc.cy, sc.cz)
    ref = O.cheb_apply(mv, v, O.cheb_params(lo, hi, 1.001), 31)
    assert rel_err(z.cpu().numpy(), ref) <= 1e-4
    b = W.uniform_vector(st.n, seed=2)
    x = torch.zeros(st.n, dtype=torch.float64, device="cuda")
    res = nc.pcg_solve(S, to_dev(torch, b), x, 1e-8, 3000)
    ro = O.pcg(mv, b / np.sqrt(st.c0), lambda r: O.cheb_apply(mv, r, O.cheb_params(lo, hi, 1.001), 31), m=31,
               tol=1e-8)
    assert res["status"] == 0 and res["true_relres"] <= 2e-8
    assert abs(res["iters"] - ro.iters) <= max(2, 0.1 * ro.iters)


def test_stencil_lanczos_and_gershgorin(env):
    torch, nc = env
    st = _stencil((30, 20, 10), 11)
    M = nc.nc_matrix_stencil7(st.nx, st.ny, st.nz, st.c0, st.cx, st.cy, st.cz)
    lo_ex, hi_ex = W.stencil7_bounds(st)
    g = nc.nc_gershgorin(M)
    assert abs(g - (st.c0 + 2 * (st.cx + st.cy + st.cz))) < 1e-14
    v0 = W.uniform_vector(st.n, seed=3)
    lo, hi, rmin, rmax = nc.nc_bounds_lanczos(M, 20, to_dev(torch, v0))
    mv = O.stencil7_matvec(st.nx, st.ny, st.nz, st.c0, st.cx, st.cy, st.cz)
    lo_o, hi_o, _ = O.lanczos_bounds(mv, v0, 20, gershgorin=g)
    assert abs(lo - lo_o) <= 1e-9 * lo_o and abs(hi - hi_o) <= 1e-9 * hi_o
    assert hi >= hi_ex and lo >= lo_ex


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_stencil_tuned_chunking_is_bit_identical(env, dt):
    """The tuner picks the z-chunk (and, in float, the planes per batch) of
    the plain steps by measurement; every candidate computes each point by the
    same operations, so P_k(A)v is bit-identical to the size policy's, and
    matches the oracle."""
    torch, nc = env
    st = _stencil((100, 90, 120), 5)   # 1,080,000 points: AUTO tunes it too
    M = nc.nc_matrix_stencil7(st.nx, st.ny, st.nz, st.c0, st.cx, st.cy, st.cz)
    Ms = nc.nc_matrix_jacobi(M)
    sc = W.Stencil7(st.nx, st.ny, st.nz, 1.0, st.cx / st.c0, st.cy / st.c0, st.cz / st.c0)
    lo, hi = W.stencil7_bounds(sc)
    vd = to_dev(torch, W.uniform_vector(st.n, seed=8))
    out = {}
    for mode in ("direct", "tune", "auto"):
        S = nc.pcg_setup(Ms, lo, hi, 9, 1.001, apply_dtype=dt, step_kernel=mode)
        z = torch.empty(st.n, dtype=torch.float64, device="cuda")
        nc.pcg_apply_poly(S, vd, z)
        info = nc.pcg_get_info(S)
        out[mode] = (info, nc.pcg_tune_candidates(S), z.cpu().numpy())
    info_d, cands_d, zd = out["direct"]
    info_t, cands_t, zt = out["tune"]
    assert not cands_d and info_d["stencil_zchunk"] > 0
    assert len(cands_t) >= 3 and sum(c["chosen"] for c in cands_t) == 1
    chosen = [c for c in cands_t if c["chosen"]][0]
    assert chosen["us"] == min(c["us"] for c in cands_t)
    assert info_t["stencil_zchunk"] == chosen["zchunk"] and chosen["zchunk"] >= 4
    assert np.array_equal(zt, zd) and np.array_equal(out["auto"][2], zd)
    mv = O.stencil7_matvec(st.nx, st.ny, st.nz, 1.0, sc.cx, sc.cy, sc.cz)
    ref = O.cheb_apply(mv, vd.cpu().numpy(), O.cheb_params(lo, hi, 1.001), 9)
    tol = 1e-12 if dt == "f64" else 1e-5
    assert rel_err(zd, ref) <= tol and elem_err(zd, ref) <= tol
