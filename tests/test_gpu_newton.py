"""The Newton form of the preconditioner (Algorithm 1) on the GPU.

- Against the oracle's recursive apply (oracle.newton_apply, same algorithm):
  1e-12 relative, norm-wise and element by element.
- Theorem 3.1 at scale: for k = 2^nlev - 1 the Newton polynomial equals the
  Chebyshev one, so the GPU's two forms agree on the full 128^3 system, and
  both agree with the oracle's Chebyshev apply (1e-10: two different
  evaluation orders of a degree-31 polynomial).
- PCG with the Newton form: the oracle's iteration count within +-1, Table 4
  counts.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
import workloads as W
from conftest import GOLDEN
from nchelpers import csr_to_gpu, elem_err, need_gpu, rel_err, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    import paper_2008_01440_gb300 as nc
    return torch, nc


def newton_ref(A, lo, hi, s, nlev, v):
    theta = s * (lo + hi) / 2
    delta = (hi - lo) / 2
    z = O.newton_zetas(theta - delta, theta + delta, nlev)
    return O.newton_apply(O.csr_matvec(A.rowptr, A.col, A.val, A.n), v, z, nlev)


@pytest.mark.parametrize("fmt", ["csr", "sell", "psell"])
@pytest.mark.parametrize("nlev", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("s", [1.0, 1.001])
def test_newton_apply_matches_oracle(env, nlev, s, fmt):
    torch, nc = env
    A = W.laplacian_2d_5pt(64, 64)
    lo, hi = W.laplacian_2d_bounds(64, 64)
    k = 2 ** nlev - 1
    S = nc.pcg_setup(csr_to_gpu(torch, nc, A), lo, hi, k, s, poly="newton", spmv_format=fmt)
    v = W.uniform_vector(A.n, seed=nlev)
    z = torch.empty(A.n, dtype=torch.float64, device="cuda")
    nc.pcg_apply_poly(S, to_dev(torch, v), z)
    got = z.cpu().numpy()
    ref = newton_ref(A, lo, hi, s, nlev, v)
    assert rel_err(got, ref) <= 1e-12 and elem_err(got, ref) <= 1e-12
    # the Chebyshev form of the same degree (Theorem 3.1)
    cheb = O.cheb_apply(O.csr_matvec(A.rowptr, A.col, A.val, A.n), v, O.cheb_params(lo, hi, s), k)
    assert rel_err(got, cheb) <= 1e-10


def test_newton_ragged_and_tiny(env):
    torch, nc = env
    for n in (1, 2, 33, 257, 1000):
        A = W.laplacian_1d(n)
        lo = 4 * np.sin(np.pi / (2 * (n + 1))) ** 2
        hi = max(4 * np.sin(n * np.pi / (2 * (n + 1))) ** 2, 1.5 * lo)
        S = nc.pcg_setup(csr_to_gpu(torch, nc, A), lo, hi, 7, 1.001, poly="newton")
        v = W.uniform_vector(n, seed=n)
        z = torch.empty(n, dtype=torch.float64, device="cuda")
        nc.pcg_apply_poly(S, to_dev(torch, v), z)
        assert rel_err(z.cpu().numpy(), newton_ref(A, lo, hi, 1.001, 3, v)) <= 1e-12


def test_newton_equals_chebyshev_at_scale(env):
    """Theorem 3.1 on the 128^3 variable-coefficient system (n = 2,097,152),
    Jacobi scaled, with the oracle's Lanczos bounds: nlev = 3 and 5."""
    torch, nc = env
    with open(os.path.join(GOLDEN, "c2_oracle.json")) as f:
        g = json.load(f)
    A = W.diffusion_3d_7pt_lognormal(128, seed=g["seed_matrix"])
    M = nc.nc_matrix_jacobi(csr_to_gpu(torch, nc, A))
    lo, hi, s = g["lmin"], g["lmax"], g["theta_scale"]
    v = W.uniform_vector(A.n, seed=31)
    vd = to_dev(torch, v)
    val, _ = O.jacobi_scale_csr(A.rowptr, A.col, A.val, A.n)
    mv = O.csr_matvec(A.rowptr, A.col, val, A.n)
    for nlev in (3, 5):
        k = 2 ** nlev - 1
        out = {}
        for form in ("newton", "chebyshev"):
            S = nc.pcg_setup(M, lo, hi, k, s, poly=form)
            z = torch.empty(A.n, dtype=torch.float64, device="cuda")
            nc.pcg_apply_poly(S, vd, z)
            out[form] = z.cpu().numpy()
            S.close()
        assert rel_err(out["newton"], out["chebyshev"]) <= 1e-10, nlev
        ref = O.cheb_apply(mv, v, O.cheb_params(lo, hi, s), k)
        assert rel_err(out["newton"], ref) <= 1e-10 and elem_err(out["newton"], ref) <= 1e-10


@pytest.mark.parametrize("nlev", [2, 4])
def test_newton_pcg_matches_oracle(env, nlev):
    torch, nc = env
    A = W.diffusion_3d_7pt_lognormal(32, seed=11)
    M = nc.nc_matrix_jacobi(csr_to_gpu(torch, nc, A))
    val, dis = O.jacobi_scale_csr(A.rowptr, A.col, A.val, A.n)
    mv = O.csr_matvec(A.rowptr, A.col, val, A.n)
    lo, hi, _, _ = nc.nc_bounds_lanczos(M, 20, to_dev(torch, W.uniform_vector(A.n, seed=3)))
    k = 2 ** nlev - 1
    b = W.uniform_vector(A.n, seed=5)
    S = nc.pcg_setup(M, lo, hi, k, 1.001, poly="newton")
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    res = nc.pcg_solve(S, to_dev(torch, b), x, 1e-8, 2000)
    theta, delta = 1.001 * (lo + hi) / 2, (hi - lo) / 2
    zt = O.newton_zetas(theta - delta, theta + delta, nlev)
    ro = O.pcg(mv, dis * b, lambda r: O.newton_apply(mv, r, zt, nlev), m=k, tol=1e-8, maxit=2000)
    assert res["status"] == 0 and ro.status == 0
    assert abs(res["iters"] - ro.iters) <= 1, (res["iters"], ro.iters)
    assert res["n_spmv"] == (k + 1) * res["iters"] and res["n_dot"] == 3 * res["iters"]
    assert res["true_relres"] <= 1e-7
    assert rel_err(x.cpu().numpy(), dis * ro.x) <= (hi / lo) * 1e-8
    # graph and host loop run the same kernels
    S2 = nc.pcg_setup(M, lo, hi, k, 1.001, poly="newton", use_graph=False)
    x2 = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    assert nc.pcg_solve(S2, to_dev(torch, b), x2, 1e-8, 2000) == res and torch.equal(x2, x)


def test_newton_argument_checks(env):
    torch, nc = env
    A = W.laplacian_2d_5pt(16, 16)
    lo, hi = W.laplacian_2d_bounds(16, 16)
    M = csr_to_gpu(torch, nc, A)
    with pytest.raises(nc.NcError) as ei:
        nc.pcg_setup(M, lo, hi, 8, 1.0, poly="newton")          # 8 is not 2^j - 1
    assert ei.value.status == nc.NC_ERR_ARG
    with pytest.raises(nc.NcError) as ei:
        nc.pcg_setup(M, lo, hi, 7, 1.0, poly="newton", apply_dtype="f32")
    assert ei.value.status == nc.NC_ERR_UNSUPPORTED
    S = nc.pcg_setup(M, lo, hi, 7, 1.0, poly="newton", persistent=True)
    assert not nc.pcg_get_info(S)["persistent"]                 # the cluster solve is Chebyshev only
    S0 = nc.pcg_setup(M, lo, hi, 0, 1.0, poly="newton")          # nlev = 0: P = 1/theta'
    v = W.uniform_vector(A.n, seed=1)
    z = torch.empty(A.n, dtype=torch.float64, device="cuda")
    nc.pcg_apply_poly(S0, to_dev(torch, v), z)
    assert rel_err(z.cpu().numpy(), v / ((lo + hi) / 2)) <= 1e-15
