"""The paper's FD-3D Poisson problem (Sec. 5.3) at a reduced size, in the
configuration bench.py --workload fd3d runs at nx = 512: matrix-free 7-point
operator on the (nx-1)^3 interior grid, x* = ones, Jacobi scaling, exact
bounds, s = 1.001, nlev = 0, 2, 5.  Iteration counts within +-1 of the
oracle (both polynomial forms), and the paper's trend: the iteration count
falls steeply with the degree (Table 8: 1300 / 325 / 45 iterations at
nx = 512).  With exact bounds and s = 1.001 the degree-3 polynomial still
clusters the smallest eigenvalues (the effect of Sec. 4), so nlev = 2 saves
about 2x here rather than the paper's 4x, whose bounds were estimates."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from nchelpers import need_gpu, rel_err

pytestmark = pytest.mark.gpu

NX = 48


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    import paper_2008_01440_gb300 as nc
    m = NX - 1
    A = nc.nc_matrix_stencil7(m, m, m, 6.0, 1.0, 1.0, 1.0)
    As = nc.nc_matrix_jacobi(A)
    lo, hi = W.stencil7_bounds(W.Stencil7(m, m, m, 1.0, 1 / 6, 1 / 6, 1 / 6))
    ones = torch.ones(m ** 3, dtype=torch.float64, device="cuda")
    b = torch.empty_like(ones)
    nc.nc_matvec(A, ones, b)
    mv = O.stencil7_matvec(m, m, m, 1.0, 1 / 6, 1 / 6, 1 / 6)
    # scaled system A_s y = D^-1/2 b with D = 6 I: D^-1/2 A x* = sqrt(6) A_s x*
    bo = np.sqrt(6.0) * mv(np.ones(m ** 3))
    return torch, nc, As, lo, hi, b, mv, bo


@pytest.mark.parametrize("nlev", [0, 2, 5])
@pytest.mark.parametrize("form", ["chebyshev", "newton"])
def test_fd3d_iterations_match_oracle(env, nlev, form):
    torch, nc, As, lo, hi, b, mv, bo = env
    k = 2 ** nlev - 1
    S = nc.pcg_setup(As, lo, hi, k, 1.001, x0_is_zero=True, poly=form)
    x = torch.zeros_like(b)
    res = nc.pcg_solve(S, b, x, 1e-8, 5000)
    prm = O.cheb_params(lo, hi, 1.001)
    ro = O.pcg(mv, bo, lambda r: O.cheb_apply(mv, r, prm, k), m=k, tol=1e-8, maxit=5000)
    assert res["status"] == 0 and ro.status == 0
    assert abs(res["iters"] - ro.iters) <= 1, (res["iters"], ro.iters)
    assert res["n_spmv"] == (k + 1) * res["iters"]
    assert rel_err(x.cpu().numpy(), np.ones(x.numel())) <= 1e-6


def test_fd3d_trend(env):
    """Fewer iterations with the degree (47^3: 118 / 58 / 9 in the oracle)."""
    torch, nc, As, lo, hi, b, mv, bo = env
    it = {}
    for nlev in (0, 2, 5):
        S = nc.pcg_setup(As, lo, hi, 2 ** nlev - 1, 1.001, x0_is_zero=True)
        x = torch.zeros_like(b)
        it[nlev] = nc.pcg_solve(S, b, x, 1e-8, 5000)["iters"]
    assert it[0] > it[2] > it[5] and it[0] >= 8 * it[5], it
