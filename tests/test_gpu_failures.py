"""Failure detection without a GPU fault: non-finite inputs and an indefinite
operator end a solve with a status code (NC_ERR_BREAKDOWN / NC_ERR_INDEFINITE)
after a bounded number of iterations, the CUDA context stays usable, and in
the batch engine one bad slot does not disturb the others."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from nchelpers import csr_to_gpu, need_gpu, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    import paper_2008_01440_gb300 as nc
    return torch, nc


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
@pytest.mark.parametrize("fmt", ["csr", "sell", "psell"])
def test_nonfinite_rhs_breaks_down_and_solver_recovers(env, bad, fmt):
    torch, nc = env
    A = W.laplacian_2d_5pt(64, 64)
    lo, hi = W.laplacian_2d_bounds(64, 64)
    S = nc.pcg_setup(csr_to_gpu(torch, nc, A), lo, hi, 8, 1.001, spmv_format=fmt)
    b = W.uniform_vector(A.n, seed=3)
    bb = b.copy()
    bb[100] = bad
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    r = nc.pcg_solve(S, to_dev(torch, bb), x, 1e-8, 500)
    assert r["status"] == nc.NC_ERR_BREAKDOWN
    assert r["iters"] == 0
    # the same solver then solves a good system normally
    x.zero_()
    r = nc.pcg_solve(S, to_dev(torch, b), x, 1e-8, 500)
    assert r["status"] == 0 and r["true_relres"] <= 2e-8


def test_nonfinite_rhs_stencil_and_blocks(env):
    torch, nc = env
    st = W.stencil7_aniso(20, 18, 16, 1.0, 0.5, 0.25)
    M = nc.nc_matrix_jacobi(nc.nc_matrix_stencil7(st.nx, st.ny, st.nz, st.c0, st.cx, st.cy, st.cz))
    sc = W.Stencil7(st.nx, st.ny, st.nz, *O.jacobi_scale_stencil7(st.c0, st.cx, st.cy, st.cz))
    lo, hi = W.stencil7_bounds(sc)
    S = nc.pcg_setup(M, lo, hi, 10, 1.001)
    b = W.uniform_vector(st.n, seed=1)
    b[7] = float("nan")
    x = torch.zeros(st.n, dtype=torch.float64, device="cuda")
    assert nc.pcg_solve(S, to_dev(torch, b), x, 1e-8, 500)["status"] == nc.NC_ERR_BREAKDOWN
    A, bq = W.elasticity_q1_bsr3(6, seed=2)
    Mb = nc.nc_matrix_jacobi(nc.nc_matrix_bsr3(to_dev(torch, A.browptr), to_dev(torch, A.bcol),
                                               to_dev(torch, A.val.reshape(-1))))
    lo, hi, _, _ = nc.nc_bounds_lanczos(Mb, 20, to_dev(torch, W.uniform_vector(A.n, seed=3)))
    Sb = nc.pcg_setup(Mb, lo, hi, 8, 1.001)
    bq = bq.copy()
    bq[-1] = float("inf")
    xb = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    assert nc.pcg_solve(Sb, to_dev(torch, bq), xb, 1e-8, 500)["status"] == nc.NC_ERR_BREAKDOWN


@pytest.mark.parametrize("persistent", [False, True])
def test_indefinite_operator_detected(env, persistent):
    """A = -T (negative definite) with the bounds of T: with k = 0, z = r/theta'
    gives (r, z) > 0 and then (p, A p) < 0 at the first iteration."""
    torch, nc = env
    n = 500
    T = W.laplacian_1d(n)
    A = W.CSR(n, T.rowptr, T.col, -T.val)
    lo = 4 * np.sin(np.pi / (2 * (n + 1))) ** 2
    hi = 4 * np.sin(n * np.pi / (2 * (n + 1))) ** 2
    S = nc.pcg_setup(csr_to_gpu(torch, nc, A), lo, hi, 0, 1.0, persistent=persistent, spmv_format="sell")
    b = W.uniform_vector(n, seed=2)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    r = nc.pcg_solve(S, to_dev(torch, b), x, 1e-8, 100)
    assert r["status"] == nc.NC_ERR_INDEFINITE
    assert r["iters"] == 0 and r["n_dot"] == 2   # (r, z) and (p, q)
    # the oracle stops the same way
    ro = O.pcg(O.csr_matvec(A.rowptr, A.col, A.val, n), b, lambda v: v / (0.5 * (lo + hi)), m=0, tol=1e-8,
               maxit=100)
    assert ro.status != 0 and ro.iters == 0


def test_batch_bad_slot_is_isolated(env):
    """One slot with a NaN right-hand side finishes with NC_ERR_BREAKDOWN; the
    other slots' results are bit-for-bit those of a batch without it."""
    torch, nc = env
    rng = np.random.default_rng(9)
    sy = []
    for i in range(5):
        nx, ny, nz = (int(v) for v in rng.integers(10, 30, 3))
        st = W.stencil7_aniso(nx, ny, nz, *rng.uniform(0.05, 1.0, 3))
        sc = W.Stencil7(nx, ny, nz, *O.jacobi_scale_stencil7(st.c0, st.cx, st.cy, st.cz))
        lo, hi = W.stencil7_bounds(sc)
        sy.append((st, lo, hi, W.uniform_vector(st.n, seed=50 + i)))
    bad = sy[2][3].copy()
    bad[5] = float("nan")

    def run(with_bad):
        B = nc.pcg_batch_create(8, sum(t[0].n for t in sy) + 10, 16)
        slots = {}
        for i, (st, lo, hi, b) in enumerate(sy):
            if i == 2 and not with_bad:
                continue
            bb = bad if i == 2 else b
            slots[i] = nc.pcg_batch_add(B, st.nx, st.ny, st.nz, st.c0, st.cx, st.cy, st.cz, lo, hi, 12, 1.001,
                                        to_dev(torch, bb))
        assert nc.pcg_batch_run(B, 1e-8, 2000) == 0
        out = {}
        for i, s in slots.items():
            done, res = nc.pcg_batch_status(B, s)
            assert done
            x = torch.empty(sy[i][0].n, dtype=torch.float64, device="cuda")
            nc.pcg_batch_collect(B, s, x)
            out[i] = (res, x.cpu().numpy())
        return out

    with_bad = run(True)
    without = run(False)
    assert with_bad[2][0]["status"] == nc.NC_ERR_BREAKDOWN
    for i in (0, 1, 3, 4):
        assert with_bad[i][0]["status"] == 0
        assert with_bad[i][0] == without[i][0] and np.array_equal(with_bad[i][1], without[i][1])
