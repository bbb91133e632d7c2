"""The no-allocation apply, nc_apply_poly_csr_noalloc, against pcg_apply_poly.

Some callers cannot allocate device memory when they apply the
preconditioner: a solver that hands out all device memory from its own fixed
arena, a real-time loop where cudaMalloc/cudaFree (and the synchronisation
they can imply) are not allowed, or a plugin inside a framework that owns the
device heap.  For them the library computes z = P_k(A) v in one fixed device
array instead of per-solver work vectors.  These tests call that entry point
through the C ABI twice in a row (the array keeps the previous call's
contents) and compare each result with the allocating entry point at the
parity tolerance of the other GPU tests.

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from nchelpers import csr_to_gpu, elem_err, need_gpu, rel_err, to_dev

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    import paper_2008_01440_gb300 as nc
    return torch, nc


def _cases():
    lap = W.laplacian_2d_5pt(64, 64)
    lo, hi = W.laplacian_2d_bounds(64, 64)
    dif = W.diffusion_3d_7pt_lognormal(40, seed=4)
    # k mod 3 = 0, 1, 2 all occur: the three rotating vectors (z and the two
    # halves of the array) take x_j in slot (k - j) mod 3, so each residue
    # puts a different vector in z between reads
    return [("laplacian64", lap, lo, hi, 8, 1.0), ("laplacian64", lap, lo, hi, 0, 1.0),
            ("laplacian64", lap, lo, hi, 1, 1.0), ("laplacian64", lap, lo, hi, 4, 1.001),
            ("laplacian64", lap, lo, hi, 3, 1.0), ("laplacian64", lap, lo, hi, 6, 1.001),
            ("laplacian64", lap, lo, hi, 9, 1.001),
            ("diffusion40", dif, None, None, 20, 1.001), ("diffusion40", dif, None, None, 31, 1.001),
            ("diffusion40", dif, None, None, 12, 1.001)]


@pytest.mark.parametrize("case", range(10))
def test_noalloc_matches_allocating_apply_twice(env, case):
    torch, nc = env
    name, A, lo, hi, k, s = _cases()[case]
    rp, cl, vl = to_dev(torch, A.rowptr), to_dev(torch, A.col), to_dev(torch, A.val)
    M = nc.nc_matrix_csr(rp, cl, vl)
    if lo is None:
        lo, hi, _, _ = nc.nc_bounds_lanczos(M, 20, to_dev(torch, W.uniform_vector(A.n, seed=3)))
    S = nc.pcg_setup(M, lo, hi, k, s)
    for call, seed in enumerate((11, 12)):
        v = to_dev(torch, W.uniform_vector(A.n, seed=seed))
        z_ref = torch.empty(A.n, dtype=torch.float64, device="cuda")
        nc.pcg_apply_poly(S, v, z_ref)
        z = torch.full((A.n,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        nc.nc_apply_poly_csr_noalloc(rp, cl, vl, lo, hi, k, s, v, z)
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        got, ref = z.cpu().numpy(), z_ref.cpu().numpy()
        assert np.all(np.isfinite(got)), (name, k, call)
        assert rel_err(got, ref) <= TOL and elem_err(got, ref) <= TOL, (name, k, call)
        if call == 1:   # the array exists since the first call: nothing more is allocated
            assert free_after == free_before


def test_noalloc_rejects_n_above_limit(env):
    torch, nc = env
    nmax = nc.nc_apply_poly_noalloc_max_n()
    assert nmax == 1 << 20
    n = nmax + 1
    rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    cl = torch.zeros(1, dtype=torch.int32, device="cuda")
    vl = torch.zeros(1, dtype=torch.float64, device="cuda")
    v = torch.zeros(n, dtype=torch.float64, device="cuda")
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(nc.NcError) as ei:
        nc.nc_apply_poly_csr_noalloc(rp, cl, vl, 0.5, 2.0, 4, 1.0, v, z)
    assert ei.value.status == nc.NC_ERR_SCRATCH_LIMIT
    assert "scratch" in str(ei.value)


@pytest.mark.parametrize("k", [3, 7])
def test_noalloc_matches_oracle_at_the_size_limit(env, k):
    """n = 2^20 exactly (the 1024 x 1024 Laplacian): the second half of the
    array ends exactly at the array's end.  Compared with the FP64 oracle's
    Algorithm 2, element by element, on two calls in a row."""
    torch, nc = env
    A = W.laplacian_2d_5pt(1024, 1024)
    assert A.n == nc.nc_apply_poly_noalloc_max_n()
    lo, hi = W.laplacian_2d_bounds(1024, 1024)
    rp, cl, vl = to_dev(torch, A.rowptr), to_dev(torch, A.col), to_dev(torch, A.val)
    mv = O.csr_matvec(A.rowptr, A.col, A.val, A.n)
    prm = O.cheb_params(lo, hi, 1.001)
    for seed in (21, 22):
        v_h = W.uniform_vector(A.n, seed=seed)
        ref = O.cheb_apply(mv, v_h, prm, k)
        z = torch.full((A.n,), float("nan"), dtype=torch.float64, device="cuda")
        nc.nc_apply_poly_csr_noalloc(rp, cl, vl, lo, hi, k, 1.001, to_dev(torch, v_h), z)
        got = z.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel_err(got, ref) <= TOL and elem_err(got, ref) <= TOL, (k, seed)
