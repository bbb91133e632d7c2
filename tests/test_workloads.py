"""Checks of the seeded generators: sizes of the named workloads, symmetry,
positive definiteness and closed-form spectra on small instances."""
import numpy as np
import pytest

import workloads as W


def test_laplacian_64_shape_and_bounds():
    A = W.laplacian_2d_5pt(64, 64)
    assert A.n == 4096 and A.nnz == 20224
    lo, hi = W.laplacian_2d_bounds(64, 64)
    assert np.isclose(lo, 8 * np.sin(np.pi / 130) ** 2)
    assert np.isclose(hi, 8 * np.sin(64 * np.pi / 130) ** 2)
    S = W.laplacian_2d_5pt(9, 7).to_scipy().toarray()
    ev = np.linalg.eigvalsh(S)
    lo, hi = W.laplacian_2d_bounds(9, 7)
    assert np.isclose(ev[0], lo) and np.isclose(ev[-1], hi)


def test_diffusion3d_structure():
    A = W.diffusion_3d_7pt_lognormal(6, seed=1)
    assert A.nnz == 7 * 216 - 6 * 36
    S = A.to_scipy().toarray()
    assert np.array_equal(S, S.T)
    assert np.linalg.eigvalsh(S)[0] > 0
    for i in range(A.n):  # columns sorted in every row
        c = A.col[A.rowptr[i]:A.rowptr[i + 1]]
        assert np.all(np.diff(c) > 0)
    # deterministic in the seed
    B = W.diffusion_3d_7pt_lognormal(6, seed=1)
    assert np.array_equal(A.val, B.val)


def test_diffusion3d_full_size_counts():
    A = W.diffusion_3d_7pt_lognormal(128, seed=7)
    assert A.n == 2_097_152 and A.nnz == 14_581_760


def test_stencil7_bounds_exact():
    st = W.stencil7_aniso(5, 8, 3, 0.9, 0.02, 0.4)
    ev = np.linalg.eigvalsh(W.stencil7_to_csr(st).to_scipy().toarray())
    lo, hi = W.stencil7_bounds(st)
    assert np.isclose(ev[0], lo) and np.isclose(ev[-1], hi)


@pytest.mark.parametrize("N", [3, 5])
def test_elasticity_spd_and_pattern(N):
    A, b = W.elasticity_q1_bsr3(N, seed=4)
    assert A.nb == N ** 3 and A.nnzb == (3 * N - 2) ** 3
    S = A.to_scipy().toarray()
    assert np.allclose(S, S.T, atol=1e-15)
    assert np.linalg.eigvalsh(S)[0] > 0
    # clamped bottom nodes: identity rows, zero load
    for node in range(N * N):
        assert np.allclose(S[3 * node:3 * node + 3, :], np.eye(3 * N ** 3)[3 * node:3 * node + 3])
        assert np.all(b[3 * node:3 * node + 3] == 0)


def test_elasticity_rigid_translation_in_kernel():
    """Before clamping, a rigid translation produces no force on interior nodes."""
    N = 5
    A, _ = W.elasticity_q1_bsr3(N, seed=1)
    S = A.to_scipy().toarray()
    u = np.tile([0.3, -1.0, 2.0], N ** 3)
    # nodes at z >= 2 do not couple to the clamped layer z = 0
    f = S @ u
    top = np.arange(2 * N * N, N ** 3)
    for node in top:
        assert np.allclose(f[3 * node:3 * node + 3], 0, atol=1e-12)


def test_elasticity_counts_full_size_formula():
    # 100^3 nodes: 298^3 blocks = 26,463,592 (checked by formula only; the
    # full assembly runs in the GPU tests and the bench)
    assert (3 * 100 - 2) ** 3 == 26_463_592
