"""Pins for the oracle's two-level (block-Jacobi first level) factorisation:
the scaled operator W^T A W against a dense evaluation, its unit diagonal
blocks, P_0 = W W^T = blockdiag(A_ii^{-1}), the reduction to scalar Jacobi
when the diagonal blocks are diagonal, and a two-level PCG solve against a
dense Cholesky solve."""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
import workloads as W


def dense(browptr, bcol, val, nb):
    A = np.zeros((3 * nb, 3 * nb))
    for i in range(nb):
        for e in range(browptr[i], browptr[i + 1]):
            j = bcol[e]
            A[3 * i:3 * i + 3, 3 * j:3 * j + 3] = val[e]
    return A


def blockdiag(B):
    return sla.block_diag(*B)


@pytest.fixture(scope="module")
def small():
    A, b = W.elasticity_q1_bsr3(4, seed=3)
    return A, b


def test_scaled_operator_matches_dense(small):
    A, _ = small
    S, Wb, Lb = O.block_jacobi_factor_bsr3(A.browptr, A.bcol, A.val, A.nb)
    Ad = dense(A.browptr, A.bcol, A.val, A.nb)
    Wd = blockdiag(Wb)
    ref = Wd.T @ Ad @ Wd
    got = dense(A.browptr, A.bcol, S, A.nb)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert np.max(np.abs(got - got.T)) <= 1e-12
    for i in range(A.nb):
        assert np.max(np.abs(got[3 * i:3 * i + 3, 3 * i:3 * i + 3] - np.eye(3))) <= 1e-13
    # P_0 = W W^T is the block-Jacobi preconditioner, L the Cholesky factor
    Dinv = blockdiag([np.linalg.inv(Ad[3 * i:3 * i + 3, 3 * i:3 * i + 3]) for i in range(A.nb)])
    assert np.max(np.abs(Wd @ Wd.T - Dinv)) <= 1e-12 * np.max(np.abs(Dinv))
    Ld = blockdiag(Lb)
    assert np.max(np.abs(Ld @ Ld.T - blockdiag([Ad[3 * i:3 * i + 3, 3 * i:3 * i + 3] for i in range(A.nb)]))) \
        <= 1e-12 * np.max(np.abs(Ad))


def test_diagonal_blocks_reduce_to_scalar_jacobi(small):
    A, _ = small
    val = A.val.copy()
    brows = np.repeat(np.arange(A.nb), np.diff(A.browptr))
    on = brows == A.bcol
    val[on] = val[on] * np.eye(3)[None]            # keep only the diagonal of the diagonal blocks
    S, Wb, _ = O.block_jacobi_factor_bsr3(A.browptr, A.bcol, val, A.nb)
    Sj, dis = O.jacobi_scale_bsr3(A.browptr, A.bcol, val, A.nb)
    assert np.max(np.abs(S - Sj)) <= 1e-13 * np.max(np.abs(Sj))
    assert np.allclose(np.einsum("bii->bi", Wb).ravel(), dis, rtol=1e-14, atol=0)


def test_two_level_pcg_solves_original_system(small):
    A, b = small
    S, Wb, Lb = O.block_jacobi_factor_bsr3(A.browptr, A.bcol, A.val, A.nb)
    mv = O.bsr3_matvec(A.browptr, A.bcol, S, A.nb)
    Wd = blockdiag(Wb)
    ev = np.linalg.eigvalsh(dense(A.browptr, A.bcol, S, A.nb))
    prm = O.cheb_params(ev[0], ev[-1], 1.001)
    res = O.pcg(mv, Wd.T @ b, lambda r: O.cheb_apply(mv, r, prm, 8), m=8, tol=1e-12, maxit=500)
    x = Wd @ res.x
    xs = sla.cho_solve(sla.cho_factor(dense(A.browptr, A.bcol, A.val, A.nb)), b)
    assert res.status == 0
    assert np.linalg.norm(x - xs) <= 1e-9 * np.linalg.norm(xs)


def test_indefinite_diagonal_block_raises(small):
    A, _ = small
    val = A.val.copy()
    brows = np.repeat(np.arange(A.nb), np.diff(A.browptr))
    first_diag = np.nonzero(brows == A.bcol)[0][0]
    val[first_diag] = -np.eye(3)
    with pytest.raises(np.linalg.LinAlgError):
        O.block_jacobi_factor_bsr3(A.browptr, A.bcol, val, A.nb)
