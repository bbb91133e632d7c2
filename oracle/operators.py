"""Matrix-vector products and symmetric diagonal scaling, float64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper needs only the action v -> A v (Sec. 1: polynomial preconditioners
work "matrix-free"), with A symmetrically scaled by its diagonal,
A = D^{-1/2} A_hat D^{-1/2} (Sec. 2, end; Sec. 5: "all matrices are
preliminary diagonally scaled").
"""
from __future__ import annotations

import numpy as np


def csr_matvec(rowptr, col, val, n):
    """Return v -> A v for a CSR matrix (scipy's sparse product as the step)."""
    import scipy.sparse as sp
    M = sp.csr_matrix((val, col, rowptr), shape=(n, n))
    return lambda v: M @ v


def bsr3_matvec(browptr, bcol, val, nb):
    """Return v -> A v for 3x3-block CSR with row-major blocks val[b, r, c]."""
    import scipy.sparse as sp
    M = sp.bsr_matrix((val, bcol, browptr), shape=(3 * nb, 3 * nb))
    return lambda v: M @ v


def stencil7_matvec(nx, ny, nz, c0, cx, cy, cz):
    """Return u -> A u for the constant 7-point stencil with zero Dirichlet halo.

    (A u)_p = c0 u_p - cx (u_{p-ex} + u_{p+ex}) - cy (...) - cz (...),
    unknown (i, j, k) at index i + nx (j + ny k).  Written directly from that
    definition on a zero-padded copy of the grid.
    """
    def mv(u):
        g = np.zeros((nz + 2, ny + 2, nx + 2))
        g[1:-1, 1:-1, 1:-1] = u.reshape(nz, ny, nx)
        c = g[1:-1, 1:-1, 1:-1]
        y = (c0 * c
             - cx * (g[1:-1, 1:-1, :-2] + g[1:-1, 1:-1, 2:])
             - cy * (g[1:-1, :-2, 1:-1] + g[1:-1, 2:, 1:-1])
             - cz * (g[:-2, 1:-1, 1:-1] + g[2:, 1:-1, 1:-1]))
        return y.ravel()
    return mv


def jacobi_scale_csr(rowptr, col, val, n):
    """A = D^{-1/2} A_hat D^{-1/2} for CSR; returns (scaled values, d^{-1/2}).

    a_ij -> a_ij / sqrt(a_ii a_jj).  The solution of A_hat x = b is
    x = D^{-1/2} y where A y = D^{-1/2} b.
    """
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    diag = np.zeros(n)
    on_diag = rows == col
    diag[rows[on_diag]] = val[on_diag]
    if np.any(diag <= 0.0):
        raise ValueError("diagonal scaling needs a positive diagonal")
    dis = 1.0 / np.sqrt(diag)
    return val * dis[rows] * dis[col], dis


def jacobi_scale_bsr3(browptr, bcol, val, nb):
    """Scalar diagonal scaling of a 3x3-block matrix; returns (values, d^{-1/2})."""
    brows = np.repeat(np.arange(nb), np.diff(browptr))
    diag = np.zeros(3 * nb)
    on_diag = brows == bcol
    for c in range(3):
        diag[3 * brows[on_diag] + c] = val[on_diag, c, c]
    if np.any(diag <= 0.0):
        raise ValueError("diagonal scaling needs a positive diagonal")
    dis = 1.0 / np.sqrt(diag)
    rs = dis[3 * brows[:, None] + np.arange(3)[None, :]]   # (nnzb, 3) row scales
    cs = dis[3 * bcol[:, None] + np.arange(3)[None, :]]    # (nnzb, 3) column scales
    return val * rs[:, :, None] * cs[:, None, :], dis


def block_jacobi_factor_bsr3(browptr, bcol, val, nb):
    """Two-level preconditioner of the paper's conclusions (Sec. 6): a first
    level in factored form P_0 = W W^T, here block Jacobi with
    W = blockdiag(L_i^{-T}), A_ii = L_i L_i^T the Cholesky factor of each 3x3
    diagonal block, and the Newton-Chebyshev polynomial applied to W^T A W.

    Returns (scaled values of W^T A W in the same block pattern, W blocks
    (nb, 3, 3), L blocks (nb, 3, 3)); the scaled system is
    (W^T A W) y = W^T b with x = W y.  numpy's Cholesky and triangular
    inverse per block; raises if a diagonal block is not positive definite.
    """
    brows = np.repeat(np.arange(nb), np.diff(browptr))
    on_diag = brows == bcol
    if np.count_nonzero(on_diag) != nb:
        raise ValueError("every block row needs its diagonal block")
    D = np.empty((nb, 3, 3))
    D[brows[on_diag]] = val[on_diag]
    L = np.linalg.cholesky(D)                      # raises LinAlgError if not SPD
    W = np.transpose(np.linalg.inv(L), (0, 2, 1))  # L^{-T}
    scaled = np.einsum("bki,bkl,blj->bij", W[brows], val, W[bcol])
    return scaled, W, L


def jacobi_scale_stencil7(c0, cx, cy, cz):
    """Constant diagonal c0: the scaled stencil is (1, cx/c0, cy/c0, cz/c0)."""
    if c0 <= 0.0:
        raise ValueError("diagonal scaling needs a positive diagonal")
    return 1.0, cx / c0, cy / c0, cz / c0
