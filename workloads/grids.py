"""Finite-difference test operators and seeded vectors.

Grid ordering everywhere: the unknown at grid point (i, j, k) (0-based,
i fastest) has index ``i + nx*(j + ny*k)``.  Dirichlet boundaries: points
outside the grid carry value zero and are not unknowns.

The paper's workloads these stand in for:
  * 2D 5-point Laplacian on the unit square with exactly known eigenvalues
    (Sec. 4, Fig. 2 and Table 3; ``Lap1600`` of Table 2),
  * 3D 7-point finite-difference Poisson operator in the unit cube
    (Sec. 5.3, Tables 7 and 8), here also with per-cell log-normal
    diffusion coefficients and per-axis (anisotropic) weights.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    """Compressed sparse row matrix: int32 row pointers / columns, f64 values.

    Columns inside each row are sorted ascending.
    """
    n: int
    rowptr: np.ndarray  # int32, length n+1
    col: np.ndarray     # int32, length nnz
    val: np.ndarray     # float64, length nnz

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))


@dataclass
class Stencil7:
    """Matrix-free constant-coefficient 7-point operator on an nx*ny*nz grid.

    (A u)_p = c0*u_p - cx*(u_{p-ex}+u_{p+ex}) - cy*(u_{p-ey}+u_{p+ey})
                     - cz*(u_{p-ez}+u_{p+ez}),  zero outside the grid.
    """
    nx: int
    ny: int
    nz: int
    c0: float
    cx: float
    cy: float
    cz: float

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_vector(n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """n float64 draws uniform on [lo, hi) from numpy's PCG64 stream ``seed``."""
    return _rng(seed).uniform(lo, hi, size=n)


def _grid_csr(shape_zyx, diag, face):
    """CSR for a 2D/3D nearest-neighbour operator.

    ``diag``: array (shape) with the diagonal.
    ``face[a]``: array (shape) with the coupling between point p and its
    +axis-a neighbour (a = 0: x, 1: y, 2: z); the entry A[p, p+e_a] =
    A[p+e_a, p] = -face[a][p].  Values for the last layer along axis a are
    ignored (no neighbour).
    """
    nz, ny, nx = shape_zyx
    n = nx * ny * nz
    strides = (1, nx, nx * ny)
    dims = (nx, ny, nz)
    # per point: slots ordered by column offset: -z, -y, -x, 0, +x, +y, +z
    vals = np.zeros((n, 7))
    cols = np.zeros((n, 7), dtype=np.int64)
    mask = np.zeros((n, 7), dtype=bool)
    idx = np.arange(n, dtype=np.int64)
    coord = [idx % nx, (idx // nx) % ny, idx // (nx * ny)]
    vals[:, 3] = diag.ravel()
    cols[:, 3] = idx
    mask[:, 3] = True
    for a in range(3):
        if dims[a] == 1:
            continue
        f = face[a].ravel()
        # + neighbour (slot 4+a)
        has_p = coord[a] < dims[a] - 1
        cols[:, 4 + a] = idx + strides[a]
        vals[:, 4 + a] = -f
        mask[:, 4 + a] = has_p
        # - neighbour (slot 2-a): coupling stored at the neighbour p - e_a
        has_m = coord[a] > 0
        src = np.where(has_m, idx - strides[a], 0)
        cols[:, 2 - a] = idx - strides[a]
        vals[:, 2 - a] = -f[src]
        mask[:, 2 - a] = has_m
    counts = mask.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2**31:
        raise ValueError("nnz exceeds int32 range")
    return CSR(n=n, rowptr=rowptr.astype(np.int32), col=cols[mask].astype(np.int32),
               val=np.ascontiguousarray(vals[mask]))


def laplacian_1d(n: int) -> CSR:
    """Tridiagonal [-1, 2, -1] of order n (Dirichlet)."""
    shape = (1, 1, n)
    diag = np.full(shape, 2.0)
    face = [np.ones(shape), np.zeros(shape), np.zeros(shape)]
    return _grid_csr(shape, diag, face)


def laplacian_2d_5pt(nx: int, ny: int) -> CSR:
    """5-point Laplacian [4 on the diagonal, -1 to each grid neighbour]."""
    shape = (1, ny, nx)
    diag = np.full(shape, 4.0)
    face = [np.ones(shape), np.ones(shape), np.zeros(shape)]
    return _grid_csr(shape, diag, face)


def laplacian_2d_bounds(nx: int, ny: int):
    """Exact extreme eigenvalues of ``laplacian_2d_5pt(nx, ny)``.

    The eigenvalues are 4 sin^2(i pi/(2(nx+1))) + 4 sin^2(j pi/(2(ny+1))),
    i = 1..nx, j = 1..ny (separable sine eigenvectors).
    """
    s = lambda i, m: 4.0 * np.sin(i * np.pi / (2.0 * (m + 1))) ** 2  # noqa: E731
    return s(1, nx) + s(1, ny), s(nx, nx) + s(ny, ny)


def diffusion_3d_7pt_lognormal(N: int, seed: int, sigma: float = 1.0) -> CSR:
    """3D 7-point variable-coefficient diffusion on an N^3 grid.

    Per-grid-point coefficient kappa = exp(sigma * N(0,1)) (numpy PCG64
    stream ``seed``).  The coupling across the face between neighbours a, b is
    the harmonic mean 2 k_a k_b / (k_a + k_b).  At the Dirichlet boundary the
    outward face carries the point's own kappa.  The diagonal is the sum of
    the six face couplings, so the matrix is a symmetric M-matrix, strictly
    diagonally dominant on boundary rows: SPD.
    """
    shape = (N, N, N)
    kap = np.exp(sigma * _rng(seed).standard_normal(size=shape))
    diag = np.zeros(shape)
    face = []
    for a in range(3):
        ax = 2 - a  # array axis of grid axis a (arrays are [z, y, x])
        nb = np.roll(kap, -1, axis=ax)
        h = 2.0 * kap * nb / (kap + nb)
        last = [slice(None)] * 3
        last[ax] = slice(N - 1, N)
        h[tuple(last)] = 0.0
        face.append(h)
        # interior faces contribute to both endpoints' diagonals
        diag += h
        diag += np.roll(h, 1, axis=ax)
        # boundary faces (Dirichlet): own kappa on the two outer layers
        first = [slice(None)] * 3
        first[ax] = slice(0, 1)
        diag[tuple(first)] += kap[tuple(first)]
        diag[tuple(last)] += kap[tuple(last)]
    return _grid_csr(shape, diag, face)


def stencil7_aniso(nx: int, ny: int, nz: int, wx: float, wy: float, wz: float) -> Stencil7:
    """Anisotropic Laplacian: weights w_a on axis a, diagonal 2(wx+wy+wz)."""
    return Stencil7(nx, ny, nz, 2.0 * (wx + wy + wz), wx, wy, wz)


def stencil7_bounds(st: Stencil7):
    """Exact extreme eigenvalues of a constant-coefficient 7-point operator.

    Eigenvalues: c0 - 2 sum_a c_a cos(i_a pi/(n_a+1)), i_a = 1..n_a, for
    c_a >= 0 (separable sine eigenvectors).  Axes of extent 1 contribute 0.
    """
    t = 0.0
    for n_a, c_a in ((st.nx, st.cx), (st.ny, st.cy), (st.nz, st.cz)):
        if n_a > 1:
            t += 2.0 * c_a * np.cos(np.pi / (n_a + 1))
    return st.c0 - t, st.c0 + t


def stencil7_to_csr(st: Stencil7) -> CSR:
    """Explicit CSR form of a constant-coefficient 7-point operator."""
    shape = (st.nz, st.ny, st.nx)
    diag = np.full(shape, float(st.c0))
    face = [np.full(shape, float(st.cx)), np.full(shape, float(st.cy)), np.full(shape, float(st.cz))]
    return _grid_csr(shape, diag, face)


def rhs_from_solution(A: CSR, xstar: np.ndarray) -> np.ndarray:
    """Right-hand side b = A x* for a manufactured solution x*."""
    return A.to_scipy() @ xstar
