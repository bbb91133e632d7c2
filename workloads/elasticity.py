"""3D linear elasticity on a structured hexahedral (Q1) mesh in 3x3-block CSR.

Stands in for the paper's finite-element structural matrices (``Cube5317k``,
``Emilia_923``, Sec. 5 and Table 2), which are not available: three
displacement dofs per node, ~80 scalar nonzeros per row.

Mesh: unit cube, N nodes per side (h = 1/(N-1)), (N-1)^3 trilinear bricks.
Material: E = 1, Poisson ratio nu_e ~ U[nu_lo, nu_hi] per element (PCG64
stream ``seed``), Lame lambda = E nu/((1+nu)(1-2nu)), mu = E/(2(1+nu)).
Element stiffness by 2x2x2 Gauss quadrature.  Nodes on the bottom face z = 0
are clamped by identity rows and columns (their couplings stay in the
pattern as explicit zeros), so the order is 3 N^3.  Load: the consistent
nodal forces of a unit downward body force, zero on clamped dofs.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class BSR3:
    """Block CSR with dense 3x3 row-major blocks: int32 block pointers/columns."""
    nb: int                # block rows (nodes); scalar order n = 3*nb
    browptr: np.ndarray    # int32, nb+1
    bcol: np.ndarray       # int32, nnzb
    val: np.ndarray        # float64, (nnzb, 3, 3)

    @property
    def n(self) -> int:
        return 3 * self.nb

    @property
    def nnzb(self) -> int:
        return int(self.browptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.bsr_matrix((self.val, self.bcol, self.browptr), shape=(self.n, self.n))


def _q1_reference_stiffness(h: float):
    """K_lambda, K_mu (24x24) of a cube brick of side h, dof = 3*corner + comp.

    Corner l = lx + 2 ly + 4 lz.  Voigt strain (xx, yy, zz, xy, yz, xz) with
    engineering shears; D = lambda m m^T + mu diag(2,2,2,1,1,1).
    """
    g = 1.0 / np.sqrt(3.0)
    corners = np.array([[lx, ly, lz] for lz in (0, 1) for ly in (0, 1) for lx in (0, 1)], float)
    sgn = 2.0 * corners - 1.0
    Kl = np.zeros((24, 24))
    Km = np.zeros((24, 24))
    m = np.array([1, 1, 1, 0, 0, 0], float)
    Dl = np.outer(m, m)
    Dm = np.diag([2.0, 2.0, 2.0, 1.0, 1.0, 1.0])
    detJ = (h / 2.0) ** 3
    for xi in (-g, g):
        for eta in (-g, g):
            for zet in (-g, g):
                p = np.array([xi, eta, zet])
                # dN/dxi_d for each corner
                fac = 1.0 + sgn * p  # (8,3)
                dN = np.zeros((8, 3))
                for d in range(3):
                    o = [k for k in range(3) if k != d]
                    dN[:, d] = sgn[:, d] * fac[:, o[0]] * fac[:, o[1]] / 8.0
                dN *= 2.0 / h
                B = np.zeros((6, 24))
                for a in range(8):
                    dx, dy, dz = dN[a]
                    c = 3 * a
                    B[0, c] = dx
                    B[1, c + 1] = dy
                    B[2, c + 2] = dz
                    B[3, c] = dy
                    B[3, c + 1] = dx
                    B[4, c + 1] = dz
                    B[4, c + 2] = dy
                    B[5, c] = dz
                    B[5, c + 2] = dx
                Kl += B.T @ Dl @ B * detJ
                Km += B.T @ Dm @ B * detJ
    return Kl, Km, corners.astype(int)


def elasticity_q1_bsr3(N: int, seed: int, nu_lo: float = 0.25, nu_hi: float = 0.45):
    """Return (BSR3 matrix, load vector b of length 3 N^3)."""
    h = 1.0 / (N - 1)
    Kl, Km, corners = _q1_reference_stiffness(h)
    ne = N - 1
    nu = np.random.Generator(np.random.PCG64(seed)).uniform(nu_lo, nu_hi, size=ne ** 3)
    lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = 1.0 / (2.0 * (1.0 + nu))
    e = np.arange(ne ** 3, dtype=np.int64)
    ex, ey, ez = e % ne, (e // ne) % ne, e // (ne * ne)
    base = ex + N * (ey + N * ez)
    nn = N ** 3
    vals = np.zeros((nn, 27, 3, 3))
    b = np.zeros((nn, 3))
    for a in range(8):
        la = corners[a]
        node_a = base + la[0] + N * la[1] + N * N * la[2]
        b[node_a, 2] -= h ** 3 / 8.0
        for c in range(8):
            lb = corners[c]
            d = lb - la
            o = (d[2] + 1) * 9 + (d[1] + 1) * 3 + (d[0] + 1)
            blk_l = Kl[3 * a:3 * a + 3, 3 * c:3 * c + 3]
            blk_m = Km[3 * a:3 * a + 3, 3 * c:3 * c + 3]
            vals[node_a, o] += lam[:, None, None] * blk_l + mu[:, None, None] * blk_m
    node = np.arange(nn, dtype=np.int64)
    ix, iy, iz = node % N, (node // N) % N, node // (N * N)
    offs = np.array([(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)])
    valid = np.ones((nn, 27), dtype=bool)
    cols = np.zeros((nn, 27), dtype=np.int64)
    for o, (dx, dy, dz) in enumerate(offs):
        valid[:, o] = ((ix + dx >= 0) & (ix + dx < N) & (iy + dy >= 0) & (iy + dy < N)
                       & (iz + dz >= 0) & (iz + dz < N))
        cols[:, o] = node + dx + N * dy + N * N * dz
    # clamp the bottom face: identity rows/columns for nodes with z = 0
    clamped = iz == 0
    vals[clamped] = 0.0
    vals[clamped, 13] = np.eye(3)
    b[clamped] = 0.0
    col_clamped = np.zeros((nn, 27), dtype=bool)
    for o, (dx, dy, dz) in enumerate(offs):
        if dz == -1:
            col_clamped[:, o] = iz == 1
    vals[col_clamped & ~clamped[:, None]] = 0.0
    counts = valid.sum(axis=1)
    browptr = np.zeros(nn + 1, dtype=np.int64)
    np.cumsum(counts, out=browptr[1:])
    A = BSR3(nb=nn, browptr=browptr.astype(np.int32), bcol=cols[valid].astype(np.int32),
             val=np.ascontiguousarray(vals[valid]))
    return A, b.ravel()
