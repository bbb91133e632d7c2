"""Seeded synthetic workloads shared as *data* by the CUDA path and the oracle.

This package holds no arithmetic of the preconditioned CG method (no scaling,
no polynomial, no Krylov step).  It only builds test matrices and vectors with
the shapes and structure of the paper's workloads (2D/3D finite-difference
Laplacians, Sec. 4 and Sec. 5.3; finite-element elasticity, Sec. 5) and their
closed-form extreme eigenvalues where such a formula exists.

Every generator is deterministic in its ``seed`` (numpy PCG64 stream).
"""
from .grids import (  # noqa: F401
    CSR,
    Stencil7,
    laplacian_2d_5pt,
    laplacian_2d_bounds,
    laplacian_1d,
    diffusion_3d_7pt_lognormal,
    stencil7_aniso,
    stencil7_bounds,
    stencil7_to_csr,
    uniform_vector,
    rhs_from_solution,
)
from .elasticity import BSR3, elasticity_q1_bsr3  # noqa: F401
