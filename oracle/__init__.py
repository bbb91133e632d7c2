"""FP64 CPU oracle for Newton-Chebyshev polynomial-preconditioned CG.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously
correct restatement of the paper (Bergamaschi & Martinez, "Parallel
Newton-Chebyshev Polynomial Preconditioners for the Conjugate Gradient
method") that the CUDA library is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it.  It shares no code with the CUDA path (``paper_2008_01440_gb300``)
and imports nothing from it; both sides take their inputs from the seeded
generators in ``workloads``.

Everything is float64 numpy; a scipy sparse matrix-vector product serves as
the matrix-vector step.  Each function cites the passage it follows.

Modules
  chebyshev  -- Sec. 3: interval parameters, rho recurrence, the p_k
                recurrence, the closed form via T_{k+1}, Algorithm 2.
  newton     -- Sec. 2: zeta coefficients (Eq. zetaNewt / Algorithm 1),
                recursive apply (Algorithm 1), dense Hotelling iteration.
  operators  -- matrix-vector products (CSR, 3x3 BSR, 7-point stencil) and
                the symmetric diagonal scaling of Sec. 2 / Sec. 5.
  lanczos    -- extreme-eigenvalue estimates (Lanczos, power method).
  pcg        -- PCG with the three dot products per iteration of Table 4.
  spectrum   -- eigenvalue statistics of P_k(A)A used in Sec. 4 (Table 3).

Parity status of every function is recorded in its docstring; all are
pinned by ``tests/test_oracle_*.py`` except where a docstring says
"parity unpinned".
"""
from .chebyshev import (  # noqa: F401
    ChebParams,
    cheb_params,
    rho_sequence,
    p_k_recurrence,
    p_k_closed_form,
    cheb_apply,
)
from .newton import newton_zetas, newton_apply, hotelling_dense  # noqa: F401
from .operators import (  # noqa: F401
    csr_matvec,
    bsr3_matvec,
    stencil7_matvec,
    jacobi_scale_csr,
    jacobi_scale_bsr3,
    block_jacobi_factor_bsr3,
    jacobi_scale_stencil7,
)
from .lanczos import lanczos_bounds, power_method  # noqa: F401
from .pcg import PCGResult, pcg  # noqa: F401
from .spectrum import preconditioned_spectrum_stats  # noqa: F401
