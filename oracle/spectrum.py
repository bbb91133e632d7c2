"""Eigenvalue statistics of the preconditioned matrix P_m(A) A (paper Sec. 4).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

For a matrix with eigenvalues lambda_s the preconditioned matrix p_m(A) A
has eigenvalues y_s = lambda_s p_m(lambda_s) (Sec. 4, the reading of Fig. 2).
Table 3 reports mu_max, mu_min, the condition number and the clustering
indicator l = #{lambda : lambda/lambda_min < 1.1} (Eq. lmin).
"""
from __future__ import annotations

import numpy as np

from .chebyshev import ChebParams, p_k_recurrence


def preconditioned_spectrum_stats(lam: np.ndarray, prm: ChebParams, m: int):
    """Return dict(mu_max, mu_min, l, kappa) for eigenvalues lam of A."""
    mu = lam * p_k_recurrence(lam, prm, m)
    mu_min = float(mu.min())
    mu_max = float(mu.max())
    return dict(mu_max=mu_max, mu_min=mu_min,
                l=int(np.count_nonzero(mu / mu_min < 1.1)),
                kappa=mu_max / mu_min)
