"""Preconditioned Conjugate Gradient with operation counters.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper runs standard PCG accelerated by P_m (Algorithm 1 step 4, Sec. 5.1)
and counts three dot products per iteration and (m+1) matrix-vector products
per iteration (Table 4: ddot = 3 iter, A x v = (m+1) iter).  Stopping test:
relative residual norm ||r_i|| / ||b|| below tol (Sec. 5: tol = 1e-8), with
r_i the recurrence residual.  x0 = 0 unless given.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

OK, MAXIT, INDEFINITE = 0, 1, 2


@dataclass
class PCGResult:
    x: np.ndarray
    iters: int
    status: int            # OK / MAXIT / INDEFINITE
    relres: float          # ||r_i|| / ||b||, recurrence residual
    true_relres: float     # ||b - A x|| / ||b||
    n_dot: int             # dot products (||b|| not counted, as in Table 4)
    n_matvec: int          # A p products, plus m per preconditioner call
    n_precond: int
    history: list = field(default_factory=list)


def pcg(matvec, b: np.ndarray, precond=None, m: int = 0, x0=None, tol: float = 1e-8,
        maxit: int = 10000, rr_period: int = 0) -> PCGResult:
    """Solve A x = b by PCG with preconditioner z = precond(r).

    ``rr_period`` > 0: after every rr_period-th iteration that does not stop,
    the recurrence residual is replaced by the true residual b - A x (the
    search direction is kept).  This is not part of the paper's method; in
    exact arithmetic it changes nothing, which is what pins it.

    ``m`` is the number of matrix-vector products one preconditioner call
    costs (the degree of P_m), used only for the counters.

    Per iteration: q = A p; alpha = (r, z)/(p, q)  [dot 1];
    x += alpha p; r -= alpha q; ||r||^2            [dot 2];
    stop if ||r|| <= tol ||b||;
    z = P r; beta = (r, z)_new/(r, z)_old           [dot 3]; p = z + beta p.
    """
    if precond is None:
        precond = lambda r: r.copy()  # noqa: E731
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = float(np.linalg.norm(b))
    r = b - matvec(x) if x0 is not None else b.copy()
    n_dot = n_mv = n_pc = 0
    hist = []
    if bnorm == 0.0 or float(np.linalg.norm(r)) <= tol * bnorm:
        return PCGResult(x, 0, OK, 0.0 if bnorm == 0.0 else float(np.linalg.norm(r)) / bnorm,
                         0.0 if bnorm == 0.0 else float(np.linalg.norm(b - matvec(x))) / bnorm,
                         0, 0, 0, hist)
    z = precond(r)
    n_pc += 1
    n_mv += m
    rz = float(np.dot(r, z))
    n_dot += 1
    if not rz > 0.0:
        return PCGResult(x, 0, INDEFINITE, 1.0, 1.0, n_dot, n_mv, n_pc, hist)
    p = z.copy()
    it = 0
    status = MAXIT
    relres = float(np.linalg.norm(r)) / bnorm
    while it < maxit:
        q = matvec(p)
        n_mv += 1
        pq = float(np.dot(p, q))
        n_dot += 1
        if not pq > 0.0:
            status = INDEFINITE
            break
        alpha = rz / pq
        x = x + alpha * p
        r = r - alpha * q
        rr = float(np.dot(r, r))
        n_dot += 1
        it += 1
        relres = np.sqrt(rr) / bnorm
        hist.append(relres)
        if np.sqrt(rr) <= tol * bnorm:
            status = OK
            break
        if it >= maxit:
            break
        if rr_period > 0 and it % rr_period == 0:
            r = b - matvec(x)
        z = precond(r)
        n_pc += 1
        n_mv += m
        rz_new = float(np.dot(r, z))
        n_dot += 1
        if not rz_new > 0.0:
            status = INDEFINITE
            break
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    true_relres = float(np.linalg.norm(b - matvec(x))) / bnorm
    return PCGResult(x, it, status, float(relres), true_relres, n_dot, n_mv, n_pc, hist)
