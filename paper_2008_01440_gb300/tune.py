"""Choice of the polynomial degree k and the theta scale s for one system.

The paper leaves the optimal scale open (Sec. 6, conclusions) and the degree is a
trade-off its results show (Sec. 5): the iteration
count falls roughly like 1/k while every iteration costs k + 1 products, and
s > 1 avoids the clustering of the smallest eigenvalues of P_k(A) A (Sec. 4)
at a cost that depends on the spectrum.  This tuner measures instead of
modelling: for every candidate (k, s) it runs a short PCG probe on the
device (a seeded right-hand side, two probe lengths m1 < m2), takes

  * the time per iteration from CUDA events around the probes (their
    difference over m2 - m1 iterations, so the fixed cost of a solve drops
    out), and
  * the residual contraction per iteration over the later window,
    rho = (||r_m2|| / ||r_m1||)^(1 / (m2 - m1)),

predicts the iterations to reach `tol` as m2 + log(tol / (||r_m2||/||b||)) /
log(rho) and the solve time as their product, and returns the candidates
ranked by it.  Every product and reduction runs in the library's kernels;
this module only sequences the calls.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

from . import binding as nc


@dataclass
class Candidate:
    k: int
    s: float
    probe_iters: int
    rho: float                  # residual contraction per iteration
    ms_per_iter: float
    predicted_iters: float
    predicted_ms: float


def predict_iterations(ia: int, rel_a: float, ib: int, rel_b: float, tol: float):
    """(rho, predicted iterations to ||r||/||b|| <= tol) from two probes:
    relative residuals rel_a after ia iterations and rel_b after ib > ia.
    The contraction rho is taken over the later window; when the short probe
    already met tol, from its start instead."""
    rel_a, rel_b = max(rel_a, 1e-300), max(rel_b, 1e-300)
    if rel_a <= tol:
        rho = rel_a ** (1.0 / max(ia, 1))
        return rho, (math.log(tol) / math.log(rho) if 0.0 < rho < 1.0 else float(ia))
    rho = (rel_b / rel_a) ** (1.0 / max(ib - ia, 1))
    # the crossing of tol, from whichever probe end lies above it
    ref_i, ref_r = (ia, rel_a) if rel_b <= tol else (ib, rel_b)
    return rho, (ref_i + math.log(tol / ref_r) / math.log(rho) if 0.0 < rho < 1.0 else math.inf)


def tune_degree(A, lmin: float, lmax: float, degrees=(0, 2, 4, 8, 12, 16, 20, 30, 40),
                scales=(1.0, 1.001, 1.01), tol: float = 1e-8, probe_iters: int = 8, apply_dtype: str = "f64",
                seed: int = 17, stream=None) -> list:
    """Rank (k, s) candidates for solving with matrix handle `A` (bounds of
    the operator P is applied to).  Returns a list of Candidate, fastest
    predicted first."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    b = torch.rand(A.n, generator=g, dtype=torch.float64, device="cuda") * 2.0 - 1.0
    x = torch.zeros_like(b)
    st = torch.cuda.current_stream() if stream is None else stream
    m1, m2 = max(1, probe_iters // 4), max(probe_iters, 2)
    out = []

    def timed(S, iters):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        res = nc.pcg_solve(S, b, x, 0.0, iters, stream=stream)
        e1.record(st)
        torch.cuda.synchronize()
        return res, e0.elapsed_time(e1)

    for k in degrees:
        for s in scales:
            if k == 0 and s != scales[0]:
                continue          # P = 1/theta': the scale does not change the iterates
            S = nc.pcg_setup(A, lmin, lmax, k, s, apply_dtype=apply_dtype, x0_is_zero=True, stream=stream)
            try:
                timed(S, 1)                                        # build the graph, warm up
                ra, ta = timed(S, m1)
                rb, tb = timed(S, m2)
            finally:
                S.close()
            ia, ib = ra["iters"], rb["iters"]
            ms = (tb - ta) / max(ib - ia, 1)
            rho, pred = predict_iterations(ia, ra["relres"], ib, rb["relres"], tol)
            out.append(Candidate(k, s, ib, rho, ms, pred, pred * ms))
    out.sort(key=lambda c: c.predicted_ms)
    return out
