"""Continuous-batching request loop over the batch engine (pcg_batch_*).

Requests (matrix-free 7-point systems of any size, each with its own
right-hand side already in device memory) arrive over time.  The server
admits them first-in first-out whenever the engine has a free slot and
enough pooled memory (the HBM budget), runs a few PCG iterations of every
admitted slot per tick (one graph launch), and retires finished slots, whose
memory is then reused.  Requests that arrive while others are on the GPU join
at the next tick, so their work overlaps on the device.

The reference point is the plain method served one request at a time: a
float64 solver (stencil handle, Jacobi scaling, pcg_setup, pcg_solve) per
request, in arrival order.

Both loops use the wall clock: a request's latency is its completion time
minus its arrival time (queueing included).
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

from . import binding as nc


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    nx: int
    ny: int
    nz: int
    c: tuple                # (c0, cx, cy, cz) of the unscaled stencil
    lmin: float             # spectral bounds of the Jacobi-scaled operator
    lmax: float
    k: int
    s: float
    b: object               # torch CUDA float64 tensor (n)
    x: object = None        # solution (filled by the server)
    result: dict = field(default_factory=dict)
    t_admit: float = -1.0
    t_done: float = -1.0

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz


def _wait_until(t0: float, t: float):
    while time.perf_counter() - t0 < t:
        pass


def serve_continuous(reqs, budget_unknowns: int, max_slots: int, kmax: int, tol: float = 1e-8,
                     maxit: int = 5000, iters_per_tick: int = 2, stream=None, stats=None, f64_apply: bool = False):
    """Serve `reqs` (sorted by arrival) with continuous batching; returns the
    wall-clock span of the run.  Fills each request's x, result, t_done (the
    time its solution is in x).  `stats` (a dict, optional) receives the
    engine's iteration and kernel-launch counts.  `f64_apply` runs P_k in
    float64 (default: float32 apply, float64 outer CG)."""
    import torch
    eng = nc.pcg_batch_create(max_slots, budget_unknowns, kmax, stream, f64_apply=f64_apply)
    for r in reqs:
        if r.n > budget_unknowns:
            raise ValueError(f"request {r.rid} ({r.n} unknowns) exceeds the budget")
        if r.x is None:
            r.x = torch.empty(r.n, dtype=torch.float64, device=r.b.device)
    pending = deque(reqs)
    queue = deque()
    live = {}
    t0 = time.perf_counter()
    done = 0
    while done < len(reqs):
        now = time.perf_counter() - t0
        while pending and pending[0].arrival <= now:
            queue.append(pending.popleft())
        while queue:
            r = queue[0]
            slot = nc.pcg_batch_add(eng, r.nx, r.ny, r.nz, *r.c, r.lmin, r.lmax, r.k, r.s, r.b, stream)
            if slot is None:
                break
            r.t_admit = time.perf_counter() - t0
            live[slot] = r
            queue.popleft()
        if not live:
            if pending:
                _wait_until(t0, pending[0].arrival)
                continue
            break
        nc.pcg_batch_run(eng, tol, maxit, iters_per_tick, stream)
        finished = []
        for slot, r in live.items():
            is_done, res = nc.pcg_batch_status(eng, slot)
            if is_done:
                nc.pcg_batch_collect(eng, slot, r.x, stream)
                r.result = res
                finished.append(slot)
        if finished:
            # the collects are enqueued: a solution counts as delivered when its copy is done
            if not torch.cuda.is_available():
                pass                       # no device work to wait for
            elif stream is None:
                torch.cuda.current_stream().synchronize()
            elif hasattr(stream, "synchronize"):
                stream.synchronize()
            else:
                torch.cuda.synchronize()
            tnow = time.perf_counter() - t0
            for slot in finished:
                nc.pcg_batch_release(eng, slot, stream)
                live.pop(slot).t_done = tnow
                done += 1
    span = time.perf_counter() - t0
    if stats is not None:
        stats["iterations"], stats["launches"] = nc.pcg_batch_stats(eng)
    eng.close()
    return span


def serve_one_at_a_time_fp64(reqs, tol: float = 1e-8, maxit: int = 5000, stream=None):
    """The plain float64 method, one request at a time in arrival order."""
    import torch
    t0 = time.perf_counter()
    for r in reqs:
        now = time.perf_counter() - t0
        if now < r.arrival:
            _wait_until(t0, r.arrival)
        r.t_admit = time.perf_counter() - t0
        A = nc.nc_matrix_stencil7(r.nx, r.ny, r.nz, *r.c)
        As = nc.nc_matrix_jacobi(A)
        S = nc.pcg_setup(As, r.lmin, r.lmax, r.k, r.s, stream, x0_is_zero=True)
        if r.x is None:
            r.x = torch.empty(r.n, dtype=torch.float64, device=r.b.device)
        r.result = nc.pcg_solve(S, r.b, r.x, tol, maxit, stream)
        S.close()
        As.close()
        A.close()
        r.t_done = time.perf_counter() - t0
    return time.perf_counter() - t0
