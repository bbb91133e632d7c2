"""Continuous-batching serving loop: requests arriving while others are on
the GPU are admitted as slots and memory free up; every result matches the
plain float64 solver's within the tolerance both reach (relative residual
1e-8, so solutions agree to about kappa * 1e-8) and the admitted result is
bit-for-bit the one the engine gives the request alone."""
import math

import numpy as np
import pytest

from nchelpers import need_gpu

pytestmark = pytest.mark.gpu


def make_requests(torch, serving, n, seed):
    rng = np.random.default_rng(seed)
    out = []
    t = 0.0
    for i in range(n):
        N = int(rng.integers(12, 40))
        c = math.cos(math.pi / (N + 1))
        g = torch.Generator(device="cuda")
        g.manual_seed(seed * 100 + i)
        b = torch.rand(N ** 3, generator=g, dtype=torch.float64, device="cuda") * 2 - 1
        t += rng.exponential(0.002)
        out.append(serving.Request(rid=i, arrival=t, nx=N, ny=N, nz=N, c=(6.0, 1.0, 1.0, 1.0), lmin=1 - c,
                                   lmax=1 + c, k=int(rng.integers(8, 32)), s=1.001, b=b))
    return out


def test_serving_matches_plain_and_alone():
    torch = need_gpu()
    from paper_2008_01440_gb300 import serving
    reqs = make_requests(torch, serving, 14, seed=3)
    # a budget that holds only a few requests at a time forces queueing and reuse
    budget = 3 * max(r.n for r in reqs)
    serving.serve_continuous(reqs, budget, 8, 32, 1e-8, 3000, iters_per_tick=2)
    plain = [serving.Request(**{f: getattr(r, f) for f in ("rid", "arrival", "nx", "ny", "nz", "c", "lmin", "lmax",
                                                          "k", "s", "b")}) for r in reqs]
    serving.serve_one_at_a_time_fp64(plain, 1e-8, 3000)
    for a, p in zip(reqs, plain):
        assert a.result["status"] == 0 and p.result["status"] == 0
        assert a.result["true_relres"] <= 2e-8
        kappa = a.lmax / a.lmin
        err = float(torch.linalg.norm(a.x - p.x) / torch.linalg.norm(p.x))
        assert err <= kappa * 4e-8, (a.rid, err)
        assert a.t_done >= a.arrival
    # alone in the engine: bit-for-bit the same as in the stream
    for r in (reqs[0], reqs[7]):
        alone = serving.Request(**{f: getattr(r, f) for f in ("rid", "nx", "ny", "nz", "c", "lmin", "lmax", "k",
                                                              "s", "b")}, arrival=0.0)
        serving.serve_continuous([alone], r.n + 16, 1, 32, 1e-8, 3000, iters_per_tick=5)
        assert alone.result == r.result
        assert torch.equal(alone.x, r.x)
