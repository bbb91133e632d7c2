"""Degree / scale tuner (paper Sec. 6 leaves the optimal k and s open): its
iteration predictions against full solves, and a sensible choice on a system
where high degree pays (the 3D diffusion operator, kappa ~ 10^3)."""
import math

import pytest

import workloads as W
from nchelpers import csr_to_gpu, need_gpu, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    import paper_2008_01440_gb300 as nc
    from paper_2008_01440_gb300 import tune
    return torch, nc, tune


def test_tuner_predictions_and_choice(env):
    torch, nc, tune = env
    A = W.diffusion_3d_7pt_lognormal(32, seed=11)
    M = nc.nc_matrix_jacobi(csr_to_gpu(torch, nc, A))
    lo, hi, _, _ = nc.nc_bounds_lanczos(M, 20, to_dev(torch, W.uniform_vector(A.n, seed=3)))
    cands = tune.tune_degree(M, lo, hi, degrees=(0, 4, 12, 24), scales=(1.0, 1.001), tol=1e-8, probe_iters=12)
    assert len(cands) == 1 + 3 * 2
    assert all(c1.predicted_ms <= c2.predicted_ms for c1, c2 in zip(cands, cands[1:]))
    g = torch.Generator(device="cuda")
    g.manual_seed(17)
    b = torch.rand(A.n, generator=g, dtype=torch.float64, device="cuda") * 2 - 1
    for c in cands:
        S = nc.pcg_setup(M, lo, hi, c.k, c.s, x0_is_zero=True)
        x = torch.zeros_like(b)
        it = nc.pcg_solve(S, b, x, 1e-8, 5000)["iters"]
        assert math.isfinite(c.predicted_iters)
        assert abs(c.predicted_iters - it) <= max(3, 0.3 * it), (c.k, c.s, c.predicted_iters, it)
    # unpreconditioned-in-effect k = 0 is not the fastest on this spectrum
    assert cands[0].k > 0
