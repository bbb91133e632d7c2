"""Batched / continuous-batching engine (one graph launch advances every slot).

Each slot: an anisotropic 7-point Laplacian (Jacobi scaled inside the engine),
exact bounds of the scaled operator, its own degree; float32 P_k with a
float64 outer CG.  Checked against the float64 oracle, and for identity:
a slot's result must be bit-for-bit the same alone and in any mix, whenever
it was admitted.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from nchelpers import need_gpu, rel_err, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    import paper_2008_01440_gb300 as nc
    return torch, nc


def systems(count, seed, side_lo=8, side_hi=40):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        nx, ny, nz = (int(v) for v in rng.integers(side_lo, side_hi + 1, 3))
        wx, wy, wz = rng.uniform(0.01, 1.0, 3)
        st = W.stencil7_aniso(nx, ny, nz, wx, wy, wz)
        k = int(rng.integers(8, 33))
        b = W.uniform_vector(st.n, seed=seed * 1000 + i)
        out.append((st, k, b))
    return out


def scaled_bounds(st):
    sc = W.Stencil7(st.nx, st.ny, st.nz, *O.jacobi_scale_stencil7(st.c0, st.cx, st.cy, st.cz))
    return sc, W.stencil7_bounds(sc)


def add(nc, torch, B, st, k, b):
    sc, (lo, hi) = scaled_bounds(st)
    return nc.pcg_batch_add(B, st.nx, st.ny, st.nz, st.c0, st.cx, st.cy, st.cz, lo, hi, k, 1.001, to_dev(torch, b))


def collect(nc, torch, B, slot, n):
    done, res = nc.pcg_batch_status(B, slot)
    assert done
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    nc.pcg_batch_collect(B, slot, x)
    return res, x.cpu().numpy()


@pytest.mark.parametrize("f64", [False, True])
def test_batch_matches_oracle(env, f64):
    """float32 apply (default) and float64 apply (NC_BATCH_F64_APPLY): the
    oracle's iteration count within 10 % / +-1."""
    torch, nc = env
    sy = systems(12, seed=1)
    B = nc.pcg_batch_create(32, sum(s.n for s, _, _ in sy) + 1000, 32, f64_apply=f64)
    slots = [add(nc, torch, B, st, k, b) for st, k, b in sy]
    assert all(s is not None for s in slots)
    left = nc.pcg_batch_run(B, 1e-8, 3000)
    assert left == 0
    for (st, k, b), s in zip(sy, slots):
        res, x = collect(nc, torch, B, s, st.n)
        sc, (lo, hi) = scaled_bounds(st)
        mv = O.stencil7_matvec(sc.nx, sc.ny, sc.nz, sc.c0, sc.cx, sc.cy, sc.cz)
        d = 1.0 / np.sqrt(st.c0)
        ro = O.pcg(mv, d * b, lambda r: O.cheb_apply(mv, r, O.cheb_params(lo, hi, 1.001), k), m=k, tol=1e-8)
        assert res["status"] == 0 and res["true_relres"] <= 2e-8
        slack = 1 if f64 else max(2, 0.1 * ro.iters)
        assert abs(res["iters"] - ro.iters) <= slack, (res["iters"], ro.iters)
        assert res["n_dot"] == 3 * res["iters"]
        assert rel_err(x, d * ro.x) <= (hi / lo) * 2e-8


def test_batch_result_independent_of_mix(env):
    """Bit-for-bit identity: a system alone, in a mix, and admitted while
    other slots are mid-solve (continuous batching)."""
    torch, nc = env
    sy = systems(10, seed=2)
    probe = sy[3]
    # alone
    B1 = nc.pcg_batch_create(4, probe[0].n + 10, 32)
    s = add(nc, torch, B1, *probe)
    nc.pcg_batch_run(B1, 1e-8, 3000)
    res_a, x_a = collect(nc, torch, B1, s, probe[0].n)
    # in a mix, all admitted together
    B2 = nc.pcg_batch_create(16, sum(t[0].n for t in sy) + 10, 32)
    slots = [add(nc, torch, B2, *t) for t in sy]
    nc.pcg_batch_run(B2, 1e-8, 3000)
    res_b, x_b = collect(nc, torch, B2, slots[3], probe[0].n)
    assert res_a == res_b and np.array_equal(x_a, x_b)
    # continuous batching: half admitted, a few iterations, then the rest
    B3 = nc.pcg_batch_create(16, sum(t[0].n for t in sy) + 10, 32)
    first = [add(nc, torch, B3, *t) for i, t in enumerate(sy) if i % 2 == 0]
    nc.pcg_batch_run(B3, 1e-8, 3000, iter_limit=5)
    later = {i: add(nc, torch, B3, *t) for i, t in enumerate(sy) if i % 2 == 1}
    ticks = 0
    while nc.pcg_batch_run(B3, 1e-8, 3000, iter_limit=3) > 0:
        ticks += 1
        assert ticks < 1000
    res_c, x_c = collect(nc, torch, B3, later[3], probe[0].n)
    assert res_a == res_c and np.array_equal(x_a, x_c)
    assert len(first) == 5


def test_batch_admission_and_release(env):
    torch, nc = env
    sy = systems(3, seed=3, side_lo=20, side_hi=24)
    cap = sy[0][0].n + sy[1][0].n   # room for the first two only
    B = nc.pcg_batch_create(8, cap, 32)
    s0 = add(nc, torch, B, *sy[0])
    s1 = add(nc, torch, B, *sy[1])
    assert s0 is not None and s1 is not None
    if sy[2][0].n > 0:
        assert add(nc, torch, B, *sy[2]) is None          # refused: pool full
    nc.pcg_batch_run(B, 1e-8, 3000)
    collect(nc, torch, B, s0, sy[0][0].n)
    nc.pcg_batch_release(B, s0)
    lg, tot = nc.pcg_batch_free_units(B)
    assert lg >= sy[0][0].n
    if sy[2][0].n <= lg:
        s2 = add(nc, torch, B, *sy[2])
        assert s2 is not None
        nc.pcg_batch_run(B, 1e-8, 3000)
        res, _ = collect(nc, torch, B, s2, sy[2][0].n)
        assert res["status"] == 0


def test_batch_zero_rhs_and_maxit(env):
    torch, nc = env
    st = W.stencil7_aniso(10, 12, 9, 0.5, 0.2, 0.9)
    sc, (lo, hi) = scaled_bounds(st)
    B = nc.pcg_batch_create(4, 3 * st.n, 32)
    s0 = nc.pcg_batch_add(B, st.nx, st.ny, st.nz, st.c0, st.cx, st.cy, st.cz, lo, hi, 12, 1.001,
                          torch.zeros(st.n, dtype=torch.float64, device="cuda"))
    s1 = nc.pcg_batch_add(B, st.nx, st.ny, st.nz, st.c0, st.cx, st.cy, st.cz, lo, hi, 12, 1.001,
                          to_dev(torch, W.uniform_vector(st.n, seed=1)))
    nc.pcg_batch_run(B, 1e-14, 2)
    r0, x0 = collect(nc, torch, B, s0, st.n)
    assert r0["status"] == 0 and r0["iters"] == 0 and np.all(x0 == 0)
    r1, _ = collect(nc, torch, B, s1, st.n)
    assert r1["status"] == nc.NC_ERR_MAXIT and r1["iters"] == 2


def test_batch_f64_apply_identity(env):
    """float64 apply: a slot's result is bit-for-bit the same alone and in a mix."""
    torch, nc = env
    sy = systems(6, seed=8)
    probe = sy[2]
    B1 = nc.pcg_batch_create(4, probe[0].n + 10, 32, f64_apply=True)
    s = add(nc, torch, B1, *probe)
    nc.pcg_batch_run(B1, 1e-8, 3000)
    ra, xa = collect(nc, torch, B1, s, probe[0].n)
    B2 = nc.pcg_batch_create(8, sum(t[0].n for t in sy) + 10, 32, f64_apply=True)
    slots = [add(nc, torch, B2, *t) for t in sy]
    nc.pcg_batch_run(B2, 1e-8, 3000)
    rb, xb = collect(nc, torch, B2, slots[2], probe[0].n)
    assert ra == rb and np.array_equal(xa, xb)


def test_batch_host_loop_identical(env):
    """The host-driven loop (for profilers) runs the same kernels: results
    are bit-for-bit those of the graph."""
    torch, nc = env
    sy = systems(4, seed=5)
    out = []
    for host in (False, True):
        B = nc.pcg_batch_create(8, sum(t[0].n for t in sy) + 10, 32, host_loop=host)
        slots = [add(nc, torch, B, *t) for t in sy]
        nc.pcg_batch_run(B, 1e-8, 3000)
        out.append([collect(nc, torch, B, s, t[0].n) for s, t in zip(slots, sy)])
    for (ra, xa), (rb, xb) in zip(*out):
        assert ra == rb and np.array_equal(xa, xb)
