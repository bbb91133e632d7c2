"""Explicit matrices in the batched engine (pcg_batch_add_solver,
pcg_batch_add_solver_multi, pcg_solve_batched): every (system, right-hand
side) pair of several CSR systems -- each with its own solver, layout,
degree and bounds -- runs as a slot of one engine, in one graph launch per
run; a system's right-hand sides may share its matrix reads as a group.

Checked: each slot against the FP64 oracle's PCG on the same scaled system
(iterations +-1 with the float64 apply, the solution within the tolerance's
reach), against the solver's own pcg_solve, bit-for-bit identity of a
slot's result alone and in a mix (every slot reduces its own dot products in
a fixed order), of a group's columns and single slots, a group column
released mid-run with its range reused, explicit and stencil slots in one
engine, and the combinations the engine refuses."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from nchelpers import csr_to_gpu, need_gpu, rel_err, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = need_gpu()
    import paper_2008_01440_gb300 as nc
    return torch, nc


def _systems():
    """(CSR, Jacobi-scale?, degree) of a few uneven explicit systems."""
    st = W.stencil7_aniso(17, 9, 13, 1.0, 0.4, 0.2)
    return [(W.diffusion_3d_7pt_lognormal(20, seed=1), True, 10),
            (W.laplacian_2d_5pt(50, 40), False, 8),
            (W.stencil7_to_csr(st), True, 16),
            (W.diffusion_3d_7pt_lognormal(24, seed=2), True, 5)]


def _setup(torch, nc, dt, systems):
    out = []
    for A, scale, k in systems:
        M = csr_to_gpu(torch, nc, A)
        if scale:
            M = nc.nc_matrix_jacobi(M)
        lo, hi, _, _ = nc.nc_bounds_lanczos(M, 20, to_dev(torch, W.uniform_vector(A.n, seed=3)))
        S = nc.pcg_setup(M, lo, hi, k, 1.001, apply_dtype=dt, x0_is_zero=True)
        out.append((A, scale, k, M, S, lo, hi))
    return out


def _oracle(A, scale, k, lo, hi, b):
    if scale:
        val, dis = O.jacobi_scale_csr(A.rowptr, A.col, A.val, A.n)
    else:
        val, dis = A.val, np.ones(A.n)
    mv = O.csr_matvec(A.rowptr, A.col, val, A.n)
    prm = O.cheb_params(lo, hi, 1.001)
    ro = O.pcg(mv, dis * b, lambda r: O.cheb_apply(mv, r, prm, k), m=k, tol=1e-8, maxit=5000)
    return ro, dis * ro.x


@pytest.mark.parametrize("dt", ["f64", "f32", "bf16"])
def test_batched_explicit_systems_match_oracle_and_solver(env, dt):
    torch, nc = env
    sy = _setup(torch, nc, dt, _systems())
    nrhs = [2, 1, 3, 2]
    Bh = [np.stack([W.uniform_vector(A.n, seed=100 * i + c) for c in range(m)]) for i, ((A, *_), m) in
          enumerate(zip(sy, nrhs))]
    Bs = [to_dev(torch, b) for b in Bh]
    Xs = [torch.full_like(b, float("nan")) for b in Bs]
    res = nc.pcg_solve_batched([s[4] for s in sy], Bs, Xs, 1e-8, 5000)
    assert len(res) == sum(nrhs)
    q = 0
    for i, (A, scale, k, M, S, lo, hi) in enumerate(sy):
        for c in range(nrhs[i]):
            r = res[q]
            q += 1
            x = Xs[i][c].cpu().numpy()
            assert r["status"] == 0 and r["true_relres"] <= 2e-8, (i, c, r)
            assert r["n_spmv"] == (k + 1) * r["iters"] and r["n_dot"] == 3 * r["iters"]
            ro, xo = _oracle(A, scale, k, lo, hi, Bh[i][c])
            assert abs(r["iters"] - ro.iters) <= (1 if dt == "f64" else 3), (i, c, r["iters"], ro.iters)
            assert rel_err(x, xo) <= (hi / lo) * 1e-8, (i, c)
            # the solver on its own
            xs = torch.zeros(A.n, dtype=torch.float64, device="cuda")
            rs = nc.pcg_solve(S, Bs[i][c].contiguous(), xs, 1e-8, 5000)
            assert abs(rs["iters"] - r["iters"]) <= 1
            assert rel_err(x, xs.cpu().numpy()) <= (hi / lo) * 1e-8


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_batched_slot_is_the_same_alone_and_in_a_mix(env, dt):
    torch, nc = env
    sy = _setup(torch, nc, dt, _systems())
    A0, S0 = sy[0][0], sy[0][4]
    b0 = to_dev(torch, W.uniform_vector(A0.n, seed=7)).reshape(1, -1)
    x_alone = torch.zeros_like(b0)
    r_alone = nc.pcg_solve_batched([S0], [b0], [x_alone], 1e-8, 5000)
    others = [sy[2], sy[1], sy[3]]
    Bs = [to_dev(torch, W.uniform_vector(s[0].n, seed=30 + j)).reshape(1, -1) for j, s in enumerate(others)]
    solvers = [others[0][4], S0, others[1][4], others[2][4]]
    Bmix = [Bs[0], b0, Bs[1], Bs[2]]
    Xmix = [torch.zeros_like(b) for b in Bmix]
    r_mix = nc.pcg_solve_batched(solvers, Bmix, Xmix, 1e-8, 5000)
    assert r_mix[1]["iters"] == r_alone[0]["iters"]
    assert torch.equal(Xmix[1], x_alone)


def test_explicit_and_stencil_slots_in_one_engine(env):
    torch, nc = env
    sy = _setup(torch, nc, "f32", _systems()[:2])
    eng = nc.pcg_batch_create(8, 200_000, 32)
    st = W.stencil7_aniso(12, 10, 9, 1.0, 0.5, 0.3)
    sc = W.Stencil7(st.nx, st.ny, st.nz, 1.0, st.cx / st.c0, st.cy / st.c0, st.cz / st.c0)
    lo_s, hi_s = W.stencil7_bounds(sc)
    bst = to_dev(torch, W.uniform_vector(st.n, seed=5))
    slots = [nc.pcg_batch_add(eng, st.nx, st.ny, st.nz, st.c0, st.cx, st.cy, st.cz, lo_s, hi_s, 12, 1.001, bst)]
    bs = []
    for i, s in enumerate(sy):
        b = to_dev(torch, W.uniform_vector(s[0].n, seed=60 + i))
        bs.append(b)
        slots.append(nc.pcg_batch_add_solver(eng, s[4], b))
    assert nc.pcg_batch_run(eng, 1e-8, 5000) == 0
    for j, sl in enumerate(slots):
        done, r = nc.pcg_batch_status(eng, sl)
        assert done and r["status"] == 0 and r["true_relres"] <= 2e-8
    # the explicit slots against the oracle
    for i, s in enumerate(sy):
        A, scale, k, M, S, lo, hi = s
        x = torch.empty(A.n, dtype=torch.float64, device="cuda")
        nc.pcg_batch_collect(eng, slots[1 + i], x)
        torch.cuda.synchronize()
        _, xo = _oracle(A, scale, k, lo, hi, bs[i].cpu().numpy())
        assert rel_err(x.cpu().numpy(), xo) <= (hi / lo) * 1e-8
    eng.close()


def test_engine_refuses_what_it_cannot_run(env):
    torch, nc = env
    A = W.laplacian_2d_5pt(30, 30)
    lo, hi = W.laplacian_2d_bounds(30, 30)
    M = csr_to_gpu(torch, nc, A)
    b = to_dev(torch, W.uniform_vector(A.n, seed=1))
    eng = nc.pcg_batch_create(4, 10_000, 16)   # float32 engine
    S64 = nc.pcg_setup(M, lo, hi, 8, 1.001)   # float64 apply: not this engine's precision
    with pytest.raises(nc.NcError) as e1:
        nc.pcg_batch_add_solver(eng, S64, b)
    assert e1.value.status == nc.NC_ERR_UNSUPPORTED
    Sdeep = nc.pcg_setup(M, lo, hi, 20, 1.001, apply_dtype="f32")   # degree above kmax
    with pytest.raises(nc.NcError) as e2:
        nc.pcg_batch_add_solver(eng, Sdeep, b)
    assert e2.value.status == nc.NC_ERR_ARG
    Srr = nc.pcg_setup(M, lo, hi, 8, 1.001, apply_dtype="f32", rr_period=10)   # residual replacement
    with pytest.raises(nc.NcError) as e3:
        nc.pcg_batch_add_solver(eng, Srr, b)
    assert e3.value.status == nc.NC_ERR_UNSUPPORTED
    eng.close()
    eng64 = nc.pcg_batch_create(4, 10_000, 16, f64_apply=True)
    Snewton = nc.pcg_setup(M, lo, hi, 7, 1.001, poly="newton")   # Algorithm 1's form: not in the engine
    with pytest.raises(nc.NcError) as e4:
        nc.pcg_batch_add_solver(eng64, Snewton, b)
    assert e4.value.status == nc.NC_ERR_UNSUPPORTED
    assert nc.pcg_batch_add_solver(eng64, S64, b) is not None
    eng64.close()


def _run_singles(torch, nc, S, B, f64):
    """Every row of B as a slot of its own in a fresh engine; (X, results)."""
    eng = nc.pcg_batch_create(B.shape[0], B.shape[0] * S.n, 32, f64_apply=f64)
    slots = [nc.pcg_batch_add_solver(eng, S, B[c]) for c in range(B.shape[0])]
    assert nc.pcg_batch_run(eng, 1e-8, 5000) == 0
    X = torch.empty_like(B)
    res = []
    for c, sl in enumerate(slots):
        res.append(nc.pcg_batch_status(eng, sl)[1])
        nc.pcg_batch_collect(eng, sl, X[c])
    torch.cuda.synchronize()
    eng.close()
    return X, res


@pytest.mark.parametrize("dt", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("m", [2, 3, 5, 8])
def test_group_columns_are_bit_identical_to_single_slots(env, dt, m):
    """m right-hand sides admitted together (groups of up to 4 reading the
    matrix once per step -- 3 runs a width-4 kernel with a column masked, 5
    a group of 4 and a plain slot, 8 two groups) give every column exactly
    the iterates of a slot of its own."""
    torch, nc = env
    A, scale, k, M, S, lo, hi = _setup(torch, nc, dt, [_systems()[m % 2 * 2]])[0]
    B = to_dev(torch, np.stack([W.uniform_vector(A.n, seed=500 + c) for c in range(m)]))
    eng = nc.pcg_batch_create(m, m * A.n, 32, f64_apply=(dt == "f64"))
    slots = nc.pcg_batch_add_solver_multi(eng, S, B)
    assert len(slots) == m
    assert nc.pcg_batch_run(eng, 1e-8, 5000) == 0
    X = torch.empty_like(B)
    res = []
    for c, sl in enumerate(slots):
        res.append(nc.pcg_batch_status(eng, sl)[1])
        nc.pcg_batch_collect(eng, sl, X[c])
    torch.cuda.synchronize()
    eng.close()
    Xs, rs = _run_singles(torch, nc, S, B, dt == "f64")
    for c in range(m):
        assert res[c]["status"] == 0 and res[c]["iters"] == rs[c]["iters"], (c, res[c], rs[c])
        assert res[c]["n_spmv"] == (k + 1) * res[c]["iters"] and res[c]["n_dot"] == 3 * res[c]["iters"]
    assert torch.equal(X, Xs)


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_group_column_released_mid_run_and_its_range_reused(env, dt):
    """Continuous batching with a group: a column that stops at once (b = 0)
    is collected and released while the others run; a new slot admitted into
    the freed range runs beside them.  Neither disturbs the other: every
    column and the newcomer match their own runs bit for bit."""
    torch, nc = env
    sy = _setup(torch, nc, dt, _systems()[:2])
    A, S = sy[0][0], sy[0][4]
    A1, S1 = sy[1][0], sy[1][4]
    Bh = np.stack([W.uniform_vector(A.n, seed=700 + c) for c in range(4)])
    Bh[1] = 0.0
    B = to_dev(torch, Bh)
    # room for the group and nothing else: the newcomer must take the freed range
    eng = nc.pcg_batch_create(5, 4 * A.n, 32, f64_apply=(dt == "f64"))
    slots = nc.pcg_batch_add_solver_multi(eng, S, B)
    nc.pcg_batch_run(eng, 1e-8, 5000, 2)
    done, r1 = nc.pcg_batch_status(eng, slots[1])
    assert done and r1["status"] == 0 and r1["iters"] == 0
    x1 = torch.full((A.n,), float("nan"), dtype=torch.float64, device="cuda")
    nc.pcg_batch_collect(eng, slots[1], x1)
    nc.pcg_batch_release(eng, slots[1])
    assert A1.n <= A.n
    b_new = to_dev(torch, W.uniform_vector(A1.n, seed=777))
    s_new = nc.pcg_batch_add_solver(eng, S1, b_new)
    assert s_new is not None
    assert nc.pcg_batch_run(eng, 1e-8, 5000) == 0
    X = torch.empty_like(B)
    for c in (0, 2, 3):
        nc.pcg_batch_collect(eng, slots[c], X[c])
    x_new = torch.empty_like(b_new)
    nc.pcg_batch_collect(eng, s_new, x_new)
    torch.cuda.synchronize()
    res = {c: nc.pcg_batch_status(eng, slots[c])[1] for c in (0, 2, 3)}
    r_new = nc.pcg_batch_status(eng, s_new)[1]
    eng.close()
    assert torch.count_nonzero(x1) == 0
    Xs, rs = _run_singles(torch, nc, S, B[[0, 2, 3]].contiguous(), dt == "f64")
    for i, c in enumerate((0, 2, 3)):
        assert res[c]["iters"] == rs[i]["iters"]
        assert torch.equal(X[c], Xs[i]), c
    xn, rn = _run_singles(torch, nc, S1, b_new.reshape(1, -1), dt == "f64")
    assert r_new["iters"] == rn[0]["iters"] and torch.equal(x_new, xn[0])


def test_group_admission_limits(env):
    torch, nc = env
    A, scale, k, M, S, lo, hi = _setup(torch, nc, "f32", _systems()[1:2])[0]
    eng = nc.pcg_batch_create(8, 3 * A.n, 32)
    B = to_dev(torch, np.stack([W.uniform_vector(A.n, seed=c) for c in range(9)]))
    with pytest.raises(nc.NcError) as e:
        nc.pcg_batch_add_solver_multi(eng, S, B)          # more than 8 columns
    assert e.value.status == nc.NC_ERR_ARG
    assert nc.pcg_batch_add_solver_multi(eng, S, B[:4].contiguous()) is None   # 4 n unknowns > 3 n
    sl = nc.pcg_batch_add_solver_multi(eng, S, B[:3].contiguous())
    assert sl is not None and len(set(sl)) == 3
    assert nc.pcg_batch_run(eng, 1e-8, 5000) == 0
    eng.close()
