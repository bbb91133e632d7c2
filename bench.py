#!/usr/bin/env python3
"""Benchmark of Newton-Chebyshev preconditioned CG on one GB300.

Workload (one "step" = one full PCG solve to ||r||/||b|| <= 1e-8):
3D 7-point variable-coefficient diffusion on a 128^3 grid (n = 2,097,152,
nnz = 14,581,760), per-point log-normal coefficients (sigma = 1),
harmonic face averages, Dirichlet boundary; CSR float64; Jacobi scaled;
20-step Lanczos bounds; polynomial degree k (default 20), theta scale
1.001; right-hand sides U[-1,1] from seeds.  Inputs (A = 183 MB) are larger
than L2 (129 MB), so no flush is needed between steps.

Prints ONE JSON line: solves/s (whole job), p50/p99 solve latency, the
end-to-end rate through the host-buffer C-ABI call, the roofline of the
fused SpMV + Chebyshev step kernel and the FP64 oracle timed on the host.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--k 20] [--apply f64|f32|bf16]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the same workload
N > 1 runs independent replicas (one per GPU, launched by torchrun).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solves/s and p50/p99 latency at rel. resid 1e-8; P_k(A)v HBM GB/s vs peak"
GRID, SEED_A, SEED_V0, SEED_B, S_THETA, TOL, MAXIT = 128, 7, 3, 5, 1.001, 1e-8, 5000
GOLDEN = os.path.join(ROOT, "tests", "golden", "c2_oracle.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--k", type=int, default=20)
    ap.add_argument("--apply", default="f64", choices=["f64", "f32", "bf16"])
    ap.add_argument("--grid", type=int, default=GRID)
    ap.add_argument("--no-modes", action="store_true", help="skip the other apply precisions")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--oracle-iters", type=int, default=6, help="PCG iterations per oracle sample")
    ap.add_argument("--host-loop", action="store_true",
                    help="drive the PCG loop from the host instead of the device-side graph "
                         "(same kernels; lets a profiler list every launch)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


# ---------------------------------------------------------------- clocks ----
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_uuid):
        self.proc = None
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "100"]
        if dev_uuid:
            cmd += ["-i", dev_uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------ workload ------
def make_system(grid):
    import workloads as W
    A = W.diffusion_3d_7pt_lognormal(grid, seed=SEED_A)
    return A


def algorithmic_step_bytes(n, nnz, sv=8, sx=8):
    """Bytes one fused Chebyshev step must move: A once (values + int32
    columns + int32 row pointers), x_{k-1}, x_{k-2}, r read once, x_k written."""
    return nnz * (sv + 4) + 4 * (n + 1) + 4 * n * sx


# ---------------------------------------------------------------- ours ------
def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    torch.cuda.set_device(local_rank)
    from paper_2008_01440_gb300.build import build
    build()
    import paper_2008_01440_gb300 as nc
    import workloads as W

    A = make_system(args.grid)
    n, nnz = A.n, A.nnz
    dev = torch.device("cuda", local_rank)
    rp = torch.from_numpy(A.rowptr).to(dev)
    cl = torch.from_numpy(A.col).to(dev)
    vl = torch.from_numpy(A.val).to(dev)
    M0 = nc.nc_matrix_csr(rp, cl, vl)
    M = nc.nc_matrix_jacobi(M0)
    v0 = torch.from_numpy(W.uniform_vector(n, seed=SEED_V0)).to(dev)
    lo, hi, rmin, rmax = nc.nc_bounds_lanczos(M, 20, v0)
    n_rhs = 4
    bs = [torch.from_numpy(W.uniform_vector(n, seed=SEED_B + i)).to(dev) for i in range(n_rhs)]
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def timed_solves(S, steps, warmup):
        for i in range(warmup):
            nc.pcg_solve(S, bs[i % n_rhs], x, TOL, MAXIT)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        results = []
        for i in range(steps):
            ev[i][0].record(stream)
            results.append(nc.pcg_solve(S, bs[i % n_rhs], x, TOL, MAXIT))
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        lat = [a.elapsed_time(b) for a, b in ev]
        total = ev[0][0].elapsed_time(ev[-1][1])
        return lat, total, results

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def allmax(v):
        if world == 1:
            return v
        import torch.distributed as dist
        t = torch.tensor([v], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def time_step_kernel(S, mode):
        """Average duration of one fused-step launch: CUDA events around
        `reps` applications of P_k (k launches each) on the launching stream."""
        z = torch.empty(n, dtype=torch.float64, device=dev)
        reps = 10
        for _ in range(2):
            nc.pcg_apply_poly(S, bs[0], z)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            nc.pcg_apply_poly(S, bs[0], z)
        e1.record(stream)
        torch.cuda.synchronize()
        per_launch_s = e0.elapsed_time(e1) / 1e3 / (reps * max(args.k, 1))
        sv = {"f64": 8, "f32": 4, "bf16": 2}[mode]
        sx = 8 if mode == "f64" else 4
        nbytes = algorithmic_step_bytes(n, nnz, sv, sx)
        return per_launch_s, nbytes

    modes = [args.apply] + ([] if args.no_modes else [m for m in ("f64", "f32", "bf16") if m != args.apply])
    out_modes = {}
    main = None
    for mode in modes:
        S = nc.pcg_setup(M, lo, hi, args.k, S_THETA, apply_dtype=mode, x0_is_zero=True,
                         use_graph=not args.host_loop)
        barrier()
        clk = None
        if mode == args.apply:
            uuid = None
            try:
                uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
            except Exception:
                uuid = None
            clk = Clocks(uuid)
        torch.cuda.synchronize()
        barrier()
        lat, total_ms, results = timed_solves(S, args.steps, args.warmup)
        barrier()
        clocks = clk.stop() if clk else None
        total_ms = allmax(total_ms)
        iters = [r["iters"] for r in results]
        ok = all(r["status"] == 0 for r in results)
        rec = {"solves_per_s": world * args.steps / (total_ms / 1e3), "ms_per_solve": total_ms / args.steps,
               "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
               "iters": iters[0], "iters_range": [min(iters), max(iters)], "all_converged": ok,
               "max_relres": max(r["relres"] for r in results),
               "max_true_relres": max(r["true_relres"] for r in results)}
        t_launch, nbytes = time_step_kernel(S, mode)
        rec["step_us"] = round(t_launch * 1e6, 2)
        rec["step_GBps"] = round(nbytes / t_launch / 1e9, 1)
        out_modes[mode] = rec
        if mode == args.apply:
            main = dict(rec=rec, S=S, clocks=clocks, results=results)
        else:
            S.close()

    S = main["S"]
    rec = main["rec"]
    k = max(args.k, 1)
    # --- kernel timing: the fused step kernel, k launches per apply ---------------------
    per_launch_s, step_bytes = time_step_kernel(S, args.apply)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    achieved = step_bytes / per_launch_s / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": None, "peak_source": peak_src,
                "kernel": "csr_step_kernel (fused SpMV + Chebyshev recurrence)",
                "bytes_per_launch": step_bytes, "us_per_launch": round(per_launch_s * 1e6, 2)}

    # --- end to end through the host-buffer C-ABI call ---------------------------------
    hb = [bb.cpu().pin_memory() for bb in bs]
    hx = torch.zeros(n, dtype=torch.float64).pin_memory()
    for i in range(2):
        nc.pcg_solve_host(S, hb[i % n_rhs], hx, TOL, MAXIT)
    barrier()
    t0 = time.perf_counter()
    e2e_res = []
    for i in range(args.steps):
        e2e_res.append(nc.pcg_solve_host(S, hb[i % n_rhs], hx, TOL, MAXIT))
    torch.cuda.synchronize()
    e2e_s = allmax(time.perf_counter() - t0)
    e2e = {"value": world * args.steps / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": n * 8,
           "d2h_bytes_per_step": n * 8 + 48}

    # --- oracle on the host (rank 0, one GPU only) ---------------------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline_subprocess(args)

    iters = rec["iters"]
    launches_per_solve = 1 + (4 + k + (1 if args.apply != "f64" else 0)) + iters * (k + 3) + 3
    line = {
        "metric": METRIC, "value": round(rec["solves_per_s"], 3), "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(rec["ms_per_solve"], 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.apply == "f64" else f"{args.apply}-apply+f64-outer",
        "data": "synthetic (seeded generators, no dataset)",
        "config": {"workload": f"diffusion3d-7pt lognormal {args.grid}^3 CSR (n={n}, nnz={nnz}), Jacobi-scaled",
                   "degree_k": args.k, "theta_scale": S_THETA, "tol": TOL, "bounds": "lanczos-20",
                   "lmin": lo, "lmax": hi, "rhs": f"{n_rhs} seeded U[-1,1], cycled",
                   "l2": "inputs larger than L2 (A = %.0f MB)" % (nnz * 12 / 1e6), "parallelism": f"replicas x{world}"},
        "p50_ms": round(rec["p50_ms"], 3), "p99_ms": round(rec["p99_ms"], 3), "iters": iters,
        "all_converged": rec["all_converged"], "max_relres": rec["max_relres"],
        "clocks": main["clocks"], "e2e": e2e, "gpu_launches": launches_per_solve * args.steps,
        "roofline": roofline, "cpu_baseline": cpu, "modes": out_modes,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def cpu_baseline_subprocess(args):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, os.path.abspath(__file__), "--impl", "reference", "--steps", "1", "--warmup", "0",
           "--k", str(args.k), "--grid", str(args.grid), "--oracle-iters", str(args.oracle_iters)]
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=900)
        line = [ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1]
        ref = json.loads(line)
        cb = ref.get("cpu_baseline", {})
        return {"value": ref["value"], "unit": ref["unit"], "cores": cb.get("cores", 1), "kind": "oracle",
                "sample": cb.get("sample")}
    except Exception as e:  # report, do not fail the GPU measurement
        return {"value": None, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": f"failed: {e}"}


# ----------------------------------------------------------- reference ------
def run_reference(args, rank, world):
    """The FP64 oracle as it stands, timed on the host cores: each step runs
    `oracle_iters` PCG iterations of the full workload and the rate is
    extrapolated with the oracle's own full-solve iteration count."""
    if rank != 0:
        return
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    import numpy as np
    import oracle as O
    import workloads as W
    A = make_system(args.grid)
    val, dis = O.jacobi_scale_csr(A.rowptr, A.col, A.val, A.n)
    mv = O.csr_matvec(A.rowptr, A.col, val, A.n)
    golden = None
    if args.grid == GRID and os.path.exists(GOLDEN):
        with open(GOLDEN) as f:
            golden = json.load(f)
    if golden is not None and str(args.k) in golden["solves"]:
        lo, hi = golden["lmin"], golden["lmax"]
        full_iters = golden["solves"][str(args.k)]["iters"]
    else:
        rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
        g = float(np.bincount(rows, weights=np.abs(val), minlength=A.n).max())
        lo, hi, _ = O.lanczos_bounds(mv, W.uniform_vector(A.n, seed=SEED_V0), 20, gershgorin=g)
        full_iters = None
    prm = O.cheb_params(lo, hi, S_THETA)
    b = dis * W.uniform_vector(A.n, seed=SEED_B)
    m = args.oracle_iters
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        res = O.pcg(mv, b, lambda r: O.cheb_apply(mv, r, prm, args.k), m=args.k, tol=TOL, maxit=m)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt / max(res.iters, 1))
        if full_iters is None and i == 0:
            full = O.pcg(mv, b, lambda r: O.cheb_apply(mv, r, prm, args.k), m=args.k, tol=TOL, maxit=MAXIT)
            full_iters = full.iters
    t_iter = statistics.median(times)
    value = 1.0 / (t_iter * full_iters)
    sample = (f"{m} PCG iterations (k={args.k}, {m * (args.k + 1)} SpMVs) of the full {args.grid}^3 system per step, "
              f"extrapolated to the oracle's {full_iters}-iteration solve; scipy CSR matvec + numpy, 1 thread")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_iter * full_iters * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded generators, no dataset)",
            "config": {"workload": f"diffusion3d-7pt lognormal {args.grid}^3 CSR (n={A.n}, nnz={A.nnz}), Jacobi-scaled",
                       "degree_k": args.k, "theta_scale": S_THETA, "tol": TOL},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local_rank = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        else:
            run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
