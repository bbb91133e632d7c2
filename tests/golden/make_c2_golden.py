"""Write tests/golden/c2_oracle.json: oracle results for the 128^3 workload.

Workload: 3D 7-point variable-coefficient diffusion on a 128^3 grid
(n = 2,097,152, log-normal coefficients, sigma = 1, seed 7), Jacobi scaled,
right-hand side U[-1,1] (seed 5), 20-step Lanczos bounds from a U[-1,1]
start vector (seed 3) with the Gershgorin cap, theta scale s = 1.001,
tol = 1e-8, degrees k = 10, 20, 40.

Calls only ``oracle`` and ``workloads`` (the CUDA path is never involved).
Run:  python tests/golden/make_c2_golden.py   (several minutes of CPU)
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402

N, SEED_A, SEED_B, SEED_V0, S_THETA, TOL = 128, 7, 5, 3, 1.001, 1e-8
DEGREES = (10, 20, 40)


def main():
    A = W.diffusion_3d_7pt_lognormal(N, seed=SEED_A)
    val, dis = O.jacobi_scale_csr(A.rowptr, A.col, A.val, A.n)
    mv = O.csr_matvec(A.rowptr, A.col, val, A.n)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    gersh = float(np.bincount(rows, weights=np.abs(val), minlength=A.n).max())
    lo, hi, info = O.lanczos_bounds(mv, W.uniform_vector(A.n, seed=SEED_V0), 20, gershgorin=gersh)
    b = dis * W.uniform_vector(A.n, seed=SEED_B)
    out = dict(workload="diffusion3d-lognormal-128^3 CSR, Jacobi scaled", n=A.n, nnz=A.nnz,
               seed_matrix=SEED_A, seed_rhs=SEED_B, seed_v0=SEED_V0, theta_scale=S_THETA, tol=TOL,
               lanczos_steps=20, lmin=lo, lmax=hi, ritz_min=float(info["ritz"].min()),
               ritz_max=float(info["ritz"].max()), gershgorin=gersh, solves={})
    for k in DEGREES:
        prm = O.cheb_params(lo, hi, S_THETA)
        t = time.time()
        res = O.pcg(mv, b, lambda r: O.cheb_apply(mv, r, prm, k), m=k, tol=TOL, maxit=5000)
        out["solves"][str(k)] = dict(iters=res.iters, status=res.status, relres=res.relres,
                                     true_relres=res.true_relres, seconds=time.time() - t)
        print(k, out["solves"][str(k)], flush=True)
    with open(os.path.join(HERE, "c2_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
