"""Write tests/golden/c3_oracle.json: oracle results for the elasticity workload.

Workload: Q1-hex linear elasticity, 100^3 nodes x 3 dofs (n = 3,000,000,
26,463,592 3x3 blocks), E = 1, nu ~ U[0.25, 0.45] per element (seed 7),
bottom face clamped, unit downward body load; Jacobi scaled; 20-step
Lanczos bounds from a U[-1,1] start vector (seed 3) with the Gershgorin cap;
theta scale 1.001; tol 1e-8; degrees k = 20 and 60 (the workload's two).

Calls only ``oracle`` and ``workloads``.  Degrees already stored for the same
bounds are kept, only missing ones are solved.  Run:
    python tests/golden/make_c3_golden.py     (about half an hour of CPU per degree)
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

N, SEED_A, SEED_V0, S_THETA, TOL = 100, 7, 3, 1.001, 1e-8
DEGREES = (20, 60)


def main():
    A, b = W.elasticity_q1_bsr3(N, seed=SEED_A)
    val, dis = O.jacobi_scale_bsr3(A.browptr, A.bcol, A.val, A.nb)
    mv = O.bsr3_matvec(A.browptr, A.bcol, val, A.nb)
    brows = np.repeat(np.arange(A.nb), np.diff(A.browptr))
    rs = np.zeros(A.n)
    np.add.at(rs, (3 * brows[:, None] + np.arange(3)[None, :]).ravel(), np.abs(val).sum(axis=2).ravel())
    gersh = float(rs.max())
    lo, hi, info = O.lanczos_bounds(mv, W.uniform_vector(A.n, seed=SEED_V0), 20, gershgorin=gersh)
    out = dict(workload="elasticity Q1-hex 100^3 nodes x 3 dofs, 3x3 BSR, Jacobi scaled", n=A.n, nnzb=A.nnzb,
               seed_matrix=SEED_A, seed_v0=SEED_V0, theta_scale=S_THETA, tol=TOL, lanczos_steps=20, lmin=lo,
               lmax=hi, ritz_min=float(info["ritz"].min()), ritz_max=float(info["ritz"].max()), gershgorin=gersh,
               solves={})
    path = os.path.join(HERE, "c3_oracle.json")
    if os.path.exists(path):
        with open(path) as f:
            old = json.load(f)
        if old.get("lmin") == lo and old.get("lmax") == hi:
            out["solves"].update(old.get("solves", {}))
    for k in DEGREES:
        if str(k) in out["solves"]:
            continue
        prm = O.cheb_params(lo, hi, S_THETA)
        t = time.time()
        res = O.pcg(mv, dis * b, lambda r: O.cheb_apply(mv, r, prm, k), m=k, tol=TOL, maxit=5000)
        out["solves"][str(k)] = dict(iters=res.iters, status=res.status, relres=res.relres,
                                     true_relres=res.true_relres, seconds=time.time() - t)
        print(k, out["solves"][str(k)], flush=True)
        with open(path, "w") as f:
            json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
