"""Records how many iterations the oracle's solvers need on the 1,048,576-point
random-sphere workload (K = 20, u = 5z^3 - 3z, f = 13u, rtol 1e-8):

* "multigrid": the oracle's FP64 aggregation-multigrid BiCGSTAB (oracle/amg.py,
  the solver the GPU path also uses) on the rows relabelled along a Z-order
  curve; minutes on a few cores;
* "bicgstab": its unpreconditioned FP64 BiCGSTAB (oracle.bicgstab); about ten
  minutes on 8 cores, run only with --bicgstab.

The benchmark's reference arm and CPU baseline time a bounded sample of the
oracle (kNN, assembly, the hierarchy and a few preconditioned iterations) and
project the full solve with the "multigrid" count.  Calls only oracle/ and the
seeded input generator."""
import argparse
import json
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[1]
sys.path.insert(0, str(ROOT))

import oracle  # noqa: E402
from oracle import amg as OA  # noqa: E402
from paper_1603_04100_gb300 import inputs as I  # noqa: E402

OUT = Path(__file__).resolve().parent / "iterations_random_sphere_1m_k20.json"
WORKLOAD = "random unit sphere n=1048576 seed=0, K=20, MEAN_NN(6), u=5z^3-3z, f=13u, sigma=1, rtol=1e-8"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--bicgstab", action="store_true", help="also rerun the unpreconditioned solve")
    args = ap.parse_args()
    rec = json.loads(OUT.read_text()) if OUT.exists() else {}
    rec["workload"] = WORKLOAD
    n, k = 1_048_576, 20
    pr = I.random_sphere_problem(n, k, seed=0)
    nbr = oracle.knn_grid(pr.pts, k)
    val, st, _, _ = oracle.assemble(pr.pts, nbr, delta_m=6)
    f = pr.f[:, 0]
    if args.bicgstab or "bicgstab" not in rec:
        t0 = time.perf_counter()
        u, it, rr, status = oracle.bicgstab(val, nbr, f, rtol=1e-8, maxit=100000)
        rec["bicgstab"] = {"solver": "unpreconditioned BiCGSTAB (oracle.bicgstab, C, OpenMP)", "iters": it,
                           "relres": rr, "status": status,
                           "err_exact_inf": float(abs(u - pr.u_exact[:, 0]).max()),
                           "solve_seconds": time.perf_counter() - t0, "threads": oracle.threads()}
    perm = I.morton_permutation(pr.pts)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(n)
    t0 = time.perf_counter()
    levels = OA.hierarchy(val[perm], inv[nbr[perm]].astype(np.int32), 1.0)
    t1 = time.perf_counter()
    x, it, rr = OA.bicgstab_right(levels, np.ascontiguousarray(f[perm]), rtol=1e-8)
    t2 = time.perf_counter()
    u = np.empty_like(x)
    u[perm] = x
    rec["multigrid"] = {"solver": "aggregation-multigrid right-preconditioned BiCGSTAB (oracle/amg.py, numpy, "
                                  "rows in Z-order)", "iters": it, "relres": rr,
                        "err_exact_inf": float(abs(u - pr.u_exact[:, 0]).max()),
                        "hierarchy_seconds": t1 - t0, "solve_seconds": t2 - t1}
    OUT.write_text(json.dumps(rec, indent=1) + "\n")
    print(OUT.read_text())


if __name__ == "__main__":
    main()
