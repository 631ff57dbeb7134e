"""Runs the oracle's unpreconditioned FP64 BiCGSTAB to a 1e-8 relative residual
on the 1,048,576-point random-sphere workload (K = 20, u = 5z^3 - 3z,
f = 13u) and records how many iterations it needed.  The benchmark's CPU
baseline times a bounded number of oracle iterations and scales by this count.
Calls only oracle/ and the seeded input generator.  Takes minutes."""
import json
import sys
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]
sys.path.insert(0, str(ROOT))

import oracle  # noqa: E402
from paper_1603_04100_gb300 import inputs as I  # noqa: E402

OUT = Path(__file__).resolve().parent / "iterations_random_sphere_1m_k20.json"


def main():
    n, k = 1_048_576, 20
    pr = I.random_sphere_problem(n, k, seed=0)
    nbr = oracle.knn_grid(pr.pts, k)
    val, st, _, _ = oracle.assemble(pr.pts, nbr, delta_m=6)
    t0 = time.perf_counter()
    u, it, rr, status = oracle.bicgstab(val, nbr, pr.f[:, 0], rtol=1e-8, maxit=100000)
    dt = time.perf_counter() - t0
    err = float(abs(u - pr.u_exact[:, 0]).max())
    OUT.write_text(json.dumps({"workload": "random unit sphere n=1048576 seed=0, K=20, MEAN_NN(6), "
                                           "u=5z^3-3z, f=13u, sigma=1, unpreconditioned BiCGSTAB, rtol=1e-8",
                               "iters": it, "relres": rr, "status": status, "err_exact_inf": err,
                               "solve_seconds": dt, "threads": oracle.threads()}, indent=1) + "\n")
    print(OUT.read_text())


if __name__ == "__main__":
    main()
