"""Profiling driver: kNN + assembly + a solve capped at a few iterations on a
random unit sphere (K = 20), run twice, for Nsight Compute captures.

    python -m paper_1603_04100_gb300.profile_case [n] [prec: 0 FP64 | 1 FP32+refine] [iterations]
                                                  [precond: 1 row scaling | 2 multigrid]
"""
import sys

import torch

from . import api
from . import inputs as I


def main(argv):
    n = int(argv[1]) if len(argv) > 1 else 262144
    prec = int(argv[2]) if len(argv) > 2 else 1
    iters = int(argv[3]) if len(argv) > 3 else 30
    precond = int(argv[4]) if len(argv) > 4 else 1
    dev = torch.device("cuda:0")
    pr = I.random_sphere_problem(n, 20, seed=0)
    pts = torch.from_numpy(pr.pts).to(dev)
    f = torch.from_numpy(pr.f).to(dev)
    for _ in range(2):
        nbr, order = api.knn(pts, 20, want_order=True)
        op = api.assemble(pts, nbr, prec=prec, order=order)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        r = api.solve(op, f, rtol=1e-8, precond=precond, maxit=iters)
        t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    its = r.iters[0]
    print("ok", r.iters, r.outer, "solve %.3f ms, %.1f us per iteration" % (ms, 1e3 * ms / max(1, its)))


if __name__ == "__main__":
    main(sys.argv)
