"""Oracle-side helpers shared by the parity tests (CPU only, FP64)."""
from __future__ import annotations

import numpy as np

from oracle import amg as OA
from paper_1603_04100_gb300 import inputs as I


def reference_solution(pts, nbr, val, f, rtol: float = 1e-11):
    """The oracle's solution of (I - L) u = f for rows given in point order.

    The oracle's multigrid aggregates consecutive rows, so it runs on the same
    rows relabelled along a Z-order curve of the points (P A P^T x' = P f, the
    same system); FP64 iterative refinement around its preconditioned BiCGSTAB
    takes the true residual to `rtol`.  Returns (u in point order, iterations,
    relative residual)."""
    perm = I.morton_permutation(np.asarray(pts))
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size)
    nbr_m = inv[np.asarray(nbr)[perm]].astype(np.int32)
    levels = OA.hierarchy(np.asarray(val)[perm], nbr_m, 1.0)
    f2 = np.asarray(f, dtype=np.float64).reshape(perm.size, -1)
    u = np.empty_like(f2)
    its, rels = [], []
    for c in range(f2.shape[1]):
        x, it, rel = OA.solve_refined(levels, np.ascontiguousarray(f2[perm, c]), rtol)
        u[perm, c] = x
        its.append(it)
        rels.append(rel)
    return u.reshape(np.shape(f)), its, rels


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def backward_ok(val, nbr, u, f, rtol: float) -> bool:
    """The GPU solution's residual with the oracle's FP64 operator meets rtol, up
    to what the GPU's own residual cannot see: its weights differ from the
    oracle's by at most 2^-48 relative (hi + lo of the FP64 weight) plus the FP64
    rounding of a (k+2)-term sum, so |r_or - r_gpu| <= 2^-46 |L| |u| row by row."""
    import oracle
    u = np.asarray(u, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    r = f - oracle.spmv(val, nbr, u, sigma=1.0)
    slack = oracle.spmv(np.abs(val), nbr, np.abs(u), sigma=0.0, alpha=-1.0)  # |L| |u|
    return bool(np.linalg.norm(r) <= rtol * np.linalg.norm(f) + 2.0 ** -46 * np.linalg.norm(slack))
