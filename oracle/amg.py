"""Aggregation multigrid for (sigma I - L) -- TEST INFRASTRUCTURE ONLY (FP64).

The paper solves its MVGD systems with algebraic multigrid (Sec. 4.2, with its
CPU-time table) but does not say which variant.  The CUDA path
uses plain (unsmoothed) aggregation multigrid as a right preconditioner of
BiCGSTAB; this module restates that preconditioner step by step from its
definition, in FP64, so that the GPU hierarchy and V-cycle can be compared
against it.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU leg may import it; it shares no code with the CUDA path.

Definitions (Braess 1995 for plain aggregation; Baker, Falgout, Kolev and Yang
2011 for the l1-Jacobi smoother):

* level 0 is A = sigma I - L in the operator's stored row order;
* an aggregate is `agg` consecutive rows of a level; the prolongation P is
  piecewise constant (P[i, i // agg] = 1) and the next level is the Galerkin
  product P^T A P, i.e. entry (I, J) is the sum of a_ij over rows i of
  aggregate I and columns j of aggregate J;
* coarsening stops at the first level with at most `coarsest` rows, which is
  solved exactly (its dense inverse);
* the smoother is one Jacobi step x += D^-1 (b - A x) with a per-row choice
  of D: d_i = OMEGA / a_ii on rows whose diagonal is strong (a_ii > THETA
  sum_j |a_ij|), and the l1 scaling d_i = 1 / sum_j |a_ij| elsewhere (rows with
  a small or non-positive diagonal, which MVGD rows with few neighbours on
  irregular samples do have);
* one V-cycle on b: y = D^-1 b (pre-smoothing from zero), r = b - A y,
  x_c = V-cycle of the next level on P^T r, x = y + P x_c, then one
  post-smoothing step x += D^-1 (b - A x).
"""
from __future__ import annotations

import numpy as np

AGG = 8
COARSEST = 512
OMEGA = 0.9   # damping of the Jacobi step on diagonally strong rows
THETA = 0.3   # a row is diagonally strong when a_ii > THETA * sum_j |a_ij|


class Level:
    """One level: a sparse matrix as (rows, cols, vals) sorted by (row, col),
    without duplicate entries, plus its diagonal, its row l1 norms and the
    smoother's scaling d.  Duplicate (row, col) entries are summed; the
    products use the same entries as a scipy CSR matrix (a library sparse
    product, FP64)."""

    def __init__(self, n: int, rows, cols, vals):
        import scipy.sparse as sp
        self.n = int(n)
        rows = np.asarray(rows, dtype=np.int64)
        cols = np.asarray(cols, dtype=np.int64)
        vals = np.asarray(vals, dtype=np.float64)
        m = sp.coo_matrix((vals, (rows, cols)), shape=(self.n, self.n)).tocsr()
        m.sum_duplicates()
        m.sort_indices()
        self.csr = m
        self.rows = np.repeat(np.arange(self.n, dtype=np.int64), np.diff(m.indptr))
        self.cols = m.indices.astype(np.int64)
        self.vals = m.data
        self.l1 = np.asarray(abs(m).sum(axis=1)).ravel()
        self.diag = m.diagonal().astype(np.float64)
        strong = self.diag > THETA * self.l1
        self.d = np.where(strong, OMEGA / np.where(strong, self.diag, 1.0), 1.0 / self.l1)

    def matvec(self, x: np.ndarray) -> np.ndarray:
        return self.csr @ x

    def dense(self) -> np.ndarray:
        A = np.zeros((self.n, self.n))
        A[self.rows, self.cols] = self.vals
        return A

    def width(self) -> int:
        return int(np.diff(self.csr.indptr).max()) if self.n else 0


def fine_level(val: np.ndarray, nbr: np.ndarray, sigma: float = 1.0) -> Level:
    """A = sigma I - L from the MVGD rows (slot 0 = the point itself)."""
    n, k = nbr.shape
    rows = np.repeat(np.arange(n), k + 1)
    cols = np.concatenate([np.arange(n)[:, None], nbr.astype(np.int64)], axis=1).ravel()
    vals = -np.asarray(val, dtype=np.float64).ravel()
    rows = np.concatenate([rows, np.arange(n)])
    cols = np.concatenate([cols, np.arange(n)])
    vals = np.concatenate([vals, np.full(n, float(sigma))])
    return Level(n, rows, cols, vals)


def galerkin(A: Level, agg: int = AGG) -> Level:
    """P^T A P for the piecewise-constant P over `agg` consecutive rows."""
    nc = (A.n + agg - 1) // agg
    return Level(nc, A.rows // agg, A.cols // agg, A.vals)


def hierarchy(val, nbr, sigma: float = 1.0, agg: int = AGG, coarsest: int = COARSEST) -> list:
    """Levels 0..m; the last one has at most `coarsest` rows."""
    levels = [fine_level(val, nbr, sigma)]
    while levels[-1].n > coarsest:
        levels.append(galerkin(levels[-1], agg))
    return levels


def coarsest_inverse(levels) -> np.ndarray:
    return np.linalg.inv(levels[-1].dense())


def vcycle(levels, b: np.ndarray, agg: int = AGG, inv: np.ndarray | None = None, lvl: int = 0) -> np.ndarray:
    """One V(1,1)-cycle applied to b (a vector of level `lvl`)."""
    A = levels[lvl]
    if lvl == len(levels) - 1:
        X = coarsest_inverse(levels) if inv is None else inv
        return X @ b
    d = A.d
    y = d * b
    r = b - A.matvec(y)
    bc = np.bincount(np.arange(A.n) // agg, weights=r, minlength=levels[lvl + 1].n)
    xc = vcycle(levels, bc, agg, inv, lvl + 1)
    x = y + xc[np.arange(A.n) // agg]
    return x + d * (b - A.matvec(x))


def bicgstab_right(levels, f: np.ndarray, rtol: float = 1e-8, maxit: int = 5000, agg: int = AGG):
    """Right-preconditioned BiCGSTAB on the level-0 matrix with one V-cycle per
    preconditioner application; returns (x, iterations, relative residual)."""
    A = levels[0]
    inv = coarsest_inverse(levels)
    M = lambda v: vcycle(levels, v, agg, inv)
    x = np.zeros_like(f)
    r = f.copy()
    rh = r.copy()
    fn = np.linalg.norm(f)
    rho = alpha = omega = 1.0
    p = np.zeros_like(f)
    v = np.zeros_like(f)
    for it in range(1, maxit + 1):
        rho1 = rh @ r
        beta = (rho1 / rho) * (alpha / omega)
        p = r + beta * (p - omega * v)
        ph = M(p)
        v = A.matvec(ph)
        alpha = rho1 / (rh @ v)
        s = r - alpha * v
        sh = M(s)
        t = A.matvec(sh)
        omega = (t @ s) / (t @ t)
        x = x + alpha * ph + omega * sh
        r = s - omega * t
        rho = rho1
        if np.linalg.norm(r) <= rtol * fn:
            break
    return x, it, np.linalg.norm(f - A.matvec(x)) / fn


def solve_refined(levels, f: np.ndarray, rtol: float = 1e-12, inner_rtol: float = 1e-7, max_outer: int = 8,
                  maxit: int = 5000, agg: int = AGG):
    """A reference solution of A x = f (A = level 0) to a tight relative residual:
    FP64 iterative refinement around the preconditioned BiCGSTAB above.  Each
    pass solves A dx = f - A x to `inner_rtol` and adds dx; the true residual is
    recomputed in FP64 every pass, so the recursive residual's drift in a long
    Krylov run cannot stop the result short of `rtol`.  Returns (x, total
    iterations, final relative residual)."""
    A = levels[0]
    fn = np.linalg.norm(f)
    x = np.zeros_like(f)
    total = 0
    rel = 1.0
    for _ in range(max_outer):
        r = f - A.matvec(x)
        rel = np.linalg.norm(r) / fn
        if rel <= rtol:
            break
        dx, it, _ = bicgstab_right(levels, r, rtol=inner_rtol, maxit=maxit, agg=agg)
        x = x + dx
        total += it
    else:
        rel = np.linalg.norm(f - A.matvec(x)) / fn
    return x, total, rel
