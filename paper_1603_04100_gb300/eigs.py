"""Lowest eigenpairs of the discrete LB operator (Sec. 4.3: -Delta_S v = lambda v).

Shift-invert subspace iteration on A = sigma I - L, whose smallest eigenvalues
1 + lambda belong to the smallest lambda:
  Y = A^-1 X           p/8 calls of mvgd_solve, 8 right-hand sides each, with the
                       multigrid preconditioner built once (mvgd_amg_setup);
  X = orthonormal(Y)   Cholesky QR twice: G = Y^T Y (mvgd_block_gram),
                       X = Y R^-1 (mvgd_block_combine);
  H = X^T (L X)        mvgd_spmv with sigma = 0, alpha = -1 per block, then a Gram;
and the Ritz values of the p x p matrix H estimate the eigenvalues of L
(lambda = -theta).  Every O(n) step runs in the library's kernels; the p x p
Cholesky inverse and the Ritz values of H (p <= 128) run in the library's host
code (mvgd_block_chol_inverse, mvgd_ritz_values), as in reverse-communication
eigensolvers.  The operator is not
symmetric, so H is not either; its eigenvalues near a multiplet of the
sphere come out real up to rounding, and their real parts are reported.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as LB
from . import api

W = 8  # columns per block: the solver's right-hand-side limit


def _rows(n: int) -> int:
    """Rows of a block: n rounded up to a multiple of 4, so that every block of
    8 FP64 columns starts on the 256-byte boundary the library's entry points
    require; the extra rows stay zero and add nothing to any Gram matrix."""
    return (n + 3) // 4 * 4


@dataclass
class EigResult:
    values: np.ndarray      # the nev smallest lambda, ascending
    vectors: torch.Tensor   # [p/8][n][8] orthonormal basis of the converged subspace (stored order; a view)
    iterations: int
    change: float           # largest relative change of the nev values in the last iteration
    solves: int             # mvgd_solve calls made


def _blocks(n: int, p: int, device) -> torch.Tensor:
    return torch.zeros((p // W, _rows(n), W), dtype=torch.float64, device=device)


class _Kit:
    """Gram and combination calls on block-major [p/8][n][8] sets."""

    def __init__(self, n: int, p: int, device, stream):
        self.L = LB.load()
        self.n, self.p, self.dev = _rows(n), p, device
        self.s = api._stream(stream)
        self.ws = torch.empty(self.L.mvgd_block_gram_workspace_bytes(p, p), dtype=torch.uint8, device=device)
        self.G = torch.empty((p, p), dtype=torch.float64, device=device)
        self.Cm = torch.empty((p, p), dtype=torch.float64, device=device)

    def gram(self, X: torch.Tensor, Y: torch.Tensor) -> np.ndarray:
        LB.check("mvgd_block_gram", self.L.mvgd_block_gram(api._vp(X), self.p, api._vp(Y), self.p, self.n, W,
                                                            api._vp(self.G), api._vp(self.ws), self.ws.numel(),
                                                            self.s))
        return self.G.cpu().numpy()

    def combine(self, X: torch.Tensor, Cm: np.ndarray, Y: torch.Tensor) -> None:
        self.Cm.copy_(torch.from_numpy(np.ascontiguousarray(Cm)))
        LB.check("mvgd_block_combine", self.L.mvgd_block_combine(api._vp(X), self.p, api._vp(self.Cm), self.p,
                                                                  self.n, W, api._vp(Y), self.s))

    def orthonormalize(self, Y: torch.Tensor, X: torch.Tensor) -> None:
        """X = Y R^-1 with R^T R = Y^T Y, twice (the second pass restores orthogonality)."""
        src = Y
        for _ in range(2):
            G = np.ascontiguousarray(self.gram(src, src))
            Rinv = np.empty((self.p, self.p))
            LB.check("mvgd_block_chol_inverse", self.L.mvgd_block_chol_inverse(
                G.ctypes.data_as(C.c_void_p), self.p, Rinv.ctypes.data_as(C.c_void_p)))
            dst = X if src is Y else Y
            self.combine(src, Rinv, dst)
            src = dst
        if src is not X:
            X.copy_(src)


def lowest_eigenpairs(op: api.Operator, nev: int, *, extra: int = 8, sigma: float = 1.0, tol: float = 1e-8,
                      maxit: int = 200, rtol_solve: float = 1e-10, seed: int = 0, stream=None,
                      boundary: torch.Tensor | None = None) -> EigResult:
    """The nev smallest eigenvalues lambda of -L (op assembled in stored order).

    boundary (uint8 [n], point order, as given to mvgd_dirichlet_rows on op): the
    Dirichlet problem -- the spectrum of L on the interior points with v = 0 on the
    boundary.  The basis is kept at zero on the boundary rows (a solve with zero
    right-hand side there returns zero up to its tolerance; the rows are re-zeroed
    after each solve, since A^-1 amplifies them by 1 / sigma against 1 / (sigma + lambda))."""
    p = ((nev + extra + W - 1) // W) * W
    if p > 128:
        raise ValueError("nev + extra must be at most 128")
    dev = op.col.device
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    mask = None
    if boundary is not None:  # the mask in stored row order, padded like the blocks
        m = boundary[op.order.long()] if op.order is not None else boundary
        mask = torch.zeros(_rows(op.n), dtype=torch.uint8, device=m.device)
        mask[:op.n] = m
    with torch.cuda.stream(st):  # torch's copies and the library's calls on one stream
        return _iterate(op, nev, p, st, sigma, tol, maxit, rtol_solve, seed, mask)


def _iterate(op, nev, p, st, sigma, tol, maxit, rtol_solve, seed, mask) -> EigResult:
    n, dev = op.n, op.col.device
    # every vector stays in stored row order: the products read it so, and the
    # solves are told there is no point order to map from
    op = dataclasses.replace(op, order=None)
    kit = _Kit(n, p, dev, st)
    L = LB.load()
    H_amg = api.amg_setup(op, sigma, stream=st)
    X = _blocks(n, p, dev)
    Y = _blocks(n, p, dev)
    Z = _blocks(n, p, dev)
    X[:, :n].copy_(torch.from_numpy(np.random.default_rng(seed).standard_normal((p // W, n, W))))

    def off_boundary(V):
        if mask is not None:
            LB.check("mvgd_block_zero_rows", L.mvgd_block_zero_rows(api._vp(V), p, kit.n, W, api._vp(mask),
                                                                    api._stream(st)))

    off_boundary(X)
    kit.orthonormalize(X.clone(), X)
    prev = None
    change = np.inf
    solves = 0
    it = 0
    for it in range(1, maxit + 1):
        for b in range(p // W):  # Y = (sigma I - L)^-1 X
            res = api.solve(op, X[b, :n], rtol=rtol_solve, amg=H_amg, stream=st)
            if any(s != LB.OK for s in res.status):
                raise LB.MvgdError("mvgd_solve (shift-invert)", max(res.status))
            Y[b, :n].copy_(res.u)
            solves += 1
        off_boundary(Y)
        kit.orthonormalize(Y, X)
        mode = LB.SPMV_F64 if op.prec == LB.FP64 else LB.SPMV_F64_HILO  # FP64 (or hi + lo) weights
        for b in range(p // W):  # Z = L X
            c = op.cstruct()
            LB.check("mvgd_spmv", L.mvgd_spmv(C.byref(c), mode, W, 0.0, -1.0, api._vp(X[b, :n]), 0.0,
                                                api._vp(Z[b, :n]), api._stream(st)))
        Hm = np.ascontiguousarray(kit.gram(X, Z))
        re, im = np.empty(p), np.empty(p)
        LB.check("mvgd_ritz_values", L.mvgd_ritz_values(Hm.ctypes.data_as(C.c_void_p), p,
                                                          re.ctypes.data_as(C.c_void_p), im.ctypes.data_as(C.c_void_p)))
        lam = np.sort(-re)[:nev]
        if prev is not None:
            change = float(np.max(np.abs(lam - prev) / np.maximum(np.abs(lam), 1.0)))
            if change <= tol:
                break
        prev = lam
    return EigResult(values=lam, vectors=X[:, :n], iterations=it, change=change, solves=solves)
