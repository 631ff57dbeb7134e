"""FP64 CPU oracle for the MVGD hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``mvgd_oracle.c`` (plain C,
FP64, no FMA contraction) with ctypes and numpy arrays; it shares no code with
the CUDA path.

Functions (each mirrors one C entry point; see the C file for the passages of
the paper they follow):

* ``knn_brute(pts, k)`` / ``knn_grid(pts, k)``: K nearest neighbours, key
  (squared distance, index); the grid variant gives the same lists faster.
* ``assemble(pts, nbr, delta, variant)``: MVGD (or plain least-squares) rows,
  [n][k+1] with slot 0 = the point itself.
* ``spmv``, ``bicgstab``, ``gmres``: y = alpha (sigma x - L x) + beta y and
  solvers of (sigma I - L) u = f.
* ``line_weights``: the 1-D worked example of Sec. 3.2.
* ``row_sign_counts``: the M-matrix sign pattern of rows (Sec. 3.2, Sec. 4.1).
* ``dirichlet_rows``: boundary rows of open surfaces (Sec. 3.1).
* ``lb_eigenvalues``, ``multiplet_errors``: the lowest LB eigenvalues and the
  error measures of Sec. 4.3.
* ``normal_matrix``: the 6x6 normal-equation matrix of Sec. 2 as printed.
* ``system_matrix``, ``gs_eigenvalues``, ``gs_power``: sigma I - L in a given
  row order and the spectrum of its Gauss-Seidel iteration matrix (Sec. 4.1).
* ``neumann_ghosts``, ``neumann_fold``, ``neumann_rhs`` (``oracle/neumann.py``):
  the reflection method for a Neumann boundary (Sec. 3.1).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build
from .neumann import fold as neumann_fold  # noqa: F401
from .neumann import neumann_ghosts  # noqa: F401
from .neumann import neumann_rhs  # noqa: F401

DELTA_QUARTER_RANGE = 0
DELTA_MEAN_NN = 1
VARIANT_MVGD = 0
VARIANT_LS = 1
DIAG_FIELDS = ("A1", "A2", "A3", "A4", "A5", "h", "nx", "ny", "nz", "gap", "rank")

_lib = None
_P = C.c_void_p


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(str(path))
        L.or_threads.argtypes = [C.c_int]; L.or_threads.restype = C.c_int
        L.or_knn_brute.argtypes = [_P, C.c_int64, C.c_int, _P]; L.or_knn_brute.restype = C.c_int
        L.or_knn_grid.argtypes = [_P, C.c_int64, C.c_int, _P]; L.or_knn_grid.restype = C.c_int
        L.or_assemble.argtypes = [_P, C.c_int64, C.c_int, _P, C.c_int, C.c_int, C.c_double,
                                  C.c_int, _P, _P, _P, _P]
        L.or_assemble.restype = C.c_int
        L.or_spmv.argtypes = [_P, _P, C.c_int64, C.c_int, C.c_int, C.c_double, C.c_double, _P,
                              C.c_double, _P]
        L.or_spmv.restype = None
        L.or_bicgstab.argtypes = [_P, _P, C.c_int64, C.c_int, C.c_double, _P, _P, C.c_double,
                                  C.c_int, _P]
        L.or_bicgstab.restype = C.c_int
        L.or_gmres.argtypes = [_P, _P, C.c_int64, C.c_int, C.c_double, _P, _P, C.c_double,
                               C.c_int, C.c_int, _P]
        L.or_gmres.restype = C.c_int
        L.or_line_weights.argtypes = [_P, C.c_int, C.c_int, C.c_double, C.c_int, _P]
        L.or_line_weights.restype = C.c_int
        L.or_normal_matrix.argtypes = [_P, _P, C.c_int, _P]; L.or_normal_matrix.restype = None
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def threads(n: int = 0) -> int:
    """Set (n > 0) and return the OpenMP thread count the oracle uses."""
    return lib().or_threads(int(n))


def knn_brute(pts, k: int) -> np.ndarray:
    pts = _f64(pts)
    nbr = np.empty((pts.shape[0], k), dtype=np.int32)
    if lib().or_knn_brute(_ptr(pts), pts.shape[0], k, _ptr(nbr)) != 0:
        raise ValueError("or_knn_brute: bad arguments")
    return nbr


def knn_grid(pts, k: int) -> np.ndarray:
    pts = _f64(pts)
    nbr = np.empty((pts.shape[0], k), dtype=np.int32)
    if lib().or_knn_grid(_ptr(pts), pts.shape[0], k, _ptr(nbr)) != 0:
        raise ValueError("or_knn_grid: bad arguments")
    return nbr


def assemble(pts, nbr, delta_kind: int = DELTA_MEAN_NN, delta_m: int = 6,
             delta_scale: float = 1.0, variant: int = VARIANT_MVGD, want_p00: bool = False):
    """Returns (val [n][k+1], status [n] uint8, diag [n][11], p00 or None)."""
    pts = _f64(pts)
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    n, k = nbr.shape
    val = np.empty((n, k + 1))
    status = np.empty(n, dtype=np.uint8)
    diag = np.empty((n, len(DIAG_FIELDS)))
    p00 = np.empty((n, k + 1)) if want_p00 else None
    rc = lib().or_assemble(_ptr(pts), n, k, _ptr(nbr), delta_kind, delta_m, delta_scale, variant,
                           _ptr(val), _ptr(status), _ptr(diag),
                           _ptr(p00) if p00 is not None else None)
    if rc == 1:
        raise ValueError("or_assemble: bad arguments")
    return val, status, diag, p00


def spmv(val, nbr, x, sigma: float = 1.0, alpha: float = 1.0, beta: float = 0.0, y=None):
    val = _f64(val)
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    x = _f64(x)
    n, k = nbr.shape
    x2 = x.reshape(n, -1)
    nr = x2.shape[1]
    out = np.zeros_like(x2) if y is None else _f64(y).reshape(n, nr).copy()
    lib().or_spmv(_ptr(val), _ptr(nbr), n, k, nr, sigma, alpha, _ptr(x2), beta, _ptr(out))
    return out.reshape(x.shape)


def bicgstab(val, nbr, f, sigma: float = 1.0, rtol: float = 1e-13, maxit: int = 100000, x0=None):
    """Solve (sigma I - L) u = f for one right-hand side; returns (u, iters, relres, status)."""
    val = _f64(val)
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    f = _f64(f).ravel()
    x = np.zeros_like(f) if x0 is None else _f64(x0).ravel().copy()
    info = np.zeros(2)
    st = lib().or_bicgstab(_ptr(val), _ptr(nbr), nbr.shape[0], nbr.shape[1], sigma, _ptr(f),
                           _ptr(x), rtol, maxit, _ptr(info))
    return x, int(info[0]), float(info[1]), st


def gmres(val, nbr, f, sigma: float = 1.0, rtol: float = 1e-13, maxit: int = 100000,
          restart: int = 50, x0=None):
    val = _f64(val)
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    f = _f64(f).ravel()
    x = np.zeros_like(f) if x0 is None else _f64(x0).ravel().copy()
    info = np.zeros(2)
    st = lib().or_gmres(_ptr(val), _ptr(nbr), nbr.shape[0], nbr.shape[1], sigma, _ptr(f),
                        _ptr(x), rtol, maxit, min(int(restart), 1024), _ptr(info))
    return x, int(info[0]), float(info[1]), st


def solve(val, nbr, f, sigma: float = 1.0, rtol: float = 1e-13, maxit: int = 100000):
    """Column-by-column BiCGSTAB for f of shape [n] or [n][r]."""
    f2 = _f64(f).reshape(nbr.shape[0], -1)
    u = np.empty_like(f2)
    its, res = [], []
    for c in range(f2.shape[1]):
        u[:, c], it, rr, st = bicgstab(val, nbr, f2[:, c], sigma, rtol, maxit)
        its.append(it)
        res.append(rr)
    return u.reshape(np.shape(f)), its, res


def line_weights(xs, c: int, h: float, variant: int = VARIANT_MVGD) -> np.ndarray:
    xs = _f64(xs)
    w = np.empty(xs.shape[0])
    if lib().or_line_weights(_ptr(xs), xs.shape[0], c, h, variant, _ptr(w)) != 0:
        raise ValueError("or_line_weights: bad arguments")
    return w


def row_sign_counts(val) -> tuple:
    """Sign pattern of MVGD rows [n][k+1] (slot 0 = the point itself), Sec. 3.2 and
    Sec. 4.1: (rows whose neighbour weights are all >= 0 -- with zero row sums the
    M-matrix pattern of sigma I - L --, neighbour weights < 0, rows whose self
    weight is >= 0)."""
    val = _f64(val)
    nbrs = val[:, 1:]
    return (int(np.count_nonzero(np.all(nbrs >= 0.0, axis=1))), int(np.count_nonzero(nbrs < 0.0)),
            int(np.count_nonzero(val[:, 0] >= 0.0)))


def dirichlet_rows(val, boundary) -> np.ndarray:
    """Open surfaces with U = g on the boundary (Sec. 3.1): the rows [n][k+1] of the
    boundary points become zero, so those rows of sigma I - L read sigma u_i = f_i,
    and every interior row keeps its MVGD weights."""
    out = np.array(val, dtype=np.float64, copy=True)
    out[np.asarray(boundary).astype(bool)] = 0.0
    return out


def lb_eigenvalues(val, nbr, nev: int, shift: float = 0.5, boundary=None) -> np.ndarray:
    """The nev smallest eigenvalues lambda of -L (Sec. 4.3), as the paper takes them:
    a sparse eigensolver on the assembled matrix (ARPACK in shift-invert mode about
    lambda = -shift).  Real parts, ascending; the matrix is not symmetric, so a
    multiplet can carry small imaginary parts.  With a boundary mask: the Dirichlet
    problem, L restricted to the interior rows and columns."""
    import scipy.sparse.linalg as spl
    Lm = to_csr(val, nbr).tocsr()
    if boundary is not None:
        inner = np.flatnonzero(np.asarray(boundary) == 0)
        Lm = Lm[inner][:, inner]
    Lm = Lm.tocsc()
    w = spl.eigs(Lm, k=nev, sigma=shift, which="LM", return_eigenvectors=False)
    return np.sort(-w.real)


def multiplet_errors(lams, n: int) -> tuple:
    """E^2_n and E^inf_n of Sec. 4.3 for the sphere's n-th eigenvalue n (n + 1),
    multiplicity 2n + 1: relative errors of the eigenvalues n^2 .. n^2 + 2n of the
    ascending list lams (RMS and maximum)."""
    lam = n * (n + 1.0)
    r = (np.asarray(lams, dtype=np.float64)[n * n:n * n + 2 * n + 1] - lam) / lam
    return float(np.sqrt(np.mean(r * r))), float(np.abs(r).max())


def system_matrix(val, nbr, sigma: float = 1.0, order=None):
    """sigma I - L as scipy CSR with rows and columns in stored order: stored row r
    is point order[r] (order None: point r), so the result is P (sigma I - L) P^T."""
    import scipy.sparse as sp
    A = (sigma * sp.identity(nbr.shape[0], format="csr") - to_csr(val, nbr)).tocsr()
    if order is not None:
        o = np.asarray(order, dtype=np.int64)
        A = A[o][:, o].tocsr()
    return A


def gs_eigenvalues(A) -> np.ndarray:
    """Eigenvalues of the Gauss-Seidel iteration matrix M^-1 N of A (Sec. 4.1), where
    A = M + N with N the strictly upper triangle of A.  Dense: small n only."""
    import scipy.linalg as sl
    Ad = A.toarray() if hasattr(A, "toarray") else np.asarray(A, dtype=np.float64)
    T = sl.solve_triangular(np.tril(Ad), np.triu(Ad, 1), lower=True)
    return np.linalg.eigvals(T)


def gs_power(A, x0, iters: int) -> tuple:
    """Power iteration on M^-1 N (Sec. 4.1): x_0 = x0 / ||x0||, y_t = M^-1 (N x_t),
    nu_t = ||y_t||, x_{t+1} = y_t / nu_t.  Returns (nu [iters], x_iters)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    A = sp.csr_matrix(A)
    M = sp.tril(A, 0, format="csr")
    N = sp.triu(A, 1, format="csr")
    x = np.asarray(x0, dtype=np.float64) / np.linalg.norm(x0)
    nu = np.empty(iters)
    for t in range(iters):
        y = spl.spsolve_triangular(M, N @ x, lower=True)
        nu[t] = np.linalg.norm(y)
        x = y / nu[t]
    return nu, x


def normal_matrix(x, y) -> np.ndarray:
    x, y = _f64(x), _f64(y)
    A = np.empty((6, 6))
    lib().or_normal_matrix(_ptr(x), _ptr(y), x.shape[0], _ptr(A))
    return A


def to_csr(val, nbr):
    """scipy CSR of L (test helper: an independent product for pins)."""
    import scipy.sparse as sp
    n, k = nbr.shape
    rows = np.repeat(np.arange(n), k + 1)
    cols = np.concatenate([np.arange(n)[:, None], nbr], axis=1).ravel()
    return sp.csr_matrix((np.asarray(val).ravel(), (rows, cols)), shape=(n, n))
