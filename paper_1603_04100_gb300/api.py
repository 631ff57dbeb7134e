"""PyTorch-facing API over the C ABI: tensors supply device memory and streams,
every step of the path runs in libmvgd's CUDA kernels.

    nbr, order = knn(pts, k, want_order=True)
    op = assemble(pts, nbr, prec=FP32_REFINE, order=order)
    u, info = solve(op, f, rtol=1e-8)
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib as LB
from ._lib import (DELTA_MEAN_NN, DELTA_QUARTER_RANGE, FP32_REFINE, FP64, SPMV_F32, SPMV_F64,  # noqa: F401
                   SPMV_F64_HILO, ROW_LS, ROW_MVGD, MvgdError)

SLICE = 32


def _vp(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _require_cuda(t: torch.Tensor, dtype, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def n_padded(n: int) -> int:
    return (n + SLICE - 1) // SLICE * SLICE


def knn(pts: torch.Tensor, k: int, *, want_order: bool = False, cell_size: float = 0.0, stream=None,
        workspace: torch.Tensor | None = None):
    """K nearest neighbours (int32 [n][k], ascending (d2, index)); optionally a locality order."""
    _require_cuda(pts, torch.float64, "pts")
    n = pts.shape[0]
    L = LB.load()
    nbr = torch.empty((n, k), dtype=torch.int32, device=pts.device)
    order = torch.empty(n, dtype=torch.int32, device=pts.device) if want_order else None
    need = L.mvgd_knn_workspace_bytes(n, k)
    ws = workspace if workspace is not None and workspace.numel() >= need else _workspace(need, pts.device)
    LB.check("mvgd_knn", L.mvgd_knn(_vp(pts), n, k, _vp(nbr), _vp(order), float(cell_size), _vp(ws), ws.numel(),
                                     _stream(stream)))
    return (nbr, order) if want_order else nbr


@dataclass
class Operator:
    """The assembled MVGD operator L in sliced ELL form (device tensors)."""
    n: int
    k: int
    prec: int
    col: torch.Tensor
    val: torch.Tensor
    val_lo: torch.Tensor | None
    order: torch.Tensor | None = None
    h: torch.Tensor | None = None
    status: torch.Tensor | None = None
    bad_rows: torch.Tensor | None = None
    _c: LB.Ell = field(default=None, repr=False)

    def cstruct(self) -> LB.Ell:
        self._c = LB.Ell(self.n, self.k, self.prec, _vp(self.order), _vp(self.col), _vp(self.val),
                         _vp(self.val_lo))
        return self._c

    def rows(self, which: str = "val") -> np.ndarray:
        """Host copy [n][k+1] (val / val_lo) or [n][k] (col), stored row order."""
        t = {"val": self.val, "val_lo": self.val_lo, "col": self.col}[which]
        w = self.k if which == "col" else self.k + 1
        return sell_to_rows(t.cpu().numpy(), self.n, w)

    def weights(self) -> np.ndarray:
        """FP64 weights [n][k+1] in stored row order (hi + lo in the mixed format)."""
        v = self.rows("val").astype(np.float64)
        if self.prec == FP32_REFINE:
            v = v + self.rows("val_lo").astype(np.float64)
        return v


def sell_to_rows(a: np.ndarray, n: int, w: int) -> np.ndarray:
    """Sliced-ELL storage (slice height 32, slot-major inside a slice) -> [n][w]."""
    npad = n_padded(n)
    return a[: npad * w].reshape(npad // SLICE, w, SLICE).transpose(0, 2, 1).reshape(npad, w)[:n]


def ell_alloc(n: int, k: int, prec: int, device) -> tuple:
    L = LB.load()
    col = torch.empty(L.mvgd_ell_bytes(n, k, prec, LB.ELL_COL) // 4, dtype=torch.int32, device=device)
    vdt = torch.float64 if prec == FP64 else torch.float32
    vbytes = L.mvgd_ell_bytes(n, k, prec, LB.ELL_VAL)
    val = torch.empty(vbytes // vdt.itemsize, dtype=vdt, device=device)
    lo = None
    if prec == FP32_REFINE:
        lo = torch.empty(L.mvgd_ell_bytes(n, k, prec, LB.ELL_VAL_LO) // 4, dtype=torch.float32, device=device)
    return col, val, lo


def assemble(pts: torch.Tensor, nbr: torch.Tensor, *, prec: int = FP64, order: torch.Tensor | None = None,
             delta_kind: int = DELTA_MEAN_NN, delta_m: int = 6, delta_scale: float = 1.0,
             want_h: bool = True, want_status: bool = True, stream=None, out: Operator | None = None,
             variant: int = LB.ROW_MVGD, arith: int = 0) -> Operator:
    """MVGD rows (Sec. 2, Sec. 3.1) for every point into a sliced ELL operator; variant
    ROW_LS forms the plain least-squares comparator rows instead.  FP32_REFINE rows are
    formed on the FP32 pipe (arith 0) or in FP64 arithmetic (arith 1)."""
    _require_cuda(pts, torch.float64, "pts")
    _require_cuda(nbr, torch.int32, "nbr")
    n, k = nbr.shape
    if order is not None:
        _require_cuda(order, torch.int32, "order")
    L = LB.load()
    if out is None:
        col, val, lo = ell_alloc(n, k, prec, pts.device)
        op = Operator(n, k, prec, col, val, lo, order)
        op.h = torch.empty(n, dtype=torch.float64, device=pts.device) if want_h else None
        op.status = torch.empty(n, dtype=torch.uint8, device=pts.device) if want_status else None
        op.bad_rows = torch.zeros(1, dtype=torch.int32, device=pts.device)
    else:
        op = out
        op.order = order
    need_ws = order is not None or (prec == FP32_REFINE and arith == 0)
    ws = _workspace(L.mvgd_assemble_workspace_bytes(n), pts.device) if need_ws else None
    rule = LB.DeltaRule(delta_kind, delta_m if delta_kind == DELTA_MEAN_NN else 0, float(delta_scale),
                        int(variant), int(arith))
    c = op.cstruct()
    LB.check("mvgd_assemble", L.mvgd_assemble(_vp(pts), n, k, _vp(nbr), rule, C.byref(c), _vp(op.h),
                                               _vp(op.status), _vp(op.bad_rows), _vp(ws),
                                               ws.numel() if ws is not None else 0, _stream(stream)))
    return op


def spmv(op: Operator, x: torch.Tensor, *, mode: int | None = None, sigma: float = 1.0, alpha: float = 1.0,
         beta: float = 0.0, y: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """y = alpha (sigma x - L x) + beta y, x and y [n] or [n][nrhs] in stored row order."""
    if mode is None:
        mode = SPMV_F64 if op.prec == FP64 else SPMV_F32
    dt = torch.float32 if mode == SPMV_F32 else torch.float64
    _require_cuda(x, dt, "x")
    nrhs = 1 if x.dim() == 1 else x.shape[1]
    if y is None:
        y = torch.empty_like(x)
        beta = 0.0
    L = LB.load()
    c = op.cstruct()
    LB.check("mvgd_spmv", L.mvgd_spmv(C.byref(c), mode, nrhs, sigma, alpha, _vp(x), beta, _vp(y), _stream(stream)))
    return y


def row_signs(op: Operator, stream=None) -> dict:
    """Sign pattern of the operator's rows (mvgd_row_signs): rows whose neighbour
    weights are all >= 0 (the M-matrix pattern of sigma I - L), negative
    neighbour weights, rows with a non-negative self weight."""
    counts = torch.zeros(3, dtype=torch.int64, device=op.col.device)
    c = op.cstruct()
    LB.check("mvgd_row_signs", LB.load().mvgd_row_signs(C.byref(c), _vp(counts), _stream(stream)))
    m_rows, neg, self_nonneg = (int(v) for v in counts.cpu().tolist())
    return {"m_pattern_rows": m_rows, "negative_weights": neg, "nonneg_self_rows": self_nonneg, "rows": op.n}


def dirichlet_rows(op: Operator, boundary: torch.Tensor, stream=None) -> int:
    """Dirichlet rows (mvgd_dirichlet_rows): zero the rows of the points flagged in
    boundary (uint8 [n], point order), so those rows of sigma I - L read sigma u_i = f_i.
    Returns the number of rows zeroed."""
    _require_cuda(boundary, torch.uint8, "boundary")
    count = torch.zeros(1, dtype=torch.int32, device=op.col.device)
    c = op.cstruct()
    LB.check("mvgd_dirichlet_rows", LB.load().mvgd_dirichlet_rows(C.byref(c), _vp(boundary), _vp(count),
                                                                   _stream(stream)))
    return int(count.item())


@dataclass
class NeumannCloud:
    """Interior points and ghosts of a Neumann boundary (mvgd_neumann_ghosts, Sec. 3.1)."""
    q: torch.Tensor           # [n_interior + n_ghost][3]: interior points, then ghosts
    q_src: torch.Tensor       # int32 [n_interior + n_ghost]: the interior position each stands for
    interior: torch.Tensor    # int32 [n_interior]: point index of each interior position
    ghost_bnd: torch.Tensor   # int32 [n_ghost]: the boundary point each ghost was mirrored at
    ghost_dist: torch.Tensor  # [n_ghost]: |point - ghost|
    n_interior: int
    n_ghost: int
    n_boundary: int
    bad_frames: int
    op_q: "Operator | None" = None  # the operator over interior points and ghosts, before the fold


def neumann_ghosts(pts: torch.Tensor, nbr: torch.Tensor, boundary: torch.Tensor, kb: int = 6,
                   stream=None) -> NeumannCloud:
    """The ghosts of the interior points next to the boundary (mvgd_neumann_ghosts).
    pts, nbr (mvgd_knn of the whole cloud) and boundary (uint8) in point order."""
    _require_cuda(pts, torch.float64, "pts")
    _require_cuda(nbr, torch.int32, "nbr")
    _require_cuda(boundary, torch.uint8, "boundary")
    L = LB.load()
    n, k = nbr.shape
    dev = pts.device
    q = torch.empty((2 * n, 3), dtype=torch.float64, device=dev)
    q_src = torch.empty(2 * n, dtype=torch.int32, device=dev)
    interior = torch.empty(n, dtype=torch.int32, device=dev)
    gb = torch.empty(n, dtype=torch.int32, device=dev)
    gd = torch.empty(n, dtype=torch.float64, device=dev)
    counts = torch.zeros(4, dtype=torch.int32, device=dev)
    ws = torch.empty(L.mvgd_neumann_ghosts_workspace_bytes(n), dtype=torch.uint8, device=dev)
    LB.check("mvgd_neumann_ghosts", L.mvgd_neumann_ghosts(_vp(pts), n, k, _vp(nbr), _vp(boundary), kb, _vp(q),
                                                           _vp(q_src), _vp(interior), _vp(gb), _vp(gd),
                                                           _vp(counts), _vp(ws), ws.numel(), _stream(stream)))
    ni, ng, nb, bad = (int(v) for v in counts.cpu().tolist())
    return NeumannCloud(q=q[:ni + ng], q_src=q_src[:ni + ng], interior=interior[:ni], ghost_bnd=gb[:ng],
                        ghost_dist=gd[:ng], n_interior=ni, n_ghost=ng, n_boundary=nb, bad_frames=bad)


def neumann_fold(op_q: Operator, cloud: NeumannCloud, stream=None) -> Operator:
    """The interior rows of the operator assembled on cloud.q, every ghost column
    mapped to its point (mvgd_neumann_fold).  The result's order maps stored rows to
    interior positions, so its point order is the interior order of the cloud."""
    L = LB.load()
    dev = op_q.col.device
    ni = cloud.n_interior
    col, val, lo = ell_alloc(ni, op_q.k, op_q.prec, dev)
    out = Operator(ni, op_q.k, op_q.prec, col, val, lo, torch.empty(ni, dtype=torch.int32, device=dev))
    ws = torch.empty(L.mvgd_neumann_fold_workspace_bytes(op_q.n), dtype=torch.uint8, device=dev)
    cq, ci = op_q.cstruct(), out.cstruct()
    LB.check("mvgd_neumann_fold", L.mvgd_neumann_fold(C.byref(cq), _vp(cloud.q_src), C.byref(ci), _vp(ws),
                                                       ws.numel(), _stream(stream)))
    return out


def neumann_operator(pts: torch.Tensor, boundary: torch.Tensor, k: int, *, kb: int = 6, prec: int = FP64,
                     stream=None) -> tuple:
    """The MVGD operator of an open surface with dU/dn = 0 on its boundary (Sec. 3.1):
    kNN of the cloud, ghosts, kNN and assembly over interior points and ghosts, fold.
    Returns (operator over the interior points, NeumannCloud)."""
    nbr = knn(pts, k, stream=stream)
    cloud = neumann_ghosts(pts, nbr, boundary, kb, stream=stream)
    if cloud.bad_frames:
        raise LB.MvgdError("mvgd_neumann_ghosts", LB.EDEGENERATE)
    nq, oq = knn(cloud.q, k, want_order=True, stream=stream)
    cloud.op_q = assemble(cloud.q, nq, prec=prec, order=oq, stream=stream)
    return neumann_fold(cloud.op_q, cloud, stream=stream), cloud


def neumann_rhs(cloud: NeumannCloud, g: torch.Tensor, op_q: Operator | None = None, stream=None) -> torch.Tensor:
    """The term c that dU/dn = g adds to the right-hand side (mvgd_neumann_rhs):
    solve (sigma I - L_folded) u = f + c.  g: double [n], the original cloud's point
    order; op_q defaults to the operator neumann_operator assembled over the cloud."""
    _require_cuda(g, torch.float64, "g")
    op_q = op_q if op_q is not None else cloud.op_q
    if op_q is None:
        raise ValueError("no operator over the cloud: pass op_q")
    c = torch.empty(cloud.n_interior, dtype=torch.float64, device=g.device)
    cq = op_q.cstruct()
    LB.check("mvgd_neumann_rhs", LB.load().mvgd_neumann_rhs(C.byref(cq), cloud.n_interior, _vp(cloud.ghost_dist),
                                                            _vp(cloud.ghost_bnd), _vp(g), _vp(c),
                                                            _stream(stream)))
    return c


@dataclass
class GsPower:
    nu: np.ndarray        # [iters] ||T x_t|| for unit x_t
    x: torch.Tensor       # the last unit iterate, stored order
    status: int
    rho: float            # geometric mean of nu over the second half of the steps


def gs_power(op: Operator, x0: torch.Tensor, iters: int, sigma: float = 1.0, stream=None) -> GsPower:
    """Power iteration on the Gauss-Seidel iteration matrix of sigma I - L in stored
    row order (mvgd_gs_power, Sec. 4.1).  x0: double [n], stored order."""
    _require_cuda(x0, torch.float64, "x0")
    L = LB.load()
    dev = op.col.device
    nu = torch.empty(iters, dtype=torch.float64, device=dev)
    x = torch.empty(op.n, dtype=torch.float64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    ws = torch.empty(L.mvgd_gs_power_workspace_bytes(op.n, iters), dtype=torch.uint8, device=dev)
    c = op.cstruct()
    LB.check("mvgd_gs_power", L.mvgd_gs_power(C.byref(c), sigma, _vp(x0), iters, _vp(nu), _vp(x), _vp(status),
                                               _vp(ws), ws.numel(), _stream(stream)))
    nu_h = nu.cpu().numpy()
    tail = nu_h[iters // 2:]
    rho = float(np.exp(np.mean(np.log(tail)))) if np.all(tail > 0) else float("nan")
    return GsPower(nu=nu_h, x=x, status=int(status.item()), rho=rho)


@dataclass
class SolveResult:
    u: torch.Tensor
    iters: list
    outer: list
    relres: list
    status: list


def solve(op: Operator, f: torch.Tensor, *, u0: torch.Tensor | None = None, sigma: float = 1.0,
          rtol: float = 1e-8, maxit: int = 200000, inner_rtol: float = 1e-3, inner_maxit: int = 20000,
          max_outer: int = 60, precond: int = 0, cancel: torch.Tensor | None = None, stream=None,
          workspace: torch.Tensor | None = None, sync: bool = True, amg: "Hierarchy | None" = None) -> SolveResult:
    """Solve (sigma I - L) u = f; f, u FP64 [n] or [n][nrhs] in point order.

    precond 2 preconditions with one multigrid V-cycle: pass a Hierarchy built
    for this operator and sigma, or none to have the call build one."""
    if amg is not None:
        precond = LB.PRECOND_AMG
    _require_cuda(f, torch.float64, "f")
    nrhs = 1 if f.dim() == 1 else f.shape[1]
    u = torch.zeros_like(f) if u0 is None else u0.clone()
    L = LB.load()
    need = L.mvgd_solve_workspace_bytes(op.n, op.k, nrhs, op.prec, precond)
    if need == 0:
        raise ValueError("mvgd_solve_workspace_bytes: sizes out of range")
    if amg is not None:  # the caller's hierarchy: no room needed for one
        need -= (L.mvgd_amg_workspace_bytes(op.n, op.k) + 255) // 256 * 256
    ws = workspace if workspace is not None and workspace.numel() >= need else _workspace(need, f.device)
    opts = LB.SolveOpts(rtol, maxit, inner_maxit, inner_rtol, max_outer, precond,
                        _vp(amg.ws) if amg is not None else C.c_void_p(0))
    c = op.cstruct()
    if sync:
        info = (LB.SolveInfo * nrhs)()
        st = L.mvgd_solve(C.byref(c), nrhs, sigma, _vp(f), _vp(u), C.byref(opts), C.cast(info, C.c_void_p),
                          _vp(cancel), _vp(ws), ws.numel(), _stream(stream))
        if st in (LB.EINVAL, LB.EWORKSPACE, LB.ECUDA):
            raise MvgdError("mvgd_solve", st)
        return SolveResult(u, [i.iters for i in info], [i.outer for i in info], [i.relres for i in info],
                           [i.status for i in info])
    dinfo = torch.zeros(nrhs * C.sizeof(LB.SolveInfo), dtype=torch.uint8, device=f.device)
    LB.check("mvgd_solve", L.mvgd_solve(C.byref(c), nrhs, sigma, _vp(f), _vp(u), C.byref(opts), _vp(dinfo),
                                        _vp(cancel), _vp(ws), ws.numel(), _stream(stream)))
    return SolveResult(u, dinfo, None, None, None)


def decode_info(dinfo: torch.Tensor) -> list:
    raw = bytes(dinfo.cpu().numpy().tobytes())
    n = len(raw) // C.sizeof(LB.SolveInfo)
    arr = (LB.SolveInfo * n).from_buffer_copy(raw)
    return [(i.iters, i.outer, i.relres, i.status) for i in arr]


@dataclass
class Hierarchy:
    """Aggregation-multigrid hierarchy of sigma I - L (mvgd_amg_setup)."""
    n: int
    k: int
    sigma: float
    ws: torch.Tensor
    op: Operator

    def info(self, level: int) -> LB.AmgInfo:
        out = LB.AmgInfo()
        LB.check("mvgd_amg_describe", LB.load().mvgd_amg_describe(_vp(self.ws), level, C.byref(out)))
        return out

    @property
    def levels(self) -> int:
        return self.info(0).levels

    def level_rows(self, level: int):
        """Host copies of one level (stored order): level 0 -> (dinv,); above ->
        (cnt [n], col [n][stride], val64 [n][stride], val32 [n][stride], dinv [n])."""
        i = self.info(level)
        n = int(i.n)
        npad = n_padded(n)
        dev = self.ws.device

        def grab(ptr, count, dtype):
            return _device_view(ptr, count, dtype, dev).cpu().numpy()

        dinv = grab(i.dinv, n, torch.float32)
        if level == 0:
            return (dinv,)
        w = int(i.stride)
        cnt = grab(i.cnt, n, torch.int32)
        col = sell_to_rows(grab(i.col, npad * w, torch.int32), n, w)
        v64 = sell_to_rows(grab(i.val64, npad * w, torch.float64), n, w)
        v32 = sell_to_rows(grab(i.val, npad * w, torch.float32), n, w)
        return cnt, col, v64, v32, dinv

    def coarsest_inverse(self, fp64: bool = True) -> np.ndarray:
        """The coarsest level's inverse: the refined FP64 one the cycle uses, or the FP32 Gauss-Jordan one."""
        i = self.info(self.levels - 1)
        n = int(i.n)
        if fp64:
            return _device_view(i.cinv64, n * n, torch.float64, self.ws.device).cpu().numpy().reshape(n, n)
        # stored column-major
        return _device_view(i.cinv, n * n, torch.float32, self.ws.device).cpu().numpy().reshape(n, n).T.copy()

    def apply(self, b: torch.Tensor, stream=None) -> torch.Tensor:
        """x = one V-cycle applied to b (FP64 [n] or [n][nrhs], stored order)."""
        _require_cuda(b, torch.float64, "b")
        nrhs = 1 if b.dim() == 1 else b.shape[1]
        L = LB.load()
        x = torch.empty_like(b)
        ws = _workspace(L.mvgd_amg_apply_workspace_bytes(self.n, nrhs), b.device)
        LB.check("mvgd_amg_apply", L.mvgd_amg_apply(_vp(self.ws), self.n, nrhs, _vp(b), _vp(x), _vp(ws), ws.numel(),
                                                     _stream(stream)))
        return x


class _DeviceArray:
    """A raw device pointer seen through __cuda_array_interface__ (callers only read it)."""

    def __init__(self, ptr: int, count: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3}


def _device_view(ptr, count: int, dtype, device) -> torch.Tensor:
    typestr = {torch.float32: "<f4", torch.float64: "<f8", torch.int32: "<i4"}[dtype]
    p = ptr.value if hasattr(ptr, "value") else ptr
    if not p:
        raise ValueError("null device pointer")
    return torch.as_tensor(_DeviceArray(p, count, typestr), device=device)


def amg_setup(op: Operator, sigma: float = 1.0, stream=None) -> Hierarchy:
    """Build the multigrid hierarchy of sigma I - L for operator op."""
    L = LB.load()
    nbytes = L.mvgd_amg_workspace_bytes(op.n, op.k)
    if nbytes == 0:
        raise ValueError("mvgd_amg_workspace_bytes: sizes out of range")
    ws = _workspace(nbytes, op.col.device)
    c = op.cstruct()
    LB.check("mvgd_amg_setup", L.mvgd_amg_setup(C.byref(c), float(sigma), _vp(ws), ws.numel(), _stream(stream)))
    return Hierarchy(op.n, op.k, float(sigma), ws, op)


STEP_NAMES = {0: "PRE_A", 1: "A", 2: "PRE_B", 3: "B", 4: "C"}


def set_wait_limit(polls: int = 0) -> None:
    """Polls a device-side wait may take before it ends its launch with
    MVGD_ETIMEOUT (mvgd_set_wait_limit); 0 restores the kernels' defaults."""
    LB.check("mvgd_set_wait_limit", LB.load().mvgd_set_wait_limit(int(polls)))


def withhold_arrival(on: bool = True) -> None:
    """Arm (or disarm) the one-launch test control mvgd_test_withhold_arrival: the
    next solver or Gauss-Seidel launch has one wait that nothing ends."""
    LB.check("mvgd_test_withhold_arrival", LB.load().mvgd_test_withhold_arrival(1 if on else 0))


def trace_enable(on: bool = True) -> None:
    """Turn the solver's step trace on (clearing it) or off."""
    LB.check("mvgd_trace_enable", LB.load().mvgd_trace_enable(1 if on else 0))


def trace_read(max_entries: int = 1 << 16) -> list:
    """[(step name, ns since the previous step)] from the step trace."""
    buf = (C.c_uint64 * max_entries)()
    n = LB.load().mvgd_trace_read(buf, max_entries)
    if n < 0:
        raise MvgdError("mvgd_trace_read", LB.ECUDA)
    out = []
    prev = None
    for i in range(n):
        code, t = buf[i] >> 48, buf[i] & ((1 << 48) - 1)
        if code >= 0x1000:
            side, kind, lvl = (code >> 8) & 1, (code >> 4) & 15, code & 15
            name = f"V{'ps'[side]}:{('down', 'coarse', 'up')[kind]}{'' if kind == 1 else lvl}"
        else:
            name = STEP_NAMES.get(int(code), str(code))
        out.append((name, None if prev is None else t - prev))
        prev = t
    return out
