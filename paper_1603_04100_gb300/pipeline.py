"""One cloud end to end: kNN -> MVGD assembly -> solve, with every buffer
allocated once so that repeated runs allocate nothing.

    pipe = Pipeline(n, k, nrhs, prec=FP32_REFINE, device="cuda:0")
    info = pipe.run(pts_dev, f_dev)          # device-resident inputs
    u_host = pipe.run_host(pts_pinned, f_pinned)   # host buffers, copies included
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib as LB
from . import api

# kernels each stage launches (the C ABI's own launches, not counting memsets/copies)
KERNELS_KNN = 11          # bbox x2, occupancy, params, count, scan x3, scatter, bucket sort, query
KERNELS_ASSEMBLE = 1      # + 1 inverse-order kernel with a locality order
KERNELS_SOLVE = 9         # init: 2 gathers + state; iterate: table, count, solver, exit marks; finish: 2


class Pipeline:
    def __init__(self, n: int, k: int, nrhs: int = 1, *, prec: int = api.FP32_REFINE, device="cuda:0",
                 reorder: bool = True, delta_m: int = 6, rtol: float = 1e-8, inner_rtol: float = 1e-3,
                 maxit: int = 200000, inner_maxit: int = 20000, max_outer: int = 60, precond: int = 1,
                 stream: torch.cuda.Stream | None = None, arith: int = 0):
        self.n, self.k, self.nrhs, self.prec = n, k, nrhs, prec
        self.device = torch.device(device)
        self.reorder, self.delta_m = reorder, delta_m
        self.stream = stream
        L = LB.load()
        dev = self.device
        self.nbr = torch.empty((n, k), dtype=torch.int32, device=dev)
        self.order = torch.empty(n, dtype=torch.int32, device=dev) if reorder else None
        self.ws_knn = torch.empty(L.mvgd_knn_workspace_bytes(n, k), dtype=torch.uint8, device=dev)
        self.ws_asm = torch.empty(max(256, L.mvgd_assemble_workspace_bytes(n)), dtype=torch.uint8, device=dev)
        self.precond = precond
        solve_bytes = L.mvgd_solve_workspace_bytes(n, k, nrhs, prec, precond)
        if precond == LB.PRECOND_AMG:  # the hierarchy is built below, outside the solve workspace
            solve_bytes -= (L.mvgd_amg_workspace_bytes(n, k) + 255) // 256 * 256
        self.ws_solve = torch.empty(solve_bytes, dtype=torch.uint8, device=dev)
        # the multigrid hierarchy lives beside the solver workspace and is rebuilt every run
        self.ws_amg = (torch.empty(L.mvgd_amg_workspace_bytes(n, k), dtype=torch.uint8, device=dev)
                       if precond == LB.PRECOND_AMG else None)
        col, val, lo = api.ell_alloc(n, k, prec, dev)
        self.op = api.Operator(n, k, prec, col, val, lo, self.order)
        self.op.bad_rows = torch.zeros(1, dtype=torch.int32, device=dev)
        self.u = torch.zeros((n, nrhs), dtype=torch.float64, device=dev)
        self.info = torch.zeros(nrhs * C.sizeof(LB.SolveInfo), dtype=torch.uint8, device=dev)
        self.opts = LB.SolveOpts(rtol, maxit, inner_maxit, inner_rtol, max_outer, precond,
                                 api._vp(self.ws_amg))
        self.rule = LB.DeltaRule(api.DELTA_MEAN_NN, delta_m, 1.0, 0, arith)
        # host-side staging for run_host
        self.pts_dev = torch.empty((n, 3), dtype=torch.float64, device=dev)
        self.f_dev = torch.empty((n, nrhs), dtype=torch.float64, device=dev)
        # the kNN grid's cell edge argument (0: the library's estimate; a tuner sets a
        # negative multiple of it, see tune.py)
        self.knn_cell = 0.0

    @property
    def kernels_per_run(self) -> int:
        k = KERNELS_KNN + KERNELS_ASSEMBLE + (1 if self.reorder else 0) + KERNELS_SOLVE
        if self.precond == LB.PRECOND_ROWSCALE:
            k += 1                                   # row scaling
        if self.precond == LB.PRECOND_AMG:
            lv = 1
            m = self.n
            while m > LB.AMG_COARSEST:
                m = (m + LB.AMG_AGG - 1) // LB.AMG_AGG
                lv += 1
            k += 9 + 2 * (lv - 1)                    # hierarchy set-up (with the Newton-Schulz products)
            k += (lv - 2 if lv > 2 else 0) + 1       # level and coarsest chunk tables
        return k

    def run(self, pts: torch.Tensor, f: torch.Tensor) -> torch.Tensor:
        """Enqueue kNN + assembly + solve on the stream; returns the device info buffer."""
        return self.run_staged(pts, f, None)

    def _stream(self):
        return self.stream if self.stream is not None else torch.cuda.current_stream()

    def knn_call(self, pts: torch.Tensor) -> None:
        L = LB.load()
        vp = api._vp
        LB.check("mvgd_knn", L.mvgd_knn(vp(pts), self.n, self.k, vp(self.nbr), vp(self.order), float(self.knn_cell),
                                         vp(self.ws_knn), self.ws_knn.numel(), api._stream(self._stream())))

    def assemble_call(self, pts: torch.Tensor) -> None:
        L = LB.load()
        vp = api._vp
        c = self.op.cstruct()
        LB.check("mvgd_assemble", L.mvgd_assemble(vp(pts), self.n, self.k, vp(self.nbr), self.rule, C.byref(c),
                                                   None, None, vp(self.op.bad_rows), vp(self.ws_asm),
                                                   self.ws_asm.numel(), api._stream(self._stream())))

    def amg_call(self) -> None:
        if self.ws_amg is None:
            return
        L = LB.load()
        c = self.op.cstruct()
        LB.check("mvgd_amg_setup", L.mvgd_amg_setup(C.byref(c), 1.0, api._vp(self.ws_amg), self.ws_amg.numel(),
                                                     api._stream(self._stream())))

    def solve_call(self, f: torch.Tensor) -> None:
        L = LB.load()
        vp = api._vp
        st = self._stream()
        with torch.cuda.stream(st):
            self.u.zero_()
        c = self.op.cstruct()
        LB.check("mvgd_solve", L.mvgd_solve(C.byref(c), self.nrhs, 1.0, vp(f), vp(self.u), C.byref(self.opts),
                                             vp(self.info), None, vp(self.ws_solve), self.ws_solve.numel(),
                                             api._stream(st)))

    def run_staged(self, pts: torch.Tensor, f: torch.Tensor, events=None) -> torch.Tensor:
        """As run(); events[1] / events[2] / events[3] (if given) are recorded after kNN /
        assembly / the multigrid set-up (right after assembly without one)."""
        st = self._stream()
        self.knn_call(pts)
        if events is not None:
            events[1].record(st)
        self.assemble_call(pts)
        if events is not None:
            events[2].record(st)
        self.amg_call()
        if events is not None and len(events) > 4:
            events[3].record(st)
        self.solve_call(f)
        return self.info

    def run_host(self, pts_host: torch.Tensor, f_host: torch.Tensor, u_host: torch.Tensor) -> None:
        """Host (pinned) buffers in and out: H2D copies, the run, D2H copy of u."""
        st = self.stream if self.stream is not None else torch.cuda.current_stream()
        with torch.cuda.stream(st):
            self.pts_dev.copy_(pts_host, non_blocking=True)
            self.f_dev.copy_(f_host, non_blocking=True)
            self.run(self.pts_dev, self.f_dev)
            u_host.copy_(self.u, non_blocking=True)

    def decode(self):
        return api.decode_info(self.info)
