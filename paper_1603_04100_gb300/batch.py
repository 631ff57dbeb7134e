"""Uneven clouds through shared launches.

A batch of clouds (any sizes, K and number of right-hand sides each) runs as:
  * kNN: each cloud's grid build and queries on one of a pool of streams, so
    small clouds overlap instead of queueing;
  * assembly: ONE launch over (cloud, 32-row slice) work items
    (mvgd_assemble_batch);
  * multigrid set-up (precond 2): each cloud's hierarchy on the stream pool;
  * solve: every cloud is a request with its own solver state; ONE persistent
    launch (mvgd_iterate) advances all of them to convergence; requests that
    finish early cost nothing while the rest iterate.
The whole sequence can be captured once in a CUDA graph and replayed.

Each cloud's result does not depend on the batch it ran in: the kernels are
the per-cloud ones and every solver reduction runs per request over fixed
chunks in a fixed order.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import torch

from . import _lib as LB
from . import api
from .serve import amg_setup_kernels


@dataclass
class CloudSlot:
    n: int
    k: int
    nrhs: int
    nbr: torch.Tensor
    order: torch.Tensor
    op: api.Operator
    req_ws: torch.Tensor
    u: torch.Tensor
    info: torch.Tensor
    amg_ws: torch.Tensor | None = None


class BatchPipeline:
    """Preallocated buffers for a fixed list of (n, k, nrhs) clouds."""

    def __init__(self, sizes, *, prec: int = api.FP32_REFINE, device="cuda:0", n_streams: int = 8,
                 rtol: float = 1e-8, inner_rtol: float = 1e-3, maxit: int = 200000, inner_maxit: int = 20000,
                 max_outer: int = 60, precond: int = 1, delta_m: int = 6, cell_scale: float = 0.0):
        self.device = torch.device(device)
        self.prec = prec
        self.sizes = [(int(n), int(k), int(q)) for n, k, q in sizes]
        L = LB.load()
        dev = self.device
        self.slots: list[CloudSlot] = []
        for n, k, q in self.sizes:
            col, val, lo = api.ell_alloc(n, k, prec, dev)
            order = torch.empty(n, dtype=torch.int32, device=dev)
            op = api.Operator(n, k, prec, col, val, lo, order)
            req = torch.empty(L.mvgd_request_workspace_bytes(n, k, q, prec, precond), dtype=torch.uint8, device=dev)
            amg = (torch.empty(L.mvgd_amg_workspace_bytes(n, k), dtype=torch.uint8, device=dev)
                   if precond == LB.PRECOND_AMG else None)
            self.slots.append(CloudSlot(n, k, q, torch.empty((n, k), dtype=torch.int32, device=dev), order, op, req,
                                        torch.empty((n, q), dtype=torch.float64, device=dev),
                                        torch.zeros(q * C.sizeof(LB.SolveInfo), dtype=torch.uint8, device=dev), amg))
        self.streams = [torch.cuda.Stream(device=dev) for _ in range(max(1, n_streams))]
        nmax = max(n for n, _, _ in self.sizes)
        kmax = max(k for _, k, _ in self.sizes)
        self.knn_ws = [torch.empty(L.mvgd_knn_workspace_bytes(nmax, kmax), dtype=torch.uint8, device=dev)
                       for _ in self.streams]
        ns = (C.c_int64 * len(self.sizes))(*[n for n, _, _ in self.sizes])
        self.asm_ws = torch.empty(L.mvgd_assemble_batch_workspace_bytes(ns, len(self.sizes)), dtype=torch.uint8,
                                  device=dev)
        total = sum(n for n, _, _ in self.sizes)
        self.ctl_ws = torch.empty(L.mvgd_iterate_workspace_bytes(len(self.sizes), total), dtype=torch.uint8,
                                  device=dev)
        self.bad_rows = torch.zeros(1, dtype=torch.int32, device=dev)
        self.opts = LB.SolveOpts(rtol, maxit, inner_maxit, inner_rtol, max_outer, precond)
        self.rule = LB.DeltaRule(api.DELTA_MEAN_NN, delta_m, 1.0)
        self.cell_scale = cell_scale
        self.budget = maxit + 2 * (max_outer + 2) + 4
        cnt = len(self.slots)
        self.precond = precond
        self._reqs = LB.requests([(s.req_ws, s.n, s.nrhs, s.k) for s in self.slots])
        self._opts = []
        for sl in self.slots:
            o = LB.SolveOpts(rtol, maxit, inner_maxit, inner_rtol, max_outer, precond)
            if sl.amg_ws is not None:
                o.amg = C.c_void_p(sl.amg_ws.data_ptr())
            self._opts.append(o)
        self.graph = None

    @property
    def total_points(self) -> int:
        return sum(s.n for s in self.slots)

    def run(self, pts_list, f_list, cancel: torch.Tensor | None = None, marks=None):
        """Enqueue kNN + assembly + solve for every cloud on the current stream.  If given,
        marks[0] / [1] / [2] (CUDA events) are recorded on it once every cloud's kNN, the
        batched assembly and every multigrid set-up have been enqueued before them."""
        L = LB.load()
        vp = api._vp
        main = torch.cuda.current_stream(self.device)
        fork = torch.cuda.Event()
        fork.record(main)
        for i, (slot, pts) in enumerate(zip(self.slots, pts_list)):
            si = i % len(self.streams)
            st = self.streams[si]
            st.wait_event(fork)
            ws = self.knn_ws[si]
            LB.check("mvgd_knn", L.mvgd_knn(vp(pts), slot.n, slot.k, vp(slot.nbr), vp(slot.order), self.cell_scale,
                                             vp(ws), ws.numel(), api._stream(st)))
        for st in self.streams:
            ev = torch.cuda.Event()
            ev.record(st)
            main.wait_event(ev)
        if marks is not None:
            marks[0].record(main)
        items = (LB.AssembleItem * len(self.slots))()
        for i, (slot, pts) in enumerate(zip(self.slots, pts_list)):
            items[i] = LB.AssembleItem(vp(pts), vp(slot.nbr), slot.op.cstruct(), C.c_void_p(0), C.c_void_p(0))
        s = api._stream(main)
        LB.check("mvgd_assemble_batch", L.mvgd_assemble_batch(items, len(self.slots), self.rule, vp(self.bad_rows),
                                                               vp(self.asm_ws), self.asm_ws.numel(), s))
        if marks is not None:
            marks[1].record(main)
        if self.precond == LB.PRECOND_AMG:
            # the hierarchies on the stream pool: each set-up is a chain of small
            # launches (the coarsest inverse is one block), so clouds overlap
            built = torch.cuda.Event()
            built.record(main)
            for i, slot in enumerate(self.slots):
                st = self.streams[i % len(self.streams)]
                st.wait_event(built)
                c = slot.op.cstruct()
                LB.check("mvgd_amg_setup", L.mvgd_amg_setup(C.byref(c), 1.0, vp(slot.amg_ws), slot.amg_ws.numel(),
                                                             api._stream(st)))
            for st in self.streams:
                ev = torch.cuda.Event()
                ev.record(st)
                main.wait_event(ev)
        if marks is not None:
            marks[2].record(main)
        for slot, f, opts in zip(self.slots, f_list, self._opts):
            c = slot.op.cstruct()
            LB.check("mvgd_request_init", L.mvgd_request_init(vp(slot.req_ws), slot.req_ws.numel(), C.byref(c),
                                                               slot.nrhs, 1.0, vp(f), None, C.byref(opts), s))
        LB.check("mvgd_iterate", L.mvgd_iterate(self._reqs, len(self.slots), self.prec, self.precond, self.budget,
                                                 vp(cancel), vp(self.ctl_ws), self.ctl_ws.numel(), s))
        for slot in self.slots:
            LB.check("mvgd_request_finish", L.mvgd_request_finish(vp(slot.req_ws), slot.n, slot.nrhs, vp(slot.u),
                                                                   vp(slot.info), s))

    def capture(self, pts_list, f_list):
        """Record the whole batch once as a CUDA graph; replay() reruns it."""
        self.run(pts_list, f_list)  # warm-up outside capture (lazy module loading, attributes)
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run(pts_list, f_list)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def infos(self):
        return [api.decode_info(s.info) for s in self.slots]

    @property
    def kernels_per_run(self) -> int:
        per_cloud_knn = 11
        return (len(self.slots) * (per_cloud_knn + 1 + 3 + 2)  # knn, inverse order, init (2 gathers+1), finish (2)
                + 1 + (len(self.slots) + 47) // 48              # batched assembly + descriptor uploads
                + (len(self.slots) + 255) // 256 + 3            # iterate: tables, count, solver, exit marks
                + (sum(amg_setup_kernels(s.n) for s in self.slots) if self.precond == LB.PRECOND_AMG else 0))
