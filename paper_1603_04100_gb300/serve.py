"""Continuous-batching request loop for MVGD solves.

Requests (a cloud, its K and 1..8 right-hand sides) arrive over time.  The
loop:
  1. admits waiting requests in arrival order while their device memory fits
     the HBM budget (and a slot is free);
  2. runs the admitted clouds' kNN, ONE batched assembly launch for all of
     them, and initialises each one's solver state;
  3. advances every active request together with one persistent launch of
     `epoch_iters` Krylov iterations (mvgd_iterate);
  4. polls which requests finished, copies their solutions to the host,
     frees their memory and records completion times;
and repeats, so requests that arrive while others are on the GPU join the
running batch at the next epoch.  A request's result does not depend on what
else shared its launches (per-request reductions in a fixed order).
"""
from __future__ import annotations

import ctypes as C
import statistics
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib as LB
from . import api


@dataclass
class Request:
    rid: int
    arrival_s: float
    pts: np.ndarray          # [n][3] FP64 host
    f: np.ndarray            # [n][q] FP64 host
    k: int
    # filled by the server
    admitted_s: float = -1.0
    done_s: float = -1.0
    u: np.ndarray | None = None
    info: list = field(default_factory=list)

    @property
    def n(self) -> int:
        return self.pts.shape[0]

    @property
    def nrhs(self) -> int:
        return self.f.shape[1]


@dataclass
class _Live:
    req: Request
    nbytes: int
    pts: torch.Tensor
    f: torch.Tensor
    nbr: torch.Tensor
    order: torch.Tensor
    op: api.Operator
    ws: torch.Tensor
    u: torch.Tensor
    info: torch.Tensor
    amg: torch.Tensor | None = None
    opts: LB.SolveOpts | None = None


def request_bytes(n: int, k: int, q: int, prec: int, precond: int = 1) -> int:
    """Device bytes one admitted request holds until it retires."""
    L = LB.load()
    ell = sum(L.mvgd_ell_bytes(n, k, prec, w) for w in (LB.ELL_COL, LB.ELL_VAL, LB.ELL_VAL_LO))
    amg = L.mvgd_amg_workspace_bytes(n, k) if precond == LB.PRECOND_AMG else 0
    return (24 * n + 16 * n * q + 4 * n * k + 4 * n + ell + L.mvgd_request_workspace_bytes(n, k, q, prec, precond)
            + amg + 4 * n + 4096)


def amg_levels(n: int) -> int:
    """Levels of the multigrid hierarchy of an n-row operator (the library's rule)."""
    lv = 1
    while n > LB.AMG_COARSEST:
        n = (n + LB.AMG_AGG - 1) // LB.AMG_AGG
        lv += 1
    return lv


def amg_setup_kernels(n: int) -> int:
    """Kernels mvgd_amg_setup launches: header, level 0, two per coarser level, dense, inverse, promotion
    and four Newton-Schulz products."""
    return 9 + 2 * (amg_levels(n) - 1)


class Server:
    def __init__(self, device="cuda:0", *, hbm_budget: float = 120e9, prec: int = api.FP32_REFINE,
                 epoch_iters: int = 32, rtol: float = 1e-8, inner_rtol: float = 1e-3, precond: int = 1,
                 maxit: int = 200000, max_active: int = 1024, max_points: int = 1 << 21, max_k: int = 31,
                 pool_streams: int = 4):
        self.device = torch.device(device)
        self.budget = float(hbm_budget)
        self.prec = prec
        self.epoch_iters = epoch_iters
        self.max_active = max_active
        self.precond = precond
        self.opts = LB.SolveOpts(rtol, maxit, 20000, inner_rtol, 60, precond)
        self.rule = LB.DeltaRule(api.DELTA_MEAN_NN, 6, 1.0)
        L = LB.load()
        self.stream = torch.cuda.Stream(device=self.device)
        # admission work of different requests (kNN, multigrid set-up) overlaps on a pool
        self.pool = [torch.cuda.Stream(device=self.device) for _ in range(max(1, pool_streams))]
        self.knn_ws = [torch.empty(L.mvgd_knn_workspace_bytes(max_points, max_k), dtype=torch.uint8,
                                   device=self.device) for _ in self.pool]
        self.ctl_bytes = L.mvgd_iterate_workspace_bytes(max_active, 1 << 31)
        self.ctl_ws = torch.empty(self.ctl_bytes, dtype=torch.uint8, device=self.device)
        self.done_dev = torch.zeros(max_active, dtype=torch.int32, device=self.device)
        self.done_host = torch.zeros(max_active, dtype=torch.int32).pin_memory()
        self.used = 0.0
        self.epochs = 0
        self.launches = 0
        self.joins = 0            # requests admitted while others were running
        self.max_concurrent = 0
        self.waited = 0           # requests that found the budget or slots full

    # -- admission ------------------------------------------------------------------
    def _admit(self, reqs: list[Request]) -> list[_Live]:
        L = LB.load()
        vp = api._vp
        s = api._stream(self.stream)
        live = []
        with torch.cuda.stream(self.stream):
            # device buffers and uploads on the server's stream (which owns the memory),
            # then each request's kNN on a pool stream
            staged = []
            for r in reqs:
                n, k = r.n, r.k
                if L.mvgd_knn_workspace_bytes(n, k) > self.knn_ws[0].numel():  # pragma: no cover - max_points
                    raise ValueError("cloud larger than the server's kNN workspace")
                staged.append((torch.from_numpy(r.pts).to(self.device, non_blocking=True),
                               torch.from_numpy(np.ascontiguousarray(r.f)).to(self.device, non_blocking=True),
                               torch.empty((n, k), dtype=torch.int32, device=self.device),
                               torch.empty(n, dtype=torch.int32, device=self.device)))
            uploaded = torch.cuda.Event()
            uploaded.record(self.stream)
            for p in self.pool:
                p.wait_event(uploaded)
            for i, (r, (pts, f, nbr, order)) in enumerate(zip(reqs, staged)):
                n, k, q = r.n, r.k, r.nrhs
                ps = self.pool[i % len(self.pool)]
                ws_knn = self.knn_ws[i % len(self.pool)]
                LB.check("mvgd_knn", L.mvgd_knn(vp(pts), n, k, vp(nbr), vp(order), 0.0, vp(ws_knn), ws_knn.numel(),
                                                 api._stream(ps)))
                self.launches += 11
                col, val, lo = api.ell_alloc(n, k, self.prec, self.device)
                op = api.Operator(n, k, self.prec, col, val, lo, order)
                ws = torch.empty(L.mvgd_request_workspace_bytes(n, k, q, self.prec, self.precond), dtype=torch.uint8,
                                 device=self.device)
                u = torch.empty((n, q), dtype=torch.float64, device=self.device)
                info = torch.zeros(q * C.sizeof(LB.SolveInfo), dtype=torch.uint8, device=self.device)
                amg, opts = None, self.opts
                if self.precond == LB.PRECOND_AMG:
                    amg = torch.empty(L.mvgd_amg_workspace_bytes(n, k), dtype=torch.uint8, device=self.device)
                    opts = LB.SolveOpts(self.opts.rtol, self.opts.maxit, self.opts.inner_maxit, self.opts.inner_rtol,
                                        self.opts.max_outer, self.precond, C.c_void_p(amg.data_ptr()))
                live.append(_Live(r, request_bytes(n, k, q, self.prec, self.precond), pts, f, nbr, order, op, ws, u,
                                  info, amg, opts))
            for p in self.pool:
                ev = torch.cuda.Event()
                ev.record(p)
                self.stream.wait_event(ev)
            items = (LB.AssembleItem * len(live))()
            ns = (C.c_int64 * len(live))(*[x.req.n for x in live])
            aws = torch.empty(L.mvgd_assemble_batch_workspace_bytes(ns, len(live)), dtype=torch.uint8,
                              device=self.device)
            for i, x in enumerate(live):
                items[i] = LB.AssembleItem(vp(x.pts), vp(x.nbr), x.op.cstruct(), C.c_void_p(0), C.c_void_p(0))
            LB.check("mvgd_assemble_batch", L.mvgd_assemble_batch(items, len(live), self.rule, None, vp(aws),
                                                                   aws.numel(), s))
            self.launches += 1 + len(live) + (len(live) + 47) // 48
            if self.precond == LB.PRECOND_AMG:
                built = torch.cuda.Event()
                built.record(self.stream)
                for i, x in enumerate(live):
                    ps = self.pool[i % len(self.pool)]
                    ps.wait_event(built)
                    c = x.op.cstruct()
                    LB.check("mvgd_amg_setup", L.mvgd_amg_setup(C.byref(c), 1.0, vp(x.amg), x.amg.numel(),
                                                                 api._stream(ps)))
                    self.launches += amg_setup_kernels(x.req.n)
                for p in self.pool:
                    ev = torch.cuda.Event()
                    ev.record(p)
                    self.stream.wait_event(ev)
            for x in live:
                c = x.op.cstruct()
                LB.check("mvgd_request_init", L.mvgd_request_init(vp(x.ws), x.ws.numel(), C.byref(c), x.req.nrhs,
                                                                   1.0, vp(x.f), None, C.byref(x.opts), s))
                self.launches += 3 + (1 if self.precond == LB.PRECOND_ROWSCALE else 0)
        return live

    # -- one epoch over the active set ---------------------------------------------------
    def _epoch(self, active: list[_Live]) -> list[int]:
        L = LB.load()
        vp = api._vp
        s = api._stream(self.stream)
        cnt = len(active)
        reqs = (C.c_void_p * cnt)(*[x.ws.data_ptr() for x in active])
        descs = LB.requests([(x.ws, x.req.n, x.req.nrhs, x.req.k) for x in active])
        with torch.cuda.stream(self.stream):
            LB.check("mvgd_iterate", L.mvgd_iterate(descs, cnt, self.prec, self.precond, self.epoch_iters, None,
                                                     vp(self.ctl_ws), self.ctl_bytes, s))
            LB.check("mvgd_request_poll", L.mvgd_request_poll(reqs, cnt, vp(self.done_dev), s))
            self.done_host[:cnt].copy_(self.done_dev[:cnt], non_blocking=True)
        groups = (cnt + 255) // 256
        tables = 1
        if self.precond == LB.PRECOND_AMG:
            tables += max(amg_levels(x.req.n) - 1 for x in active)  # levels 1 .. mlev-1, and the coarsest
        self.launches += groups * tables + 3 + groups              # tables, count, solver, exit marks, poll
        self.stream.synchronize()
        self.epochs += 1
        return [i for i in range(cnt) if int(self.done_host[i]) != 0]

    def _retire(self, x: _Live, t0: float):
        L = LB.load()
        vp = api._vp
        s = api._stream(self.stream)
        with torch.cuda.stream(self.stream):
            LB.check("mvgd_request_finish", L.mvgd_request_finish(vp(x.ws), x.req.n, x.req.nrhs, vp(x.u),
                                                                   vp(x.info), s))
            u_h = x.u.to("cpu", non_blocking=False)
        self.launches += 2
        x.req.u = u_h.numpy()
        x.req.info = api.decode_info(x.info)
        x.req.done_s = time.perf_counter() - t0
        self.used -= x.nbytes

    # -- the loop -------------------------------------------------------------------------
    def serve(self, requests: list[Request], realtime: bool = True) -> dict:
        """Runs every request to completion; returns latency and throughput statistics."""
        pending = deque(sorted(requests, key=lambda r: r.arrival_s))
        waiting: deque[Request] = deque()
        active: list[_Live] = []
        t0 = time.perf_counter()
        while pending or waiting or active:
            now = time.perf_counter() - t0
            while pending and (pending[0].arrival_s <= now or not realtime):
                waiting.append(pending.popleft())
            admit = []
            while (waiting and len(active) + len(admit) < self.max_active
                   and self.used + request_bytes(waiting[0].n, waiting[0].k, waiting[0].nrhs, self.prec, self.precond)
                   <= self.budget):
                r = waiting.popleft()
                self.used += request_bytes(r.n, r.k, r.nrhs, self.prec, self.precond)
                r.admitted_s = now
                admit.append(r)
            if not admit and waiting and not active:
                raise RuntimeError(f"request {waiting[0].rid} does not fit the HBM budget")
            self.waited += len(waiting)
            if admit:
                if active:
                    self.joins += len(admit)
                active.extend(self._admit(admit))
                self.max_concurrent = max(self.max_concurrent, len(active))
            if not active:
                if pending:
                    time.sleep(max(0.0, min(0.002, pending[0].arrival_s - (time.perf_counter() - t0))))
                continue
            done = self._epoch(active)
            for i in sorted(done, reverse=True):
                self._retire(active[i], t0)
                del active[i]
        lat = [(r.done_s - r.arrival_s) * 1e3 for r in requests]
        first = min(r.arrival_s for r in requests)
        last = max(r.done_s for r in requests)
        pts = sum(r.n for r in requests)
        return {"requests": len(requests), "points": pts, "makespan_s": last - first,
                "points_per_s": pts / (last - first), "p50_ms": statistics.median(lat),
                "p99_ms": float(np.percentile(lat, 99)), "mean_ms": statistics.mean(lat), "epochs": self.epochs,
                "gpu_launches": self.launches, "joins": self.joins, "max_concurrent": self.max_concurrent,
                "waited_request_epochs": self.waited,
                "statuses": sorted({i[3] for r in requests for i in r.info})}


def requests_from_trace(specs, limit: int | None = None, time_scale: float = 1.0) -> list[Request]:
    """Builds host data for RequestSpec entries (inputs.serving_trace)."""
    out = []
    for sp in specs[:limit]:
        pr = sp.cloud.build()
        out.append(Request(sp.rid, sp.arrival_s * time_scale, pr.pts, pr.f, pr.k))
    return out
