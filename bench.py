#!/usr/bin/env python3
"""MVGD hot-path benchmark: points/s for kNN + assembly + solve of
(I - L) u = f to a 1e-8 relative residual on a 1,048,576-point random unit
sphere, K = 20, u = 5z^3 - 3z, f = 13u (synthetic, seeded).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One JSON line on rank 0.  A step is one pass of the whole path over one cloud:
kNN -> MVGD assembly -> solve.  The timed path is the FP32 + FP64-refinement
one; the plain FP64 path (same kNN, same preconditioner, FP64 assembly, FP64
Krylov) is timed beside it.  L2 is flushed (1 GiB write) before every step,
outside the per-step CUDA-event windows.  With N > 1 (torchrun) every rank
solves its own replica of the cloud (weak scaling, no collective on the data
path); the reported time is the max over ranks.

--impl reference times the FP64 CPU oracle on the host cores instead, each
step a bounded sample of the same workload scaled to points/s.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "MVGD points/s (assembly+solve to 1e-8 rel) batched/served vs plain; p50/p99 ms"
N_DEFAULT, K_DEFAULT, SEED = 1_048_576, 20, 0
RTOL = 1e-8
# DRAM bytes (read + write) per iteration of k_solve<1,1,1> on the bench workload
# (N = 1,048,576, K = 20, multigrid, FP32 inner), from an ncu capture of the
# current kernel; None until one is taken (the line then reports traffic null).
KSOLVE_MIXED_AMG_DRAM_PER_ITERATION = 1.108e9  # 22.162 GB over a 20-iteration capture
BATCH_MAXIT = 3000  # batched workload: iteration cap per cloud (see batched_measure)
SERVED_REQUESTS, SERVED_RATE = 60, 20.0  # the served slice in the default line (below saturation)
WORKLOAD = ("random unit sphere N=1,048,576 (normalised PCG64(0) Gaussian rows), K=20, delta = mean distance to "
            "6 nearest, u = 5z^3-3z, f = 13u, (I-L)u = f to 1e-8 relative residual")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--k", type=int, default=K_DEFAULT)
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 comparison")
    ap.add_argument("--workload", choices=["sphere1m", "batched", "served"], default="sphere1m",
                    help="sphere1m: the headline (1M random sphere); batched: 256 uneven clouds in one batch; "
                         "served: a Poisson request trace through the serving loop")
    ap.add_argument("--requests", type=int, default=200, help="served: requests taken from the trace")
    ap.add_argument("--rate", type=float, default=200.0, help="served: arrival rate (requests/s)")
    ap.add_argument("--paths", default="fp32_refine+amg,fp64+amg,fp32_refine,fp64",
                    help="comma list of <precision>[+amg] paths to time (the fastest is the headline)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline sample")
    ap.add_argument("--no-tune", action="store_true", help="keep the library's default launch shapes")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched / served / open-surface / eigenvalue lines after the headline")
    ap.add_argument("--profile-case", type=int, nargs=4, metavar=("N", "PREC", "ITERS", "PRECOND"),
                    help="profiling target only: kNN + assembly + a solve capped at ITERS iterations on an "
                         "N-point random sphere, PREC 0 FP64 / 1 FP32+refine, PRECOND 1 row scaling / 2 multigrid")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.file is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in Path(self.file.name).read_text().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((float(r[3]) for r in rows if r[3].replace(".", "").isdigit()), default=None)}


# ------------------------------------------------------------------------------
# algorithmic bytes of the persistent solver (per row)
# ------------------------------------------------------------------------------
def solver_bytes_per_row(k: int, mixed: bool, iters: int, restarts: int, amg_coarse: float | None = None) -> float:
    """Unique bytes one launch of the persistent solver must move per fine row.

    Row-scaled flow, mixed, per inner iteration (FP32 vectors, FP32 hi weights,
    int32 columns):
      A: col 4k + val 4k + self weight 4 + r,p,v,rh 16 + write p,v 8
      B: col 4k + val 4k + self weight 4 + r,v 8 + write s,t 8
      C: x,p,s,t,r,rh 24 + write x,r 8                      -> 16k + 80
    per restart (FP64 residual on hi + lo):
      fold u += scale x 20; residual col 4k + hi,lo 8(k+1) + u,f 16 + r64 8;
      restart r64 8 + self weight 4 + r,rh,p0,p1,v0,v1,x 28  -> 12k + 92
    Plain FP64, per iteration 24k + 160; per restart 12k + 96.

    Multigrid flow (amg_coarse = bytes per fine row of one V-cycle's levels >= 1,
    including the coarsest solve), per iteration (six grid steps; the last
    step's r = s - omega t is formed in PRE_A) with V-cycle level 0 on FP32
    weights:
      V-cycle level 0: down col 4k + val 4(k+1) + b,y 4+vt + write r + b,y of
        level 1 (1/8 each) 5; up col 4k + val 4(k+1) + y,r,d 12 + write x vt
        -> 16k + 29 + 2 vt (+ amg_coarse), twice per iteration
      mixed (vt 4): PRE_A s,t,x,ph,sh,p,v,d 32 + r,x,p,y 16; A 8k+4 + ph,rh 8 + v 4;
        PRE_B r,v,d 12 + s,y 8; B 8k+4 + sh,s,rh 12 + t 4;
        two V-cycles 32k + 74                        -> 48k + 178 + 2 amg_coarse
      FP64 (vt 8): PRE_A 60 + 28; A 12k+8 + 16 + 8; PRE_B 20 + 12; B 12k+8 + 24 + 8;
        two V-cycles 32k + 90                        -> 56k + 282 + 2 amg_coarse
    """
    if amg_coarse is not None:
        per = (48 * k + 178) if mixed else (56 * k + 282)
        return iters * (per + 2 * amg_coarse) + restarts * ((12 * k + 92) if mixed else (12 * k + 96))
    if mixed:
        return iters * (16 * k + 80) + restarts * (12 * k + 92)
    return iters * (24 * k + 160) + restarts * (12 * k + 96)


def spmv_roofline(results, n, k, flush, stream, peak, peak_kind, reps: int = 20):
    """mvgd_spmv timed alone: y = sigma x - L x, one RHS, per launch (CUDA events on the
    launching stream, L2 flushed before each launch).  Algorithmic bytes per row:
    FP32 difference form col 4k + val 4k (the self weight is implied) + x_i + y_i = 8k + 8;
    FP64 col 4k + val 8(k+1) + x_i + y_i = 12k + 24 (neighbour gathers hit L2).
    The flush before each launch writes 1 GiB (about 0.15 ms of device time), longer than
    the host needs to enqueue the product, so the event pair brackets the kernel and not
    the host's launch latency (a 35 us kernel behind a 40 us flush read as 45 us)."""
    import torch
    from paper_1603_04100_gb300 import api
    out = {}
    for nm, mode, per_row in (("fp32_difference", api.SPMV_F32, 8 * k + 8), ("fp64", api.SPMV_F64, 12 * k + 24)):
        src = next((r for r in results.values() if (r["mixed"] if mode == api.SPMV_F32 else not r["mixed"])), None)
        if src is None:
            continue
        op = src["pipe"].op
        dt = torch.float32 if mode == api.SPMV_F32 else torch.float64
        x = torch.linspace(-1.0, 1.0, n, device=flush.device, dtype=dt)
        y = torch.empty_like(x)
        ms = []
        with torch.cuda.stream(stream):
            for i in range(reps + 3):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                api.spmv(op, x, mode=mode, y=y, stream=stream)
                e1.record(stream)
                if i >= 3:
                    ms.append((e0, e1))
        stream.synchronize()
        t = statistics.median(a.elapsed_time(b) for a, b in ms)
        gbs = per_row * n / (t * 1e-3) / 1e9
        out[nm] = {"us": t * 1e3, "bytes_per_row": per_row, "achieved_gbs": gbs, "frac": gbs / peak,
                   "peak_kind": f"hbm_gbs of {peak_kind}"}
    return out


def row_sign_stats(pts, pipe, k, flush, stream):
    """Sec. 3.2 / Sec. 4.1 on the bench cloud: the share of rows with the M-matrix sign
    pattern (mvgd_row_signs) for the MVGD rows and for the plain least-squares comparator,
    and the device time of the comparator's assembly (same kernel, variant ROW_LS)."""
    import torch
    from paper_1603_04100_gb300 import api
    out = {}
    with torch.cuda.stream(stream):
        mv = api.row_signs(pipe.op, stream=stream)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ls = api.assemble(pts, pipe.nbr, prec=api.FP64, order=pipe.order, variant=api.ROW_LS, stream=stream)
        e1.record(stream)
        lsc = api.row_signs(ls, stream=stream)
    stream.synchronize()
    for nm, c in (("mvgd", mv), ("least_squares", lsc)):
        out[nm] = {"m_pattern_frac": c["m_pattern_rows"] / c["rows"], "negative_weights": c["negative_weights"],
                   "nonneg_self_rows": c["nonneg_self_rows"]}
    out["least_squares_assembly_ms"] = e0.elapsed_time(e1)
    return out


def dirichlet_hemisphere(n, k, flush, stream):
    """Open surface (Sec. 3.1): the upper hemisphere with n points and Dirichlet rows on
    its rim band, u = z, (I - L) u = 3z; kNN, assembly, boundary rows, multigrid set-up
    and the FP32 + FP64-refinement solve timed once with CUDA events (L2 flushed)."""
    import numpy as np
    import torch
    from paper_1603_04100_gb300 import api
    from paper_1603_04100_gb300 import inputs as I
    p, b = I.hemisphere(n, 5)
    z = p[:, 2]
    f_h = np.where(b == 1, z, 3.0 * z)
    dev = flush.device
    pts = torch.from_numpy(p).to(dev)
    f = torch.from_numpy(f_h).to(dev)
    bt = torch.from_numpy(b).to(dev)
    out = {}
    for rep in range(2):  # the first pass warms up
        with torch.cuda.stream(stream):
            flush.zero_()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(stream)
            nbr, order = api.knn(pts, k, want_order=True, stream=stream)
            op = api.assemble(pts, nbr, prec=api.FP32_REFINE, order=order, stream=stream)
            rows = api.dirichlet_rows(op, bt, stream=stream)
            ev[1].record(stream)
            res = api.solve(op, f, rtol=RTOL, precond=2, stream=stream)
            ev[2].record(stream)
        stream.synchronize()
        u = res.u.cpu().numpy()
        out = {"n": n, "k": k, "boundary_rows": rows, "ms": ev[0].elapsed_time(ev[2]),
               "setup_ms": ev[0].elapsed_time(ev[1]), "solve_ms": ev[1].elapsed_time(ev[2]),
               "iters": res.iters[0], "status": res.status[0], "relres": res.relres[0],
               "err_exact_inf": float(np.abs(u - z).max()), "points_per_s": n / (ev[0].elapsed_time(ev[2]) * 1e-3)}
    return out


def neumann_hemisphere(n, k, flush, stream):
    """Open surface with dU/dn = 0 on the rim (Sec. 3.1, reflection method): the upper
    hemisphere with n points, u = x, (I - L) u = 3x on the interior points; kNN of the
    cloud, ghosts, kNN and assembly over interior points and ghosts, fold, multigrid
    set-up and the FP32 + FP64-refinement solve, timed once with CUDA events (L2 flushed)."""
    import numpy as np
    import torch
    from paper_1603_04100_gb300 import api
    from paper_1603_04100_gb300 import inputs as I
    p, b = I.hemisphere(n, 5)
    dev = flush.device
    pts = torch.from_numpy(p).to(dev)
    bt = torch.from_numpy(b).to(dev)
    out = {}
    for rep in range(2):  # the first pass warms up
        with torch.cuda.stream(stream):
            flush.zero_()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(stream)
            op, cloud = api.neumann_operator(pts, bt, k, prec=api.FP32_REFINE, stream=stream)
            x = pts[cloud.interior.long(), 0].contiguous()
            f = 3.0 * x
            ev[1].record(stream)
            res = api.solve(op, f, rtol=RTOL, precond=2, stream=stream)
            ev[2].record(stream)
        stream.synchronize()
        u = res.u.cpu().numpy()
        xs = x.cpu().numpy()
        out = {"n": n, "k": k, "boundary_points": cloud.n_boundary, "interior_rows": cloud.n_interior,
               "ghosts": cloud.n_ghost, "ms": ev[0].elapsed_time(ev[2]), "setup_ms": ev[0].elapsed_time(ev[1]),
               "solve_ms": ev[1].elapsed_time(ev[2]), "iters": res.iters[0], "status": res.status[0],
               "relres": res.relres[0], "err_exact_inf": float(np.abs(u - xs).max()),
               "points_per_s": n / (ev[0].elapsed_time(ev[2]) * 1e-3)}
    return out


def lb_eigen_stats(k, stream, n_pts: int = 16000):
    """Sec. 4.3 on the paper's largest random sphere: the 25 smallest eigenvalues of -L
    (lambda_0 .. lambda_4 multiplets) by the shift-invert subspace iteration, timed with
    CUDA events, and the E^2_4 / E^inf_4 errors beside the paper's printed MVGD values
    for random samplings of 16000 points (0.069e-2 and 0.13e-2)."""
    import numpy as np
    import torch
    from paper_1603_04100_gb300 import api
    from paper_1603_04100_gb300 import inputs as I
    from paper_1603_04100_gb300.eigs import lowest_eigenpairs
    p = I.random_sphere(n_pts, 1)
    dev = torch.device("cuda", torch.cuda.current_device())
    pt = torch.from_numpy(p).to(dev)
    with torch.cuda.stream(stream):
        nbr, order = api.knn(pt, k, want_order=True, stream=stream)
        op = api.assemble(pt, nbr, prec=api.FP64, order=order, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = lowest_eigenpairs(op, 25, stream=stream)
        e1.record(stream)
    stream.synchronize()
    lam = res.values
    n4 = slice(16, 25)
    r4 = (lam[n4] - 20.0) / 20.0
    return {"n": n_pts, "k": k, "nev": 25, "ms": e0.elapsed_time(e1), "iterations": res.iterations,
            "solves": res.solves, "lambda0": float(lam[0]),
            "E2_lambda4_pct": float(100 * np.sqrt(np.mean(r4 * r4))), "Einf_lambda4_pct": float(100 * np.abs(r4).max()),
            "paper_random_16000_pct": {"E2_lambda4": 0.069, "Einf_lambda4": 0.13}}


def gs_spectral_stats(k, stream, n_pts: int = 16000, iters: int = 300):
    """Sec. 4.1 on a random sphere: the spectral radius of the Gauss-Seidel iteration
    matrix of I - L (stored row order) for the MVGD rows and for the least-squares
    comparator, by mvgd_gs_power (geometric mean of the norm ratios over the second
    half of the steps), timed with CUDA events."""
    import numpy as np
    import torch
    from paper_1603_04100_gb300 import api
    from paper_1603_04100_gb300 import inputs as I
    p = I.random_sphere(n_pts, 1)
    dev = torch.device("cuda", torch.cuda.current_device())
    pt = torch.from_numpy(p).to(dev)
    x0 = torch.from_numpy(np.random.default_rng(0).standard_normal(n_pts)).to(dev)
    out = {"n": n_pts, "k": k, "iters": iters, "sigma": 1.0, "order": "stored (Z-order)"}
    with torch.cuda.stream(stream):
        nbr, order = api.knn(pt, k, want_order=True, stream=stream)
        for nm, variant in (("mvgd", api.ROW_MVGD), ("least_squares", api.ROW_LS)):
            op = api.assemble(pt, nbr, prec=api.FP64, order=order, variant=variant, stream=stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g = api.gs_power(op, x0, iters, sigma=1.0, stream=stream)
            e1.record(stream)
            stream.synchronize()
            out[nm] = {"rho": g.rho, "nu_last": float(g.nu[-1]), "status": g.status, "ms": e0.elapsed_time(e1),
                       "us_per_step": 1e3 * e0.elapsed_time(e1) / iters}
    return out


def amg_coarse_bytes(H, n: int) -> float:
    """Bytes per fine row that one V-cycle moves on levels >= 1: per level, down
    and up read each stored entry (int32 column + FP32 value) once, plus about
    36 bytes of vectors per row; the coarsest solve reads its dense FP64 inverse."""
    total = 0.0
    for lv in range(1, H.levels):
        cnt = H.level_rows(lv)[0] if lv < H.levels - 1 else None
        info = H.info(lv)
        if lv < H.levels - 1:
            total += 16.0 * float(cnt.sum()) + 36.0 * info.n
        else:
            total += 4.0 * info.n * info.n + 8.0 * info.n
    if H.levels == 1:
        total += 8.0 * n * n
    return total / n


# ------------------------------------------------------------------------------
# the oracle on the host cores (CPU baseline and the reference arm)
# ------------------------------------------------------------------------------
ORACLE_ITERS_FILE = ROOT / "oracle" / "iterations_random_sphere_1m_k20.json"


REF_SAMPLE_ITERS = 4  # preconditioned oracle iterations timed per reference step


class OracleSampler:
    """Bounded samples of the workload on the FP64 oracle, on the host cores.

    Once: the oracle's kNN and rows of the full cloud and its multigrid
    hierarchy (oracle/amg.py, rows relabelled along a Z-order curve), timed.
    Each sample() then times the oracle's kNN (grid) and assembly of the full
    cloud again and REF_SAMPLE_ITERS iterations of its multigrid-preconditioned
    BiCGSTAB.  The full solve is projected from the recorded iteration count of
    that same solver on this workload (ORACLE_ITERS_FILE, written by
    oracle/measure_iterations.py): setup + hierarchy + iterations x time per
    iteration."""

    def __init__(self, n: int, k: int):
        import oracle
        from oracle import amg as OA
        from paper_1603_04100_gb300 import inputs as I
        self.oracle, self.OA = oracle, OA
        self.n, self.k = n, k
        self.threads = oracle.threads(os.cpu_count() or 1)
        self.pr = I.random_sphere_problem(n, k, seed=SEED)
        self.perm = I.morton_permutation(self.pr.pts)
        self.inv = np.empty_like(self.perm)
        self.inv[self.perm] = np.arange(n)
        nbr = oracle.knn_grid(self.pr.pts, k)
        val, _, _, _ = oracle.assemble(self.pr.pts, nbr, delta_m=6)
        t0 = time.perf_counter()
        self.levels = OA.hierarchy(val[self.perm], self.inv[nbr[self.perm]].astype(np.int32), 1.0)
        self.hierarchy_s = time.perf_counter() - t0
        self.f = np.ascontiguousarray(self.pr.f[self.perm, 0])
        rec = json.loads(ORACLE_ITERS_FILE.read_text()) if ORACLE_ITERS_FILE.exists() else {}
        self.iters_needed = int(rec["multigrid"]["iters"]) if "multigrid" in rec else None
        self.iters_plain = int(rec["bicgstab"]["iters"]) if "bicgstab" in rec else None

    def sample(self) -> dict:
        t0 = time.perf_counter()
        nbr = self.oracle.knn_grid(self.pr.pts, self.k)
        self.oracle.assemble(self.pr.pts, nbr, delta_m=6)
        t1 = time.perf_counter()
        self.OA.bicgstab_right(self.levels, self.f, rtol=1e-30, maxit=REF_SAMPLE_ITERS)
        t2 = time.perf_counter()
        return {"setup_s": t1 - t0, "iteration_s": (t2 - t1) / REF_SAMPLE_ITERS, "sample_s": t2 - t0}

    def summarise(self, samples) -> dict:
        setup = statistics.median(x["setup_s"] for x in samples)
        it = statistics.median(x["iteration_s"] for x in samples)
        full = setup + self.hierarchy_s + it * self.iters_needed
        return {"value": self.n / full, "unit": "points/s", "cores": self.threads, "kind": "oracle",
                "sample_ms": statistics.median(x["sample_s"] for x in samples) * 1e3,
                "projected_full_solve_ms": full * 1e3,
                "projection": f"kNN + assembly ({setup:.2f} s, timed each step) + multigrid hierarchy "
                              f"({self.hierarchy_s:.2f} s, timed once) + {self.iters_needed} iterations x "
                              f"{it * 1e3:.0f} ms (the iteration count of this oracle solver to 1e-8 on this "
                              f"cloud, {ORACLE_ITERS_FILE.name})",
                "sample": f"the oracle (C kNN and assembly with {self.threads} OpenMP threads, numpy multigrid "
                          f"BiCGSTAB) on the full {self.n}-point cloud: kNN + assembly + {REF_SAMPLE_ITERS} "
                          f"preconditioned iterations a step",
                "unpreconditioned_oracle_iters": self.iters_plain}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n, k = args.n, args.k
    if not ORACLE_ITERS_FILE.exists() or "multigrid" not in json.loads(ORACLE_ITERS_FILE.read_text()):
        print(json.dumps({"impl": "reference", "unavailable": "oracle iteration count file missing"}))
        return
    t_begin = time.perf_counter()
    samp = OracleSampler(n, k)
    samples = []
    for s in range(args.warmup + args.steps):
        x = samp.sample()
        if s >= args.warmup:
            samples.append(x)
    base = samp.summarise(samples)
    value = base["value"]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": base["sample_ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "k": k, "rtol": RTOL, "parallelism": "host cores"},
        "projected_full_solve_ms": base["projected_full_solve_ms"],
        "value_basis": "value = points / projected_full_solve_ms; ms_per_step is the bounded sample each step "
                       "actually timed",
        "cpu_baseline": base,
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": time.perf_counter() - t_begin,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------
def batched_measure(dev, reps, specs, steps: int, warmup: int, arms=(("fp32_refine+amg", 1, 2), ("fp64+amg", 0, 2)),
                    workload: str = ""):
    """Uneven clouds as one batch: kNN per cloud on a stream pool, one batched assembly, one
    multigrid set-up per cloud, one persistent solver launch for all; points/s over the batch,
    against the same clouds solved one at a time by the plain FP64 path (row scaling).  Every
    arm stops at BATCH_MAXIT iterations a cloud and reports the clouds and points that converged."""
    import torch
    from paper_1603_04100_gb300 import api
    from paper_1603_04100_gb300.batch import BatchPipeline
    from paper_1603_04100_gb300.pipeline import Pipeline
    probs = [sp.build() for sp in specs]
    pts = [torch.from_numpy(p.pts).to(dev) for p in probs]
    fs = [torch.from_numpy(np.ascontiguousarray(p.f)).to(dev) for p in probs]
    sizes = [(p.pts.shape[0], p.k, p.f.shape[1]) for p in probs]
    total = sum(s[0] for s in sizes)
    out = {"config": {"workload": workload, "clouds": len(sizes), "points": total, "maxit": BATCH_MAXIT,
                      "rhs": sum(s[2] for s in sizes)}, "paths": {}}
    for name, prec, precond in arms:
        bp = BatchPipeline(sizes, prec=prec, precond=precond, device=dev, maxit=BATCH_MAXIT,
                           inner_maxit=BATCH_MAXIT)
        for _ in range(max(1, warmup)):
            bp.run(pts, fs)
        reps.barrier()
        ms = []
        stages = {"knn": [], "assemble": [], "amg_setup": [], "solve": []}
        for _ in range(max(1, steps)):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
            ev[0].record()
            bp.run(pts, fs, marks=ev[1:4])
            ev[4].record()
            torch.cuda.synchronize()
            ms.append(ev[0].elapsed_time(ev[4]))
            for j, key in enumerate(stages):
                stages[key].append(ev[j].elapsed_time(ev[j + 1]))
        reps.barrier()
        ms_max = reps.max(statistics.mean(ms))
        infos = bp.infos()
        st = sorted({i[3] for inf in infos for i in inf})
        worst = max(i[2] for inf in infos for i in inf)
        iters = [i[0] for inf in infos for i in inf]
        conv = [all(i[3] == 0 for i in inf) for inf in infos]
        out["paths"][name] = {"value": reps.job_rate(total, ms_max), "ms": ms_max,
                              "statuses": st, "worst_relres": worst, "max_iters": max(iters),
                              "mean_iters": statistics.mean(iters),
                              "converged_clouds": sum(conv), "converged_points": sum(
                                  s[0] for s, c in zip(sizes, conv) if c),
                              "gpu_launches": bp.kernels_per_run,
                              "stage_ms": {key: statistics.mean(v) for key, v in stages.items()}}
        del bp
        torch.cuda.empty_cache()
    # plain: the same clouds one at a time, FP64 with row scaling
    t_plain = 0.0
    conv_plain = []
    for p, pt, f in zip(probs, pts, fs):
        pipe = Pipeline(p.pts.shape[0], p.k, p.f.shape[1], prec=api.FP64, device=dev, precond=1, rtol=RTOL,
                        maxit=BATCH_MAXIT)
        pipe.run(pt, f)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        pipe.run(pt, f)
        e1.record()
        torch.cuda.synchronize()
        t_plain += e0.elapsed_time(e1)
        conv_plain.append(all(i[3] == 0 for i in api.decode_info(pipe.info)))
        del pipe
    t_plain = reps.max(t_plain)
    out["paths"]["plain_fp64_one_by_one"] = {"value": reps.job_rate(total, t_plain), "ms": t_plain,
                                             "converged_clouds": sum(conv_plain), "converged_points": sum(
                                                 s[0] for s, c in zip(sizes, conv_plain) if c)}
    best = max((k for k in out["paths"] if k != "plain_fp64_one_by_one"), key=lambda k: out["paths"][k]["value"])
    out["value"] = out["paths"][best]["value"]
    out["path"] = best
    out["vs_plain"] = out["value"] / out["paths"]["plain_fp64_one_by_one"]["value"]
    return out


def served_measure(dev, reps, count: int, rate: float, arms):
    """The first `count` requests of the Poisson trace (seed 3) re-timed at `rate` requests/s
    through the serving loop (HBM-budget admission, continuous batching in epochs of the
    persistent solver).  An arm is (name, precision, preconditioner, max requests at once):
    max 1 is the plain per-request path, each request alone."""
    import torch
    from paper_1603_04100_gb300 import inputs as I
    from paper_1603_04100_gb300.serve import Server, requests_from_trace
    trace = I.serving_trace(count=count, seed=3, rate_per_s=rate)
    out = {"config": {"workload": f"served: first {count} requests of the Poisson trace (seed 3) at {rate:g}/s, "
                                  f"N log-uniform 1,000-1,048,576, K 20, 1-8 RHS, 120 GB budget"}, "paths": {}}
    for name, prec, precond, max_active in arms:
        reqs = requests_from_trace(trace)
        warm = requests_from_trace(trace[:2])
        for r in warm:
            r.arrival_s = 0.0
        Server(dev, prec=prec, precond=precond, hbm_budget=120e9, max_active=max_active).serve(warm, realtime=False)
        srv = Server(dev, prec=prec, precond=precond, hbm_budget=120e9, max_active=max_active)
        reps.barrier()
        stats = srv.serve(reqs, realtime=True)
        reps.barrier()
        # the job: every server's points over the slowest server's makespan; latencies the worst rank's
        span_ms = reps.max(stats["makespan_s"] * 1e3)
        stats["points_per_s"] = reps.job_rate(stats["points"], span_ms)
        stats["p50_ms"] = reps.max(stats["p50_ms"])
        stats["p99_ms"] = reps.max(stats["p99_ms"])
        out["paths"][name] = stats
        torch.cuda.empty_cache()
    return out


def _gpu_setup():
    import torch
    from paper_1603_04100_gb300 import build
    from paper_1603_04100_gb300.replicas import Replicas
    build.build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    return dev, Replicas("nccl", dev)


def run_batched(args):
    """256 uneven clouds (2k-262k points, sphere / ellipsoid / torus, K 12 or 20, 4 RHS)."""
    from paper_1603_04100_gb300 import inputs as I
    dev, reps = _gpu_setup()  # N GPUs: N replicas of the batch, timed by the slowest
    out = {"metric": "MVGD points/s, 256-cloud batch (assembly+solve to 1e-8 rel)", "unit": "points/s",
           "n_gpus": reps.world, "scaling": "weak", "data": "synthetic"}
    out.update(batched_measure(dev, reps, I.batched_specs(256, seed=2), args.steps, args.warmup,
                               workload="batched: 256 clouds, N log-uniform 2,000-262,144 (seed 2), "
                                        "sphere/ellipsoid/torus, K in {12, 20}, 4 RHS (x, yz, x^2-y^2, sin x e^y)"))
    if reps.leader:
        print(json.dumps(out))
    reps.close()


def run_served(args):
    """The first --requests requests of the Poisson trace through the serving loop."""
    from paper_1603_04100_gb300 import api
    dev, reps = _gpu_setup()  # N GPUs: N servers, each on its own copy of the trace
    out = {"metric": "MVGD served points/s and latency (assembly+solve to 1e-8 rel)", "unit": "points/s",
           "n_gpus": reps.world, "scaling": "weak", "data": "synthetic"}
    out.update(served_measure(dev, reps, args.requests, args.rate,
                              (("fp32_refine+amg", api.FP32_REFINE, 2, 1024), ("fp64+amg", api.FP64, 2, 1024))))
    best = max(out["paths"], key=lambda k: out["paths"][k]["points_per_s"])
    out["value"] = out["paths"][best]["points_per_s"]
    out["p50_ms"] = out["paths"][best]["p50_ms"]
    out["p99_ms"] = out["paths"][best]["p99_ms"]
    out["path"] = best
    if reps.leader:
        print(json.dumps(out))
    reps.close()


def run_profile_case(n: int, prec: int, iters: int, precond: int):
    """A profiling target (Nsight Compute): kNN + assembly + a solve capped at `iters`
    iterations on a random unit sphere of n points (K = 20), run twice."""
    import torch
    from paper_1603_04100_gb300 import api, build
    from paper_1603_04100_gb300 import inputs as I
    build.build()
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
    print("ok", r.iters, r.outer, "solve %.3f ms, %.1f us per iteration" % (ms, 1e3 * ms / max(1, r.iters[0])))


def main():
    args = parse()
    if args.profile_case:
        run_profile_case(*args.profile_case)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "batched":
        run_batched(args)
        return
    if args.workload == "served":
        run_served(args)
        return
    import torch

    from paper_1603_04100_gb300.replicas import Replicas

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    reps = Replicas("nccl", dev)
    rank, world = reps.rank, reps.world

    from paper_1603_04100_gb300 import api, build
    from paper_1603_04100_gb300 import inputs as I
    from paper_1603_04100_gb300.pipeline import Pipeline
    build.build()

    n, k = args.n, args.k
    pr = I.random_sphere_problem(n, k, seed=SEED)
    pts = torch.from_numpy(pr.pts).to(dev)
    f = torch.from_numpy(pr.f).to(dev)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(1 << 30, dtype=torch.uint8, device=dev)  # also outlasts the host's first launches

    barrier = reps.barrier

    def timed_runs(pipe, steps, warmup):
        """Per-step CUDA-event times of knn / assembly / solve on the pipeline's stream."""
        for _ in range(warmup):
            with torch.cuda.stream(stream):
                pipe.run(pts, f)
        barrier()
        rec = []
        t_wall = time.perf_counter()
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
                ev[0].record(stream)
                pipe.run_staged(pts, f, ev)
                ev[4].record(stream)
            rec.append(ev)
        barrier()
        wall = time.perf_counter() - t_wall
        out = []
        for ev in rec:  # kNN, assembly, solve stage (set-up + solver), solver call alone
            out.append((ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[4]),
                        ev[3].elapsed_time(ev[4])))
        return out, wall

    max_over_ranks = reps.max

    # Precision strategies (FP32 inner + FP64 refinement, or plain FP64) times
    # preconditioners (row abs-sum scaling, or one multigrid V-cycle), all through
    # the same pipeline (same kNN, locality order, stopping test); the fastest is
    # the headline value.
    names = [p.strip() for p in args.paths.split(",") if p.strip()]
    if args.no_plain:
        names = [p for p in names if p.startswith("fp32_refine")]
    # launch shapes (kNN cell edge, assembly warps a block, solver blocks a SM and
    # staged slices) chosen by timing on this cloud, before any timed step; they
    # change no result (tests/test_gpu_tune.py)
    from paper_1603_04100_gb300 import tune
    tuning, tuning_source = tune.Tuning(), "library defaults"
    if not args.no_tune:
        cached = tune.shape_key(n, k, api.FP32_REFINE, 2, dev) in tune.load_cache()
        tp = Pipeline(n, k, 1, prec=api.FP32_REFINE, device=dev, precond=2, rtol=RTOL, stream=stream)
        with torch.cuda.stream(stream):
            tuning = tune.tune_pipeline(tp, pts, f)
        tuning_source = "cache" if cached else "searched on this cloud"
        del tp
    tuning.apply()
    results = {}
    with ClockSampler(local) as clk:
        for name in names:
            prec = api.FP32_REFINE if name.startswith("fp32_refine") else api.FP64
            precond = 2 if name.endswith("+amg") else 1
            pipe = Pipeline(n, k, 1, prec=prec, device=dev, precond=precond, rtol=RTOL, stream=stream)
            pipe.knn_cell = tuning.knn_cell
            rec, _ = timed_runs(pipe, args.steps, args.warmup)
            info = pipe.decode()[0]
            u = pipe.u[:, 0].double().cpu().numpy()
            step_ms = [r[0] + r[1] + r[2] for r in rec]
            results[name] = {"pipe": pipe, "rec": rec, "info": info, "u": u, "step_ms": step_ms,
                             "ms": max_over_ranks(statistics.mean(step_ms)), "mixed": prec == api.FP32_REFINE,
                             "amg": precond == 2}
            if precond == 2:
                H = api.Hierarchy(n, k, 1.0, pipe.ws_amg, pipe.op)
                results[name]["amg_coarse"] = amg_coarse_bytes(H, n)
                results[name]["amg_levels"] = [int(H.info(lv).n) for lv in range(H.levels)]
                results[name]["amg_width_max"] = int(H.info(0).width_max)
    clocks = clk.summary()
    best = min(results, key=lambda nm: results[nm]["ms"])
    R = results[best]
    t_max = R["ms"]
    value = reps.job_rate(n, t_max)
    info, rec, step_ms = R["info"], R["rec"], R["step_ms"]
    err_exact = float(abs(R["u"] - pr.u_exact[:, 0]).max())

    # roofline of the dominant kernel: the persistent solver of the headline path, timed
    # as the mvgd_solve call (request set-up, the k_solve launch, the scatter of u)
    solve_ms = statistics.mean(r[3] for r in rec)
    mixed_best = R["mixed"]
    bytes_solve = solver_bytes_per_row(k, mixed_best, info[0], info[1], R.get("amg_coarse")) * n
    peak, peak_kind = measured_peaks()
    achieved = bytes_solve / (solve_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": (KSOLVE_MIXED_AMG_DRAM_PER_ITERATION * info[0]
                            if KSOLVE_MIXED_AMG_DRAM_PER_ITERATION is not None and best == "fp32_refine+amg"
                            and n == N_DEFAULT and k == K_DEFAULT else None),
                "traffic_note": "ncu DRAM bytes per iteration of the same kernel on this workload x the launch's "
                                "iterations; below the algorithmic bytes because the Krylov vectors stay in L2",
                "kernel": "k_solve (persistent BiCGSTAB, " + ("FP32 inner + FP64 refinement" if mixed_best else "FP64")
                          + (", multigrid V-cycle preconditioner)" if R["amg"] else ", row scaling)"),
                "peak_kind": f"hbm_gbs of {peak_kind}", "bytes_per_launch": bytes_solve, "launch_ms": solve_ms,
                "note": "launch_ms is the mvgd_solve call: the k_solve launch plus its request set-up and "
                        "solution scatter (the multigrid set-up is timed apart, in stage_ms.amg_setup)"}

    def summary(nm):
        r = results[nm]
        extra = {}
        if r["amg"]:
            extra = {"amg_levels": r["amg_levels"], "amg_width_max": r["amg_width_max"],
                     "amg_coarse_bytes_per_row": r["amg_coarse"]}
        return {**extra, "value": reps.job_rate(n, r["ms"]), "ms_per_step": r["ms"], "iters": r["info"][0],
                "outer": r["info"][1], "relres": r["info"][2], "status": r["info"][3],
                "err_exact_inf": float(abs(r["u"] - pr.u_exact[:, 0]).max()),
                "stage_ms": {"knn": statistics.mean(x[0] for x in r["rec"]),
                             "assemble": statistics.mean(x[1] for x in r["rec"]),
                             "solve": statistics.mean(x[2] for x in r["rec"]),
                             "amg_setup": statistics.mean(x[2] - x[3] for x in r["rec"]),
                             "solver": statistics.mean(x[3] for x in r["rec"])}}

    line = {
        "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if mixed_best else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "k": k, "rtol": RTOL,
                   "precond": "multigrid V(1,1)-cycle (aggregation)" if R["amg"] else "row abs-sum scaling",
                   "path": best, "l2": "flushed before every step (1 GiB write), outside the step events",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "p50_ms": statistics.median(step_ms),
        "p99_ms": sorted(step_ms)[min(len(step_ms) - 1, math.ceil(0.99 * len(step_ms)) - 1)],
        "stage_ms": {"knn": statistics.mean(r[0] for r in rec), "assemble": statistics.mean(r[1] for r in rec),
                     "solve": statistics.mean(r[2] for r in rec),
                     "amg_setup": statistics.mean(r[2] - r[3] for r in rec), "solver": solve_ms},
        "iters": info[0], "outer": info[1], "relres": info[2], "solve_status": info[3],
        "err_exact_inf": err_exact,
        "gpu_launches": R["pipe"].kernels_per_run * args.steps + args.steps,  # + one flush per step
        "roofline": roofline, "clocks": clocks,
        "tuning": {**tuning.__dict__, "source": tuning_source},
        "paths": {nm: summary(nm) for nm in results},
    }
    if "fp64" in results:
        b = results["fp64"]["u"]
        for nm in results:
            if nm != "fp64":
                a = results[nm]["u"]
                line["paths"][nm]["solution_rel_diff_vs_fp64"] = float(
                    ((a - b) ** 2).sum() ** 0.5 / max((b ** 2).sum() ** 0.5, 1e-300))
        line["speedup_vs_plain_fp64_rowscale"] = {nm: results["fp64"]["ms"] / results[nm]["ms"] for nm in results}
    mixed = R["pipe"]

    # a6 on its own: the standalone operator application on the assembled 1M operators
    # (FP32 difference form on hi weights, FP64 standard form), L2 flushed before each launch
    line["spmv"] = spmv_roofline(results, n, k, flush, stream, peak, peak_kind)
    line["row_signs"] = row_sign_stats(pts, mixed, k, flush, stream)
    if not args.no_extras:
        line["dirichlet_hemisphere"] = dirichlet_hemisphere(n, k, flush, stream)
        line["neumann_hemisphere"] = neumann_hemisphere(n, k, flush, stream)
        line["lb_eigenvalues"] = lb_eigen_stats(k, stream)
        line["gauss_seidel_spectral_radius"] = gs_spectral_stats(k, stream)
        from paper_1603_04100_gb300 import inputs as I
        # the batched workload's K = 20 clouds (all of them converge to 1e-8; the K = 12 ones are
        # reported by --workload batched), one batch against the plain path one cloud at a time
        line["batched_k20"] = batched_measure(
            dev, reps, [sp for sp in I.batched_specs(256, seed=2) if sp.k == 20], 2, 1,
            arms=(("fp32_refine+amg", api.FP32_REFINE, 2),),
            workload="the K = 20 clouds of the batched workload (256 clouds, seed 2): sphere/ellipsoid/torus, "
                     "N log-uniform 2,000-262,144, 4 RHS")
        # the serving loop below saturation: continuous batching against the plain
        # per-request FP64 path (one request at a time, row scaling)
        line["served"] = served_measure(dev, reps, SERVED_REQUESTS, SERVED_RATE,
                                        (("fp32_refine+amg", api.FP32_REFINE, 2, 1024),
                                         ("plain_fp64_per_request", api.FP64, 1, 1)))
        sv = line["served"]["paths"]
        line["served"]["vs_plain_points_per_s"] = (sv["fp32_refine+amg"]["points_per_s"]
                                                   / sv["plain_fp64_per_request"]["points_per_s"])

    if not args.no_e2e:
        pts_h = torch.from_numpy(pr.pts).pin_memory()
        f_h = torch.from_numpy(pr.f).pin_memory()
        u_h = torch.empty((n, 1), dtype=torch.float64).pin_memory()
        with torch.cuda.stream(stream):
            mixed.run_host(pts_h, f_h, u_h)
        barrier()
        e_ms = []
        for _ in range(max(1, args.steps)):
            with torch.cuda.stream(stream):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                mixed.run_host(pts_h, f_h, u_h)
                e1.record(stream)
            e1.synchronize()
            e_ms.append(e0.elapsed_time(e1))
        emean = max_over_ranks(statistics.mean(e_ms))
        line["e2e"] = {"value": reps.job_rate(n, emean), "unit": "points/s",
                       "h2d_bytes_per_step": pts_h.numel() * 8 + f_h.numel() * 8,
                       "d2h_bytes_per_step": u_h.numel() * 8, "ms_per_step": emean,
                       "api": "Pipeline.run_host (mvgd_knn, mvgd_assemble, mvgd_solve via ctypes)"}

    if rank == 0 and world == 1 and not args.no_cpu:  # the oracle on the host: at N = 1 only
        if ORACLE_ITERS_FILE.exists() and "multigrid" in json.loads(ORACLE_ITERS_FILE.read_text()):
            samp = OracleSampler(n, k)
            line["cpu_baseline"] = samp.summarise([samp.sample()])
    if reps.leader:
        print(json.dumps(line), flush=True)
    reps.close()


if __name__ == "__main__":
    main()
