"""Launch-shape autotuner for one cloud's pipeline.

It times, on the caller's own cloud, the knobs that change how fast a call
runs but never what it computes:
  * the kNN search grid's cell edge, as a multiple of the library's estimate
    (the neighbour lists are exact for any cell size);
  * warps per block of the assembly kernels (every row is one lane's work);
  * resident blocks per SM and staged operator slices per warp of the
    persistent solver (its reductions run over fixed chunks whatever the grid);
and keeps the fastest setting of each, one knob at a time in that order.  The
choice is cached in a JSON file keyed by (GPU name, N rounded to a power of
two, K, precision, preconditioner): a later run of the same shape applies it
without searching.  Cache file: $MVGD_TUNE_CACHE, else
~/.cache/mvgd_gb300/tune.json.

    tuning = tune_pipeline(pipe, pts, f)   # times, caches, applies
    tuning.apply()                         # process-wide launch shapes
    Tuning().apply()                       # back to the library's defaults
"""
from __future__ import annotations

import json
import math
import os
import statistics
from dataclasses import asdict, dataclass
from pathlib import Path

import torch

from . import _lib as LB

CELL_FACTORS = (0.7, 0.85, 1.0, 1.2, 1.45)
ASSEMBLE_WARPS = (1, 2, 4)
SOLVER_SHAPES = ((0, 1), (0, 2), (2, 1), (2, 2), (1, 1))  # (blocks per SM, 0 = all that fit; stage buffers)


@dataclass
class Tuning:
    cell_factor: float = 1.0
    assemble_warps: int = 1
    solver_blocks_per_sm: int = 0
    stage_buffers: int = 1

    def apply(self) -> None:
        """Set the library's process-wide launch shapes (mvgd_set_launch_tuning)."""
        LB.check("mvgd_set_launch_tuning", LB.load().mvgd_set_launch_tuning(
            int(self.solver_blocks_per_sm), int(self.stage_buffers), int(self.assemble_warps)))

    @property
    def knn_cell(self) -> float:
        """The mvgd_knn cell_size argument: a negative multiple of the library's estimate."""
        return 0.0 if self.cell_factor == 1.0 else -float(self.cell_factor)


def cache_path() -> Path:
    env = os.environ.get("MVGD_TUNE_CACHE")
    return Path(env) if env else Path.home() / ".cache" / "mvgd_gb300" / "tune.json"


def shape_key(n: int, k: int, prec: int, precond: int, device=None) -> str:
    name = torch.cuda.get_device_name(device) if torch.cuda.is_available() else "cpu"
    return f"{name}|n2^{round(math.log2(max(n, 2)))}|k{k}|prec{prec}|precond{precond}"


def load_cache(path: Path | None = None) -> dict:
    path = path or cache_path()
    try:
        return json.loads(path.read_text())
    except (OSError, ValueError):
        return {}


def save_cache(entries: dict, path: Path | None = None) -> None:
    path = path or cache_path()
    path.parent.mkdir(parents=True, exist_ok=True)
    tmp = path.with_suffix(f".{os.getpid()}.tmp")
    tmp.write_text(json.dumps(entries, indent=1, sort_keys=True) + "\n")
    os.replace(tmp, path)


def _time_ms(fn, stream, reps: int) -> float:
    """Median CUDA-event time of fn() on `stream`, after one untimed call."""
    fn()
    out = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return statistics.median(out)


def tune_pipeline(pipe, pts: torch.Tensor, f: torch.Tensor, *, reps: int = 3, use_cache: bool = True) -> Tuning:
    """Choose, apply and cache the launch shapes for `pipe` (a Pipeline) on this cloud."""
    key = shape_key(pipe.n, pipe.k, pipe.prec, pipe.precond, pipe.device)
    entries = load_cache() if use_cache else {}
    if key in entries:
        t = Tuning(**entries[key]["tuning"])
        t.apply()
        pipe.knn_cell = t.knn_cell
        return t
    st = pipe._stream()
    t = Tuning()
    t.apply()
    timings = {}

    def knn_with(c):
        pipe.knn_cell = Tuning(cell_factor=c).knn_cell
        return _time_ms(lambda: pipe.knn_call(pts), st, reps)

    timings["cell_factor"] = {str(c): knn_with(c) for c in CELL_FACTORS}
    t.cell_factor = float(min(CELL_FACTORS, key=lambda c: timings["cell_factor"][str(c)]))
    pipe.knn_cell = t.knn_cell
    pipe.knn_call(pts)

    def asm_with(w):
        Tuning(t.cell_factor, w, t.solver_blocks_per_sm, t.stage_buffers).apply()
        return _time_ms(lambda: pipe.assemble_call(pts), st, reps)

    timings["assemble_warps"] = {str(w): asm_with(w) for w in ASSEMBLE_WARPS}
    t.assemble_warps = int(min(ASSEMBLE_WARPS, key=lambda w: timings["assemble_warps"][str(w)]))
    t.apply()
    pipe.assemble_call(pts)
    pipe.amg_call()

    def solve_with(shape):
        Tuning(t.cell_factor, t.assemble_warps, shape[0], shape[1]).apply()
        return _time_ms(lambda: pipe.solve_call(f), st, max(1, reps - 1))

    timings["solver"] = {f"{b},{s}": solve_with((b, s)) for b, s in SOLVER_SHAPES}
    b, s = min(SOLVER_SHAPES, key=lambda sh: timings["solver"][f"{sh[0]},{sh[1]}"])
    t.solver_blocks_per_sm, t.stage_buffers = int(b), int(s)
    t.apply()
    if use_cache:
        entries = load_cache()
        entries[key] = {"tuning": asdict(t), "timings_ms": timings}
        save_cache(entries)
    return t
