"""Replicas across GPUs: one process per GPU, each solving its own clouds.

The MVGD path has no step that exchanges data between clouds, so N GPUs run N
independent replicas; the only collectives are the ones that time the job: a
barrier on both sides of the timed region and the maximum of the step time
over the ranks.  The whole-job rate is the units every rank processed divided
by that maximum (weak scaling: the work per rank is fixed).
"""
from __future__ import annotations

import os

import torch
import torch.distributed as dist


class Replicas:
    """Rank bookkeeping from the launcher's environment (RANK, WORLD_SIZE, LOCAL_RANK)."""

    def __init__(self, backend: str = "nccl", device: torch.device | None = None):
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.device = device if device is not None else torch.device("cpu")
        self._own = False
        if self.world > 1 and not dist.is_initialized():
            dist.init_process_group(backend)
            self._own = True

    @property
    def leader(self) -> bool:
        return self.rank == 0

    def barrier(self) -> None:
        if self.device.type == "cuda":
            torch.cuda.synchronize(self.device)
        if self.world > 1:
            dist.barrier()

    def max(self, x: float) -> float:
        """The largest x over the ranks (every rank gets it)."""
        if self.world == 1:
            return float(x)
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def job_rate(self, units_per_rank: float, ms_max: float) -> float:
        """Units all ranks processed per second, timed by the slowest rank."""
        return self.world * units_per_rank / (ms_max * 1e-3)

    def close(self) -> None:
        if self._own and dist.is_initialized():
            dist.destroy_process_group()
