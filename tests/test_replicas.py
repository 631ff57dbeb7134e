"""The replica bookkeeping of multi-GPU runs on CPU: two gloo ranks, each with its
own step time, agree on the slowest rank's time and on the whole-job rate."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    from paper_1603_04100_gb300.replicas import Replicas
    reps = Replicas("gloo")
    reps.barrier()
    ms = 10.0 + 5.0 * rank            # rank 1 is the slower one
    t = reps.max(ms)
    out.put((rank, reps.leader, t, reps.job_rate(1000, t)))
    reps.barrier()
    reps.close()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[0] for g in got] == [0, 1] and [g[1] for g in got] == [True, False]
    for _, _, t, rate in got:
        assert t == 15.0
        assert rate == 2 * 1000 / 15e-3   # both ranks' points over the slowest rank's time


def test_single_process_needs_no_group(monkeypatch):
    for v in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(v, raising=False)
    from paper_1603_04100_gb300.replicas import Replicas
    reps = Replicas("gloo")
    assert reps.world == 1 and reps.leader
    reps.barrier()
    assert reps.max(3.5) == 3.5 and reps.job_rate(100, 2.0) == 100 / 2e-3
    reps.close()
