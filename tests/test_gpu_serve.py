"""Serving: requests arriving over time join the running batch as memory
frees up, and every result is bit-identical to the same request solved alone."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1603_04100_gb300 import inputs as I
from tests.gpu_util import cuda_or_skip

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return cuda_or_skip()


def _requests():
    from paper_1603_04100_gb300.serve import requests_from_trace
    specs = I.serving_trace(count=14, seed=7, rate_per_s=60.0, n_lo=1000, n_hi=40000, k=20)
    return requests_from_trace(specs)


def _solo(dev, r, precond):
    from paper_1603_04100_gb300 import api
    pts = torch.from_numpy(r.pts).to(dev)
    nbr, order = api.knn(pts, r.k, want_order=True)
    op = api.assemble(pts, nbr, prec=api.FP32_REFINE, order=order)
    res = api.solve(op, torch.from_numpy(np.ascontiguousarray(r.f)).to(dev), rtol=1e-8, precond=precond)
    return res.u.cpu().numpy(), res


@pytest.mark.parametrize("precond", [1, 2])
def test_serving_joins_and_identity(dev, precond):
    # precond 2: each admitted request's hierarchy is built on the server's stream
    # pool; the result still equals the request solved alone, bit for bit
    from paper_1603_04100_gb300.serve import Server, request_bytes
    reqs = _requests()
    big = sorted(request_bytes(r.n, r.k, r.nrhs, 1, precond) for r in reqs)
    # room for a few requests at once, so that later ones must wait (multigrid
    # requests finish in fewer epochs: less room)
    budget = sum(big[-4:]) if precond == 1 else sum(big[-2:])
    srv = Server(dev, hbm_budget=budget, epoch_iters=16, max_points=1 << 16, max_k=20, precond=precond)
    # requests can finish before the next one arrives (on a fast enough solver):
    # queue them all at once, so that the budget makes later ones wait
    for r in reqs:
        r.arrival_s = 0.0
    stats = srv.serve(reqs)
    assert stats["statuses"] == [0], stats
    assert stats["joins"] > 0 and stats["max_concurrent"] >= 2, stats
    assert stats["waited_request_epochs"] > 0, stats
    assert srv.used == 0
    for r in reqs:
        u, res = _solo(dev, r, precond)
        assert np.array_equal(u, r.u), r.rid
        assert [i[0] for i in r.info] == res.iters
    assert stats["p99_ms"] >= stats["p50_ms"] > 0


def test_serving_rejects_request_larger_than_budget(dev):
    from paper_1603_04100_gb300.serve import Server
    reqs = _requests()[:2]
    srv = Server(dev, hbm_budget=1e5, max_points=1 << 16, max_k=20)
    with pytest.raises(RuntimeError):
        srv.serve(reqs, realtime=False)
