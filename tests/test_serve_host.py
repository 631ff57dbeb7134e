"""The serving loop's host logic on CPU: admission in arrival order under the
HBM budget and the slot limit, joins while others run, waiting, retirement and
the statistics.  The device steps (admission work, solver epochs, retirement)
are replaced by a model in which each request needs a given number of epochs."""
from __future__ import annotations

import time
from types import SimpleNamespace

import numpy as np
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def serve_mod():
    from paper_1603_04100_gb300 import build
    build.build()  # request_bytes asks the library for the operator and workspace sizes
    from paper_1603_04100_gb300 import serve
    return serve


def _requests(serve_mod, sizes, arrivals=None):
    out = []
    for i, n in enumerate(sizes):
        pts = np.zeros((n, 3))
        f = np.zeros((n, 1 + i % 3))
        out.append(serve_mod.Request(i, 0.0 if arrivals is None else arrivals[i], pts, f, 20))
    return out


def _fake(serve_mod, budget, need, max_active=1024, precond=1):
    class Fake(serve_mod.Server):
        def __init__(self):  # bookkeeping only: no device, no streams
            self.budget, self.prec, self.precond, self.max_active = float(budget), 1, precond, max_active
            self.used, self.epochs, self.launches, self.joins, self.max_concurrent, self.waited = 0.0, 0, 0, 0, 0, 0
            self.peak_used, self.admitted, self.retired = 0.0, [], []

        def _admit(self, reqs):
            self.peak_used = max(self.peak_used, self.used)
            self.admitted.append([r.rid for r in reqs])
            return [SimpleNamespace(req=r, left=need[r.rid],
                                    nbytes=serve_mod.request_bytes(r.n, r.k, r.nrhs, self.prec, self.precond))
                    for r in reqs]

        def _epoch(self, active):
            self.epochs += 1
            for x in active:
                x.left -= 1
            return [i for i, x in enumerate(active) if x.left <= 0]

        def _retire(self, x, t0):
            x.req.u = np.zeros_like(x.req.f)
            x.req.info = [(1, 1, 0.0, 0)] * x.req.nrhs
            x.req.done_s = time.perf_counter() - t0 + 1e-9
            self.retired.append(x.req.rid)
            self.used -= x.nbytes

    return Fake()


def test_budget_is_never_exceeded_and_requests_wait(serve_mod):
    sizes = [4000, 9000, 2500, 12000, 3000, 7000, 5000, 1000]
    reqs = _requests(serve_mod, sizes)
    nbytes = [serve_mod.request_bytes(n, 20, r.nrhs, 1, 1) for n, r in zip(sizes, reqs)]
    budget = sorted(nbytes)[-1] + sorted(nbytes)[-2]  # room for two large or several small
    srv = _fake(serve_mod, budget, need={i: 1 + (i * 3) % 4 for i in range(len(sizes))})
    stats = srv.serve(reqs, realtime=False)
    assert srv.peak_used <= budget and srv.used == 0
    assert sorted(srv.retired) == list(range(len(sizes)))
    # admission is first come, first served: the admitted ids, in order, are 0, 1, 2, ...
    assert [rid for batch in srv.admitted for rid in batch] == list(range(len(sizes)))
    assert stats["waited_request_epochs"] > 0 and stats["joins"] > 0
    assert stats["requests"] == len(sizes) and stats["points"] == sum(sizes)
    assert stats["statuses"] == [0] and stats["p99_ms"] >= stats["p50_ms"] > 0


def test_slot_limit_bounds_the_active_set(serve_mod):
    reqs = _requests(serve_mod, [1000] * 10)
    srv = _fake(serve_mod, 1e15, need={i: 2 for i in range(10)}, max_active=3)
    stats = srv.serve(reqs, realtime=False)
    assert stats["max_concurrent"] == 3
    assert all(len(b) <= 3 for b in srv.admitted)
    assert srv.epochs == 2 * 4  # ten requests of two epochs, three at a time: 3 + 3 + 3 + 1


def test_request_over_the_budget_is_rejected(serve_mod):
    reqs = _requests(serve_mod, [1000, 50000])
    small = serve_mod.request_bytes(1000, 20, 1, 1, 1)
    srv = _fake(serve_mod, small * 1.5, need={0: 1, 1: 1})
    with pytest.raises(RuntimeError):
        srv.serve(reqs, realtime=False)


def test_multigrid_requests_hold_their_hierarchy(serve_mod):
    # precond 2 reserves the multigrid workspace on top of the request's own bytes
    L = serve_mod.LB.load()
    a = serve_mod.request_bytes(20000, 20, 2, 1, 1)
    b = serve_mod.request_bytes(20000, 20, 2, 1, 2)
    assert b - a >= L.mvgd_amg_workspace_bytes(20000, 20)
    assert serve_mod.amg_levels(512) == 1 and serve_mod.amg_levels(513) == 2 and serve_mod.amg_levels(1 << 20) == 5
