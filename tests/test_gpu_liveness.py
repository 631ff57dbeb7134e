"""The bounded device-side waits of the persistent kernels end their launch with
MVGD_ETIMEOUT instead of hanging, and the next call on the same workspace runs
normally.

A one-launch test control (mvgd_test_withhold_arrival) leaves one block's
arrival at the solver's first grid barrier out, or never publishes row 0's
first flag in the Gauss-Seidel forward substitution: waits that nothing ends,
so they run out at a short poll limit (mvgd_set_wait_limit).  No memory is
touched that a normal launch would not touch, nothing traps or faults.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_1603_04100_gb300 import inputs as I
from tests.gpu_util import cuda_or_skip

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHORT = 1 << 14  # polls: a few ms to tens of ms


@pytest.fixture
def api_limits():
    from paper_1603_04100_gb300 import api
    yield api
    api.withhold_arrival(False)
    api.set_wait_limit(0)


def _operator(api, dev, n=6000, k=16, prec_name="FP64"):
    pr = I.random_sphere_problem(n, k, seed=21)
    pts = torch.from_numpy(pr.pts).to(dev)
    nbr, order = api.knn(pts, k, want_order=True)
    op = api.assemble(pts, nbr, prec=getattr(api, prec_name), order=order)
    return pr, op


@pytest.mark.parametrize("prec_name,precond", [("FP64", 1), ("FP32_REFINE", 2), ("FP64", 2)])
def test_solver_barrier_wait_runs_out_then_recovers(api_limits, prec_name, precond):
    api = api_limits
    dev = cuda_or_skip()
    from paper_1603_04100_gb300 import _lib as LB
    pr, op = _operator(api, dev, prec_name=prec_name)
    f = torch.from_numpy(pr.f).to(dev)
    amg = api.amg_setup(op, 1.0) if precond == 2 else None
    need = LB.load().mvgd_solve_workspace_bytes(op.n, op.k, 1, op.prec, precond)
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    api.set_wait_limit(SHORT)
    api.withhold_arrival(True)
    bad = api.solve(op, f, rtol=1e-10, precond=precond, amg=amg, workspace=ws)
    assert bad.status == [LB.ETIMEOUT], bad.status
    # the control was one-shot and the limit goes back to the default: the same
    # workspace, the same context, a normal solve
    api.set_wait_limit(0)
    good = api.solve(op, f, rtol=1e-10, precond=precond, amg=amg, workspace=ws)
    assert good.status == [0] and good.relres[0] <= 1e-10, (good.status, good.relres)
    ref = api.solve(op, f, rtol=1e-10, precond=precond, amg=amg)
    assert torch.equal(good.u, ref.u)  # a timed-out launch leaves nothing behind


def test_batched_launch_wait_runs_out_then_recovers(api_limits):
    api = api_limits
    dev = cuda_or_skip()
    from paper_1603_04100_gb300 import _lib as LB
    from paper_1603_04100_gb300.batch import BatchPipeline
    sizes = [(5000, 20, 1), (3000, 16, 2)]
    clouds = [I.random_sphere(5000, 50), I.torus(3000, 51)]
    fs = [np.stack([c[:, 0], c[:, 2]][:q], axis=1).copy() for c, (_, _, q) in zip(clouds, sizes)]
    pts = [torch.from_numpy(c).to(dev) for c in clouds]
    ft = [torch.from_numpy(x).to(dev) for x in fs]
    bp = BatchPipeline(sizes, prec=api.FP32_REFINE, precond=2, device=dev)
    api.set_wait_limit(SHORT)
    api.withhold_arrival(True)
    bp.run(pts, ft)
    torch.cuda.synchronize()
    for info in bp.infos():
        assert all(st == LB.ETIMEOUT for _, _, _, st in info), info
    api.set_wait_limit(0)
    bp.run(pts, ft)
    torch.cuda.synchronize()
    for info in bp.infos():
        assert all(st == 0 and rel <= 1e-8 for _, _, rel, st in info), info


def test_gs_power_flag_wait_runs_out_then_recovers(api_limits):
    api = api_limits
    dev = cuda_or_skip()
    from paper_1603_04100_gb300 import _lib as LB
    _, op = _operator(api, dev, n=4000, k=20)
    x0 = torch.from_numpy(np.random.default_rng(3).standard_normal(op.n)).to(dev)
    api.set_wait_limit(SHORT)
    api.withhold_arrival(True)
    bad = api.gs_power(op, x0, 20)
    assert bad.status == LB.ETIMEOUT, bad.status
    api.set_wait_limit(0)
    good = api.gs_power(op, x0, 20)
    again = api.gs_power(op, x0, 20)
    assert good.status == 0 and np.all(np.isfinite(good.nu))
    assert np.array_equal(good.nu, again.nu)  # bit-repeatable, as before the timed-out launch
