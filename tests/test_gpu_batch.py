"""Batched path: uneven clouds through one assembly launch and one persistent
solve launch.  Each cloud's result is bit-identical to the same cloud solved
alone, a CUDA-graph replay reproduces the eager run, and batched results
match the oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1603_04100_gb300 import inputs as I
from tests.gpu_util import cuda_or_skip

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return cuda_or_skip()


SPECS = [
    I.CloudSpec(I.SPHERE, 2003, 12, 101, ("x", "yz")),
    I.CloudSpec(I.TORUS, 17777, 20, 102, ("x", "yz", "x2-y2", "sinx_expy")),
    I.CloudSpec(I.ELLIPSOID, 5000, 12, 103, ("sinx_expy",)),
    I.CloudSpec(I.SPHERE, 31000, 20, 104, ("p3", "x", "z")),
    I.CloudSpec(I.TORUS, 2500, 16, 105, ("x",)),
    I.CloudSpec(I.ELLIPSOID, 12345, 24, 106, ("yz", "x2-y2")),
]


def _problems():
    return [s.build() for s in SPECS]


def _run_batch(dev, probs, prec, graph=False, rtol=1e-9):
    from paper_1603_04100_gb300.batch import BatchPipeline
    bp = BatchPipeline([(p.n, p.k, p.nrhs) for p in probs], prec=prec, device=dev, rtol=rtol, n_streams=4)
    pts = [torch.from_numpy(p.pts).to(dev) for p in probs]
    fs = [torch.from_numpy(p.f).to(dev) for p in probs]
    if graph:
        bp.capture(pts, fs)
        for s in bp.slots:
            s.u.zero_()
        bp.replay()
    else:
        bp.run(pts, fs)
    torch.cuda.synchronize()
    return bp


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32_refine"])
def test_batch_equals_solo_bitwise(dev, prec):
    from paper_1603_04100_gb300 import api
    probs = _problems()
    bp = _run_batch(dev, probs, prec)
    for slot, p, infos in zip(bp.slots, probs, bp.infos()):
        assert all(i[3] == 0 for i in infos), infos
        pts = torch.from_numpy(p.pts).to(dev)
        nbr, order = api.knn(pts, p.k, want_order=True)
        assert torch.equal(nbr, slot.nbr)
        assert torch.equal(order, slot.order)
        op = api.assemble(pts, nbr, prec=prec, order=order)
        assert np.array_equal(op.weights(), slot.op.weights())
        assert np.array_equal(op.rows("col"), slot.op.rows("col"))
        res = api.solve(op, torch.from_numpy(p.f).to(dev), rtol=1e-9, precond=1)
        assert torch.equal(res.u, slot.u), p.name
        assert res.iters == [i[0] for i in infos]


def test_batch_graph_replay_matches_eager(dev):
    probs = _problems()
    eager = _run_batch(dev, probs, 1)
    graphed = _run_batch(dev, probs, 1, graph=True)
    for a, b in zip(eager.slots, graphed.slots):
        assert torch.equal(a.u, b.u)


def test_batch_matches_oracle(dev):
    """Small randomly sampled clouds with K=12 give operators with cond_2 near
    1e6 (the 2,003-point sphere here: 1.1e6), so a residual of 1e-9 does not
    pin the solution to 1e-8; the forward comparison uses a 1e-11 solve and the
    backward error is checked with the oracle's operator."""
    probs = _problems()
    bp = _run_batch(dev, probs, 1, rtol=1e-11)
    for slot, p in zip(bp.slots, probs):
        nbr = slot.nbr.cpu().numpy()
        np.testing.assert_array_equal(nbr, oracle.knn_grid(p.pts, p.k))
        val, _, _, _ = oracle.assemble(p.pts, nbr)
        u = slot.u.cpu().numpy()
        for q in range(p.nrhs):
            uo, _, _ = oracle.solve(val, nbr, p.f[:, q], rtol=1e-13)
            assert np.linalg.norm(u[:, q] - uo) <= 1e-8 * np.linalg.norm(uo), (p.name, q)
            # the GPU stopped at 1e-11 on its own hi + lo operator, which equals the
            # oracle's to ~1e-12 in the weights: at this level the two residuals
            # differ by ~1e-11, hence the 10x slack on the oracle-side check
            r = p.f[:, q] - oracle.spmv(val, nbr, u[:, q])
            assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(p.f[:, q]), (p.name, q)
