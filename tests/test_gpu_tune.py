"""The launch-shape tuner changes speed, never results: neighbour lists, order,
weights and solutions are bit-identical under every shape it can choose, and
its choice is cached and reused."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1603_04100_gb300 import inputs as I
from tests.gpu_util import cuda_or_skip

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _run(pipe, pts, f):
    pipe.run(pts, f)
    torch.cuda.synchronize()
    lo = pipe.op.val_lo.clone() if pipe.op.val_lo is not None else torch.zeros(1)
    return pipe.nbr.clone(), pipe.order.clone(), pipe.op.val.clone(), lo, pipe.u.clone(), pipe.decode()


def _same(a, b):
    for x, y in zip(a[:5], b[:5]):
        assert torch.equal(x, y)
    assert a[5] == b[5]


@pytest.mark.parametrize("prec_name", ["FP32_REFINE", "FP64"])
def test_every_launch_shape_gives_the_same_bits(prec_name):
    dev = cuda_or_skip()
    from paper_1603_04100_gb300 import api
    from paper_1603_04100_gb300.pipeline import Pipeline
    from paper_1603_04100_gb300.tune import Tuning
    pr = I.random_sphere_problem(200_000, 20, seed=4)
    pts, f = torch.from_numpy(pr.pts).to(dev), torch.from_numpy(pr.f).to(dev)
    pipe = Pipeline(pr.n, 20, 1, prec=getattr(api, prec_name), device=dev, precond=2)
    try:
        Tuning().apply()
        ref = _run(pipe, pts, f)
        assert ref[5][0][3] == 0
        for t in (Tuning(0.7, 4, 1, 2), Tuning(1.45, 2, 2, 1), Tuning(0.85, 8, 0, 2)):
            t.apply()
            pipe.knn_cell = t.knn_cell
            _same(_run(pipe, pts, f), ref)
    finally:
        Tuning().apply()


def test_tuner_caches_its_choice(tmp_path, monkeypatch):
    dev = cuda_or_skip()
    from paper_1603_04100_gb300 import api
    from paper_1603_04100_gb300 import tune
    from paper_1603_04100_gb300.pipeline import Pipeline
    monkeypatch.setenv("MVGD_TUNE_CACHE", str(tmp_path / "tune.json"))
    pr = I.random_sphere_problem(100_000, 20, seed=5)
    pts, f = torch.from_numpy(pr.pts).to(dev), torch.from_numpy(pr.f).to(dev)
    pipe = Pipeline(pr.n, 20, 1, prec=api.FP32_REFINE, device=dev, precond=2)
    try:
        ref = _run(pipe, pts, f)
        t1 = tune.tune_pipeline(pipe, pts, f, reps=2)
        key = tune.shape_key(pr.n, 20, api.FP32_REFINE, 2, dev)
        cached = tune.load_cache()
        assert key in cached and cached[key]["tuning"]["cell_factor"] == t1.cell_factor
        assert set(cached[key]["timings_ms"]) == {"cell_factor", "assemble_warps", "solver"}
        _same(_run(pipe, pts, f), ref)
        t2 = tune.tune_pipeline(pipe, pts, f)  # from the cache: no search
        assert t2 == t1
    finally:
        tune.Tuning().apply()
