"""Host logic of the launch-shape tuner (no GPU): the cache round trip, the
kNN cell argument it passes, and the library's range checks of the shapes."""
import pytest


def test_cache_round_trip(tmp_path, monkeypatch):
    from paper_1603_04100_gb300 import tune
    monkeypatch.setenv("MVGD_TUNE_CACHE", str(tmp_path / "t.json"))
    assert tune.load_cache() == {}
    entries = {"GB300|n2^20|k20|prec1|precond2": {"tuning": {"cell_factor": 0.85, "assemble_warps": 2,
                                                               "solver_blocks_per_sm": 0, "stage_buffers": 1}}}
    tune.save_cache(entries)
    assert tune.load_cache() == entries
    t = tune.Tuning(**entries["GB300|n2^20|k20|prec1|precond2"]["tuning"])
    assert t.knn_cell == -0.85           # a negative cell_size scales the library's estimate
    assert tune.Tuning().knn_cell == 0.0  # 0: the estimate itself


def test_launch_tuning_range_checks():
    from paper_1603_04100_gb300 import _lib as LB, build
    build.build()
    L = LB.load()
    assert L.mvgd_set_launch_tuning(0, 1, 1) == LB.OK
    assert L.mvgd_set_launch_tuning(-1, 1, 1) == LB.EINVAL
    assert L.mvgd_set_launch_tuning(0, 3, 1) == LB.EINVAL
    assert L.mvgd_set_launch_tuning(0, 1, 3) == LB.EINVAL   # warps per block: a power of two <= 8
    assert L.mvgd_set_launch_tuning(2, 2, 4) == LB.OK
    assert L.mvgd_set_launch_tuning(0, 0, 0) == LB.OK      # back to the defaults
