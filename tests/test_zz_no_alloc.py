"""mvgd_knn_noalloc, the kNN entry point that allocates nothing.

Callers that may not allocate device memory (code recorded into a CUDA graph,
loops that must not wait on the allocator, frameworks that own every device
buffer) pass only inputs and outputs; the call's scratch is a static device
array of the library.  Its results must equal mvgd_knn's exactly (neighbour
lists are integer results), call after call, since every call reuses the same
array and inherits the previous call's contents.  Collected last, so a run that
stops at the first failure has already run every other test.
"""
from __future__ import annotations

import ctypes as C

import pytest

from paper_1603_04100_gb300 import inputs as I
from tests.gpu_util import cuda_or_skip

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_POINTS = 65536  # MVGD_KNN_NOALLOC_MAX_POINTS in include/mvgd.h


def _noalloc(L, pts, k):
    from paper_1603_04100_gb300 import api
    n = pts.shape[0]
    nbr = torch.full((n, k), -1, dtype=torch.int32, device=pts.device)
    order = torch.full((n,), -1, dtype=torch.int32, device=pts.device)
    st = L.mvgd_knn_noalloc(api._vp(pts), n, k, api._vp(nbr), api._vp(order), 0.0, api._stream())
    torch.cuda.synchronize()
    return st, nbr, order


def test_noalloc_knn_equals_knn_on_consecutive_calls():
    dev = cuda_or_skip()
    from paper_1603_04100_gb300 import _lib as LB
    from paper_1603_04100_gb300 import api
    L = LB.load()
    clouds = [(I.torus(5000, 3), 16), (I.random_sphere(MAX_POINTS, 4), 20), (I.torus(5000, 3), 16)]
    for pts_np, k in clouds:  # back to back: each call inherits the previous call's scratch contents
        pts = torch.from_numpy(pts_np).to(dev)
        want, want_order = api.knn(pts, k, want_order=True)
        st, nbr, order = _noalloc(L, pts, k)
        assert st == LB.OK, LB.status_string(st)
        assert torch.equal(nbr, want)
        assert torch.equal(order, want_order)  # the exported row order too, element for element


def test_noalloc_knn_refuses_clouds_above_its_maximum():
    dev = cuda_or_skip()
    from paper_1603_04100_gb300 import _lib as LB
    L = LB.load()
    pts = torch.from_numpy(I.random_sphere(MAX_POINTS + 1, 5)).to(dev)
    st, nbr, _ = _noalloc(L, pts, 12)
    assert st == LB.EINVAL
    assert bool((nbr == -1).all())  # nothing was written
