"""The FP32 assembly of the FP32_REFINE format against the FP64 oracle.

The rows of the mixed format are formed on the FP32 pipe: offsets in FP64,
then double-float (FP32 pairs) for the covariance, the h-scaled local
coordinates and the normal equations of the local fits, solved with an FP32
Cholesky factor and refined from double-float residuals; the 3x3 eigenvectors
come from an FP32 Jacobi polished in FP64.  Rows whose fit is ill-conditioned
(or degenerate, or not finite) are formed by the FP64 arithmetic instead.

Bars: hi + lo weights within 1e-10 of the oracle's, row-relative, on every
row with status 0; columns exact; h within 1e-13; row status and the bad-row
count equal to the oracle's; the rows the FP32 path hands over are bit-equal
to the FP64 arithmetic's (rule.arith = 1).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1603_04100_gb300 import inputs as I
from tests.gpu_util import cuda_or_skip, row_relerr
from tests.test_gpu_parity import CLOUDS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W_TOL = 1e-10
CLOUDS_FP32 = dict(CLOUDS)
# far from the origin relative to its spacing: |p| / h about 1e6
CLOUDS_FP32["shifted"] = lambda: I.random_sphere(20001, 7) * 0.01 + np.array([100.0, -50.0, 3.0])


@pytest.fixture(scope="module")
def dev():
    return cuda_or_skip()


def _both_arith(dev, p, k, **kw):
    from paper_1603_04100_gb300 import api
    kw.setdefault("delta_m", min(6, k))
    pt = torch.from_numpy(p).to(dev)
    nbr_t, ord_t = api.knn(pt, k, want_order=True)
    order = ord_t if kw.pop("order", False) else None
    op32 = api.assemble(pt, nbr_t, prec=api.FP32_REFINE, order=order, arith=0, **kw)
    op64 = api.assemble(pt, nbr_t, prec=api.FP32_REFINE, order=order, arith=1, **kw)
    torch.cuda.synchronize()
    return nbr_t.cpu().numpy(), op32, op64


def _stored(a, op):
    return a[op.order.cpu().numpy()] if op.order is not None else a


@pytest.mark.parametrize("name", list(CLOUDS_FP32))
@pytest.mark.parametrize("k", [5, 8, 12, 20, 31])
def test_fp32_assembly_matches_oracle(dev, name, k):
    p = CLOUDS_FP32[name]()
    order = name in ("rand20001", "torus12345")
    nbr, op32, op64 = _both_arith(dev, p, k, order=order)
    val, st, dg, _ = oracle.assemble(p, nbr, delta_m=min(6, k))
    w32, w64 = op32.weights(), op64.weights()
    ok = _stored(st, op32) == 0
    err = row_relerr(w32[ok], _stored(val, op32)[ok])
    assert err.max() <= W_TOL, (err.max(), int(err.argmax()))
    np.testing.assert_array_equal(op32.rows("col"), op64.rows("col"))
    # the rows the oracle flags are flagged; the code itself is the FP64 arithmetic's (on a
    # rank-deficient row the two FP64 codes may overflow differently: status 1 or 2)
    np.testing.assert_array_equal(op32.status.cpu().numpy() != 0, st != 0)
    np.testing.assert_array_equal(op32.status.cpu().numpy(), op64.status.cpu().numpy())
    assert int(op32.bad_rows.item()) == int((st > 0).sum())
    fine = st == 0
    np.testing.assert_allclose(op32.h.cpu().numpy()[fine], dg[fine, 5], rtol=1e-13)
    # rows with a non-zero status were formed by the FP64 arithmetic: bit-equal
    bad = ~ok
    np.testing.assert_array_equal(w32[bad].view(np.int64), w64[bad].view(np.int64))  # NaN rows too
    same = np.all(w32.view(np.int64) == w64.view(np.int64), axis=1)
    if k < 8:  # square or nearly square fits: the FP64 arithmetic throughout
        assert bool(same.all())
    print(f"[{name} k={k}] FP32 path: max row error {err.max():.2e}, median {np.median(err):.2e}; "
          f"rows bit-equal to the FP64 arithmetic {int(same.sum())} of {len(same)}")


@pytest.mark.parametrize("k", [16, 24])
def test_fp32_assembly_quarter_range(dev, k):
    # quarter-range h depends on the tangent axes: rows whose tangent eigen-gap
    # exceeds 1e-6 (elsewhere the axes are not determined)
    from paper_1603_04100_gb300 import api
    p = I.torus(9000, 4)
    nbr, op32, _ = _both_arith(dev, p, k, delta_kind=api.DELTA_QUARTER_RANGE)
    val, st, dg, _ = oracle.assemble(p, nbr, delta_kind=api.DELTA_QUARTER_RANGE)
    ok = (dg[:, 9] > 1e-6) & (st == 0)
    assert ok.mean() > 0.99
    err = row_relerr(op32.weights()[ok], val[ok])
    assert err.max() <= W_TOL, err.max()


@pytest.mark.parametrize("name", ["fib2562", "rand20001", "torus12345"])
def test_fp32_assembly_least_squares_rows(dev, name):
    from paper_1603_04100_gb300 import api
    p = CLOUDS[name]()
    nbr, op32, _ = _both_arith(dev, p, 20, variant=api.ROW_LS)
    val, st, _, _ = oracle.assemble(p, nbr, variant=oracle.VARIANT_LS)
    assert int(st.max()) == 0
    err = row_relerr(op32.weights(), val)
    assert err.max() <= W_TOL, err.max()


def test_fp32_assembly_hi_is_the_rounded_weight(dev):
    from paper_1603_04100_gb300 import api
    p = I.random_sphere(30000, 3)
    pt = torch.from_numpy(p).to(dev)
    op = api.assemble(pt, api.knn(pt, 20), prec=api.FP32_REFINE)
    hi = op.rows("val").astype(np.float64)
    lo = op.rows("val_lo").astype(np.float64)
    # a normalised pair: hi = fl32(hi + lo), |lo| <= half an FP32 ulp of hi
    np.testing.assert_array_equal((hi + lo).astype(np.float32).astype(np.float64), hi)
    assert np.all(np.abs(lo) <= 2.0 ** -24 * np.abs(hi) * (1 + 2.0 ** -20))


def test_fp32_assembly_batch_mixed_formats_equal_solo(dev):
    # one batched launch holding FP64 and FP32_REFINE clouds: each equal to its solo assembly
    from paper_1603_04100_gb300 import _lib as LB
    from paper_1603_04100_gb300 import api
    import ctypes as C
    clouds = [(I.random_sphere(5000, 60), 20, api.FP32_REFINE), (I.torus(3001, 61), 16, api.FP64),
              (np.concatenate([I.random_sphere(1500, 62), I.random_sphere(1500, 62)[:300]]), 12, api.FP32_REFINE)]
    L = LB.load()
    ops, solo = [], []
    items = (LB.AssembleItem * len(clouds))()
    keep = []
    for i, (p, k, prec) in enumerate(clouds):
        pt = torch.from_numpy(p).to(dev)
        nbr, order = api.knn(pt, k, want_order=True)
        solo.append(api.assemble(pt, nbr, prec=prec, order=order))
        col, val, lo = api.ell_alloc(len(p), k, prec, dev)
        op = api.Operator(len(p), k, prec, col, val, lo, order)
        ops.append(op)
        keep += [pt, nbr, order]
        items[i] = LB.AssembleItem(api._vp(pt), api._vp(nbr), op.cstruct(), C.c_void_p(0), C.c_void_p(0))
    ns = (C.c_int64 * len(clouds))(*[len(p) for p, _, _ in clouds])
    ws = torch.empty(L.mvgd_assemble_batch_workspace_bytes(ns, len(clouds)), dtype=torch.uint8, device=dev)
    rule = LB.DeltaRule(api.DELTA_MEAN_NN, 6, 1.0, 0, 0)
    LB.check("mvgd_assemble_batch", L.mvgd_assemble_batch(items, len(clouds), rule, None, api._vp(ws), ws.numel(),
                                                           api._stream()))
    torch.cuda.synchronize()
    def bits(a):  # bit patterns (rows with status 2 hold NaN)
        return a.view(np.int32) if a.dtype == np.float32 else a.view(np.int64)
    for a, b in zip(ops, solo):  # the rows themselves (the arrays end in alignment slack)
        np.testing.assert_array_equal(a.rows("col"), b.rows("col"))
        np.testing.assert_array_equal(bits(a.rows("val")), bits(b.rows("val")))
        if a.val_lo is not None:
            np.testing.assert_array_equal(bits(a.rows("val_lo")), bits(b.rows("val_lo")))
