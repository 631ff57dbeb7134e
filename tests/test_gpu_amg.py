"""GPU parity of the aggregation-multigrid hierarchy, its V-cycle and the
multigrid-preconditioned solves, against the FP64 oracle (oracle/amg.py).

The operators are built by the oracle (kNN + MVGD rows on Z-order-sorted
points) and uploaded as they are, so both sides aggregate the same rows.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import amg as OA
from paper_1603_04100_gb300 import inputs as I
from tests.gpu_util import cuda_or_skip, operator_from_rows
from tests.oracle_util import backward_ok, reference_solution, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _oracle_operator(n, k, seed, shape="sphere"):
    pts = I.random_sphere(n, seed) if shape == "sphere" else I.torus(n, seed)
    pts = I.morton_sorted(pts)
    nbr = oracle.knn_grid(pts, k)
    val, st, _, _ = oracle.assemble(pts, nbr)
    assert int(st.max()) == 0
    return pts, nbr, val


@pytest.mark.parametrize("n,k,prec_name", [(20000, 20, "FP64"), (7001, 12, "FP32_REFINE"),
                                           (3000, 24, "FP64"), (300, 16, "FP64")])
def test_hierarchy_matches_oracle(n, k, prec_name):
    dev = cuda_or_skip()
    from paper_1603_04100_gb300 import api
    prec = getattr(api, prec_name)
    _, nbr, val = _oracle_operator(n, k, 31, "torus" if k == 24 else "sphere")
    op = operator_from_rows(nbr, val, prec, dev)
    H = api.amg_setup(op, 1.0)
    torch.cuda.synchronize()
    levels = OA.hierarchy(val, nbr, 1.0)
    i0 = H.info(0)
    assert i0.status == 0, i0.status
    assert H.levels == len(levels)
    # level 0: the smoother's scaling (omega / a_ii on strong rows, else 1 / sum |a_ij|),
    # from FP64 sums rounded once to FP32
    (d0,) = H.level_rows(0)
    np.testing.assert_allclose(d0, levels[0].d, rtol=2 ** -23, atol=0)
    for lv in range(1, len(levels)):
        ref = levels[lv]
        cnt, col, v64, v32, dinv = H.level_rows(lv)
        want_cnt = np.bincount(ref.rows, minlength=ref.n)
        assert np.array_equal(cnt, want_cnt)                      # integer structure: exact
        starts = np.concatenate([[0], np.cumsum(want_cnt)])
        scale = np.zeros(ref.n)
        np.add.at(scale, ref.rows, np.abs(ref.vals))
        for r in range(ref.n):
            c = cnt[r]
            assert np.array_equal(col[r, :c], ref.cols[starts[r]:starts[r + 1]])
        got = np.concatenate([v64[r, :cnt[r]] for r in range(ref.n)])
        # the same FP64 sums in another order: within a few ulps of the row's magnitude
        tol = 64 * np.finfo(np.float64).eps * scale[ref.rows]
        assert np.all(np.abs(got - ref.vals) <= tol), float(np.max(np.abs(got - ref.vals) / scale[ref.rows]))
        np.testing.assert_array_equal(np.concatenate([v32[r, :cnt[r]] for r in range(ref.n)]),
                                      got.astype(np.float32))
        np.testing.assert_allclose(dinv, ref.d, rtol=2 ** -22, atol=0)
        # padding: (own row, 0) up to the stride
        r = int(np.argmin(cnt))
        assert np.all(col[r, cnt[r]:] == r) and np.all(v64[r, cnt[r]:] == 0.0)


@pytest.mark.parametrize("n", [20000, 300])
def test_coarsest_inverse(n):
    dev = cuda_or_skip()
    from paper_1603_04100_gb300 import api
    _, nbr, val = _oracle_operator(n, 20, 32)
    H = api.amg_setup(operator_from_rows(nbr, val, api.FP64, dev), 1.0)
    Ac = OA.hierarchy(val, nbr, 1.0)[-1].dense()
    nc = Ac.shape[0]
    want = np.linalg.inv(Ac)
    cond = np.linalg.cond(Ac)
    # FP32 Gauss-Jordan with partial pivoting: residual and forward error of order n u32 cond
    X32 = H.coarsest_inverse(fp64=False).astype(np.float64)
    u32, u64 = 2.0 ** -24, 2.0 ** -53
    assert np.abs(Ac @ X32 - np.eye(nc)).max() <= 4 * nc * u32 * cond
    assert np.linalg.norm(X32 - want) / np.linalg.norm(want) <= 4 * nc * u32 * cond
    # two Newton-Schulz steps in FP64 square that residual twice: down to the FP64 level
    X = H.coarsest_inverse()
    assert np.abs(Ac @ X - np.eye(nc)).max() <= 4 * nc * u64 * cond
    assert np.linalg.norm(X - want) / np.linalg.norm(want) <= 4 * nc * u64 * cond


@pytest.mark.parametrize("n,nrhs", [(20000, 1), (9000, 3), (300, 2)])
def test_vcycle_matches_oracle(n, nrhs):
    dev = cuda_or_skip()
    from paper_1603_04100_gb300 import api
    _, nbr, val = _oracle_operator(n, 20, 33)
    H = api.amg_setup(operator_from_rows(nbr, val, api.FP64, dev), 1.0)
    levels = OA.hierarchy(val, nbr, 1.0)
    b = np.random.default_rng(5).standard_normal((n, nrhs))
    x = H.apply(torch.from_numpy(b).to(dev)).cpu().numpy()
    for q in range(nrhs):
        want = OA.vcycle(levels, b[:, q])
        err = np.linalg.norm(x[:, q] - want) / np.linalg.norm(want)
        # an FP32 cycle of a fixed linear map: relative error a few hundred FP32 ulps
        assert err <= 2e-5, err


def _solve_case(n, k, seed):
    pts, nbr, val = _oracle_operator(n, k, seed)
    z = pts[:, 2]
    f = 13.0 * (5 * z ** 3 - 3 * z)
    return pts, nbr, val, f


@pytest.mark.parametrize("prec_name", ["FP64", "FP32_REFINE"])
def test_multigrid_preconditioned_solve(prec_name):
    dev = cuda_or_skip()
    from paper_1603_04100_gb300 import api
    prec = getattr(api, prec_name)
    n = 60000
    _, nbr, val, f = _solve_case(n, 20, 34)
    op = operator_from_rows(nbr, val, prec, dev)
    ft = torch.from_numpy(f).to(dev)
    # several times fewer Krylov iterations than the row-scaled solve
    plain = api.solve(op, ft, rtol=1e-9, precond=1)
    res9 = api.solve(op, ft, rtol=1e-9, precond=2)
    assert res9.status == [0], res9.status
    assert 4 * res9.iters[0] < plain.iters[0], (res9.iters, plain.iters)
    # parity: a tight solve against the oracle's (FP64 multigrid BiCGSTAB with refinement)
    res = api.solve(op, ft, rtol=1e-11, precond=2)
    assert res.status == [0] and res.relres[0] <= 1e-11, (res.status, res.relres)
    u = res.u.cpu().numpy()
    assert backward_ok(val, nbr, u, f, 1e-11)
    u_or, _, rel_or = OA.solve_refined(OA.hierarchy(val, nbr, 1.0), f, rtol=1e-11)
    assert rel_or <= 1e-11
    assert rel_l2(u, u_or) <= 1e-8, rel_l2(u, u_or)
    # the 1e-9 solve is within 1e-8 of the oracle too
    assert rel_l2(res9.u.cpu().numpy(), u_or) <= 1e-8, rel_l2(res9.u.cpu().numpy(), u_or)


def test_multigrid_solve_of_a_single_level_system_is_direct():
    # n <= 512: the hierarchy is the operator itself, inverted; the preconditioned
    # Krylov solve converges at once
    dev = cuda_or_skip()
    from paper_1603_04100_gb300 import api
    _, nbr, val, f = _solve_case(400, 16, 35)
    op = operator_from_rows(nbr, val, api.FP64, dev)
    res = api.solve(op, torch.from_numpy(f).to(dev), rtol=1e-10, precond=2)
    assert res.status == [0] and res.iters[0] <= 3, (res.status, res.iters)


def test_multigrid_batch_equals_solo():
    dev = cuda_or_skip()
    from paper_1603_04100_gb300 import api
    from paper_1603_04100_gb300.batch import BatchPipeline
    sizes = [(9000, 12, 2), (30000, 20, 1), (450, 16, 1)]
    clouds = [I.random_sphere(n, 40 + i) for i, (n, _, _) in enumerate(sizes)]
    fs = [np.stack([c[:, 0], c[:, 1] * c[:, 2]][:q], axis=1).copy() for c, (_, _, q) in zip(clouds, sizes)]
    pts = [torch.from_numpy(c).to(dev) for c in clouds]
    ft = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in fs]
    for prec in (api.FP32_REFINE, api.FP64):
        both = BatchPipeline(sizes, prec=prec, precond=2, device=dev)
        both.run(pts, ft)
        torch.cuda.synchronize()
        for i, sz in enumerate(sizes):
            solo = BatchPipeline([sz], prec=prec, precond=2, device=dev)
            solo.run([pts[i]], [ft[i]])
            torch.cuda.synchronize()
            assert torch.equal(solo.slots[0].u, both.slots[i].u), (prec, i)
            info = api.decode_info(both.slots[i].info)
            assert all(st == 0 and rel <= 1e-8 for _, _, rel, st in info), info


def test_multigrid_batch_matches_oracle():
    # every cloud of one batched launch (FP32 inner + FP64 refinement, multigrid)
    # against the oracle's own kNN, rows and tight solve of that cloud
    dev = cuda_or_skip()
    from paper_1603_04100_gb300 import api
    from paper_1603_04100_gb300.batch import BatchPipeline
    sizes = [(9000, 12, 2), (30000, 20, 1), (450, 16, 1), (20000, 16, 3)]
    clouds = [I.random_sphere(sizes[0][0], 40), I.ellipsoid(sizes[1][0], 41), I.random_sphere(sizes[2][0], 42),
              I.torus(sizes[3][0], 43)]
    fs = [np.stack([c[:, 0], c[:, 1] * c[:, 2], np.sin(c[:, 0]) * np.exp(c[:, 1])][:q], axis=1).copy()
          for c, (_, _, q) in zip(clouds, sizes)]
    bp = BatchPipeline(sizes, prec=api.FP32_REFINE, precond=2, device=dev, rtol=1e-11)
    bp.run([torch.from_numpy(c).to(dev) for c in clouds], [torch.from_numpy(x).to(dev) for x in fs])
    torch.cuda.synchronize()
    for i, (n, k, q) in enumerate(sizes):
        info = api.decode_info(bp.slots[i].info)
        assert all(st == 0 and rel <= 1e-11 for _, _, rel, st in info), (i, info)
        nbr = oracle.knn_grid(clouds[i], k)
        assert np.array_equal(bp.slots[i].nbr.cpu().numpy(), nbr)
        val, st, _, _ = oracle.assemble(clouds[i], nbr)
        assert int(st.max()) == 0
        u_or, _, rels = reference_solution(clouds[i], nbr, val, fs[i], rtol=1e-11)
        assert max(rels) <= 1e-11
        u = bp.slots[i].u.cpu().numpy()
        for c in range(q):
            assert rel_l2(u[:, c], u_or[:, c]) <= 1e-8, (i, c, rel_l2(u[:, c], u_or[:, c]))


def _zorder_keys(pts):
    """The exported row order's key: 21-bit Z-order of the bounding cube (FP64 (x - lo) * (2^21 / extent))."""
    lo = pts.min(axis=0)
    e = float((pts.max(axis=0) - lo).max())
    q = np.clip((pts - lo) * (2097152.0 / e), 0.0, 2097151.0).astype(np.uint64)
    key = np.zeros(pts.shape[0], dtype=np.uint64)
    for b in range(21):
        for a in range(3):
            key |= ((q[:, a] >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + a)
    return key


@pytest.mark.parametrize("n,seed", [(70001, 7), (4096, 8), (3, 9)])
def test_stored_order_is_the_zorder_of_the_points(n, seed):
    # the row order the kNN step exports: every point along one Z-order curve of
    # the bounding cube, ties by index -- an integer result, compared exactly
    dev = cuda_or_skip()
    from paper_1603_04100_gb300 import api
    pts = I.random_sphere(n, seed) if n > 3 else np.array([[0.0, 0, 0], [1, 1, 1], [0, 0, 0]])
    if n == 70001:
        pts[100:140] = pts[99]  # duplicated points: equal keys, ordered by index
    _, order = api.knn(torch.from_numpy(pts).to(dev), 2 if n == 3 else 12, want_order=True)
    key = _zorder_keys(pts)
    want = np.lexsort((np.arange(n), key))
    assert np.array_equal(order.cpu().numpy(), want)
