"""Neumann boundary by reflection (Sec. 3.1) on the GPU against the oracle:
the ghosts, the folded operator, the condition's right-hand-side term, solves
and the hemisphere's Neumann spectrum (Sec. 4.3: l (l + 1), multiplicity l + 1).

The oracle runs its own pipeline on the seeded clouds throughout.  Stage tests
feed the GPU stage the oracle's input of that stage (the cloud of interior
points and ghosts the oracle built); end-to-end tests run the two pipelines
side by side from the same points."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1603_04100_gb300 import inputs as I
from tests.gpu_util import cuda_or_skip, row_relerr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _half_disk(n, nb, seed):
    g = np.random.default_rng(seed)
    r = np.sqrt(g.uniform(size=n - nb))
    t = g.uniform(0.0, np.pi, size=n - nb)
    inner = np.stack([r * np.cos(t), r * np.sin(t), np.zeros(n - nb)], axis=1)
    rim = np.stack([np.linspace(-1.0, 1.0, nb), np.zeros(nb), np.zeros(nb)], axis=1)
    b = np.zeros(n, dtype=np.uint8)
    b[:nb] = 1
    q, rr = np.linalg.qr(g.standard_normal((3, 3)))
    return np.ascontiguousarray(np.concatenate([rim, inner]) @ (q * np.sign(np.diag(rr))).T), b


def _cloud(name, n):
    return I.hemisphere(n, 3) if name == "hemisphere" else _half_disk(n, 60, 1)


def _oracle(p, b, k):
    """The oracle's pipeline: ghosts, cloud, kNN and rows over it, fold."""
    nbr = oracle.knn_grid(p, k)
    g = oracle.neumann_ghosts(p, b, nbr, kb=6)
    q, q_src = g.cloud(p)
    nq = oracle.knn_grid(q, k)
    vq, st, _, _ = oracle.assemble(q, nq)
    assert int(st[:g.interior.size].max()) == 0
    val, col = oracle.neumann_fold(vq, nq, g.interior.size, q_src)
    return nbr, g, q, q_src, nq, vq, val, col


@pytest.mark.parametrize("name,n,k", [("hemisphere", 4000, 20), ("hemisphere", 1500, 12), ("half_disk", 3000, 16)])
def test_ghosts_match_oracle(name, n, k):
    dev = cuda_or_skip()
    from paper_1603_04100_gb300 import api
    p, b = _cloud(name, n)
    nbr_o = oracle.knn_grid(p, k)
    g = oracle.neumann_ghosts(p, b, nbr_o, kb=6)
    pt, bt = torch.from_numpy(p).to(dev), torch.from_numpy(b).to(dev)
    nbr_t = api.knn(pt, k)
    assert np.array_equal(nbr_t.cpu().numpy(), nbr_o)
    c = api.neumann_ghosts(pt, nbr_t, bt, kb=6)
    assert (c.n_interior, c.n_ghost, c.n_boundary, c.bad_frames) == (g.interior.size, g.src.size, int(b.sum()), 0)
    assert np.array_equal(c.interior.cpu().numpy(), g.interior)
    q_src = c.q_src.cpu().numpy()
    assert np.array_equal(q_src[:c.n_interior], np.arange(c.n_interior))
    assert np.array_equal(q_src[c.n_interior:], g.src)
    assert np.array_equal(c.ghost_bnd.cpu().numpy(), g.bnd)
    q = c.q.cpu().numpy()
    assert np.array_equal(q[:c.n_interior], p[g.interior])
    assert np.abs(q[c.n_interior:] - g.pts).max() <= 1e-11
    assert np.abs(c.ghost_dist.cpu().numpy() - g.dist).max() <= 1e-11


def _gpu_over_oracle_cloud(dev, q, q_src, g, k, prec):
    """The GPU's kNN, rows and fold over the oracle's cloud of interior points and ghosts."""
    from paper_1603_04100_gb300 import api
    qt = torch.from_numpy(q).to(dev)
    nq_t, oq_t = api.knn(qt, k, want_order=True)
    op_q = api.assemble(qt, nq_t, prec=prec, order=oq_t)
    cloud = api.NeumannCloud(q=qt, q_src=torch.from_numpy(q_src.astype(np.int32)).to(dev),
                             interior=torch.from_numpy(g.interior.astype(np.int32)).to(dev),
                             ghost_bnd=torch.from_numpy(g.bnd.astype(np.int32)).to(dev),
                             ghost_dist=torch.from_numpy(g.dist).to(dev), n_interior=g.interior.size,
                             n_ghost=g.src.size, n_boundary=0, bad_frames=0, op_q=op_q)
    return api.neumann_fold(op_q, cloud), cloud, nq_t.cpu().numpy(), oq_t.cpu().numpy()


@pytest.mark.parametrize("prec_name", ["FP64", "FP32_REFINE"])
def test_fold_matches_oracle(prec_name):
    dev = cuda_or_skip()
    from paper_1603_04100_gb300 import api
    p, b = I.hemisphere(3000, 4)
    _, g, q, q_src, nq, _, val, col = _oracle(p, b, 20)
    op, cloud, nq_g, oq = _gpu_over_oracle_cloud(dev, q, q_src, g, 20, getattr(api, prec_name))
    assert np.array_equal(nq_g, nq)
    order = op.order.cpu().numpy()
    # stored order: the interior subsequence of the cloud's stored order
    assert np.array_equal(order, oq[oq < cloud.n_interior])
    got_col = order[op.rows("col")]           # stored columns -> interior positions
    assert np.array_equal(got_col, col[order])
    assert np.any(got_col == order[:, None])  # some rows see their own ghost
    err = row_relerr(op.weights(), val[order])
    assert err.max() <= 1e-10, err.max()


def test_condition_term_matches_oracle():
    # dU/dn = g with g = the rim points' x coordinate (any function read at the boundary)
    dev = cuda_or_skip()
    from paper_1603_04100_gb300 import api
    p, b = I.hemisphere(3000, 4)
    _, g, q, q_src, nq, vq, _, _ = _oracle(p, b, 20)
    gv = np.where(b == 1, p[:, 0], np.nan)    # never read off the boundary
    want = oracle.neumann_rhs(vq, nq, g.interior.size, g, gv)
    for prec in (api.FP64, api.FP32_REFINE):
        _, cloud, _, _ = _gpu_over_oracle_cloud(dev, q, q_src, g, 20, prec)
        got = api.neumann_rhs(cloud, torch.from_numpy(gv).to(dev)).cpu().numpy()
        assert np.all(np.isfinite(got))
        scale = np.abs(vq[:g.interior.size, 1:]).sum(1) * np.nanmax(np.abs(gv)) * max(g.dist.max(), 1e-300)
        assert np.all(np.abs(got - want) <= 1e-12 * scale), np.abs(got - want).max()
    assert np.count_nonzero(want) > 0


def _sparse_solve(val, col, f):
    import scipy.sparse.linalg as spl
    A = oracle.system_matrix(val, col, 1.0)
    u = spl.spsolve(A.tocsc(), f)
    assert np.linalg.norm(f - A @ u) <= 1e-11 * np.linalg.norm(f)
    return u


@pytest.mark.parametrize("prec_name,precond", [("FP64", 1), ("FP32_REFINE", 2)])
def test_neumann_solve_end_to_end(prec_name, precond):
    # u = x is even in z, so dU/dn = 0 on the rim; -Delta x = 2 x: (I - L) u = 3 x
    dev = cuda_or_skip()
    from paper_1603_04100_gb300 import api
    p, b = I.hemisphere(16000, 3)
    _, g, _, _, _, _, val, col = _oracle(p, b, 20)
    op, cloud = api.neumann_operator(torch.from_numpy(p).to(dev), torch.from_numpy(b).to(dev), 20,
                                     prec=getattr(api, prec_name))
    assert np.array_equal(cloud.interior.cpu().numpy(), g.interior)
    x = p[g.interior, 0]
    res = api.solve(op, torch.from_numpy(3.0 * x).to(dev), rtol=1e-11, precond=precond)
    assert res.status == [0], res.status
    u = res.u.cpu().numpy()
    u_or = _sparse_solve(val, col, 3.0 * x)
    assert np.linalg.norm(u - u_or) / np.linalg.norm(u_or) <= 1e-8
    assert abs(np.abs(u - x).max() - np.abs(u_or - x).max()) <= 1e-6
    assert np.abs(u - x).max() <= 2e-2


def test_inhomogeneous_solve_end_to_end():
    # u = z: on the rim the outward normal in the tangent plane is -z, so dU/dn = -1;
    # -Delta z = 2 z: (I - L) u = 3 z + c
    dev = cuda_or_skip()
    from paper_1603_04100_gb300 import api
    errs = []
    for n in (4000, 16000):
        p, b = I.hemisphere(n, 3)
        _, g, q, q_src, nq, vq, val, col = _oracle(p, b, 20)
        gv = np.full(n, -1.0)
        z = p[g.interior, 2]
        u_or = _sparse_solve(val, col, 3.0 * z + oracle.neumann_rhs(vq, nq, g.interior.size, g, gv))
        op, cloud = api.neumann_operator(torch.from_numpy(p).to(dev), torch.from_numpy(b).to(dev), 20,
                                         prec=api.FP32_REFINE)
        c = api.neumann_rhs(cloud, torch.from_numpy(gv).to(dev))
        res = api.solve(op, torch.from_numpy(3.0 * z).to(dev) + c, rtol=1e-11, precond=2)
        assert res.status == [0], res.status
        u = res.u.cpu().numpy()
        assert np.linalg.norm(u - u_or) / np.linalg.norm(u_or) <= 1e-8
        errs.append(np.abs(u - z).max())
    # the condition's term makes u = z the discrete solution's limit: the error falls
    assert errs[0] < 0.05 and errs[1] < errs[0] / 2, errs


def test_neumann_hemisphere_eigenvalues_end_to_end():
    dev = cuda_or_skip()
    from paper_1603_04100_gb300 import api
    from paper_1603_04100_gb300.eigs import lowest_eigenpairs
    p, b = I.hemisphere(4000, 3)
    _, _, _, _, _, _, val, col = _oracle(p, b, 20)
    op, _ = api.neumann_operator(torch.from_numpy(p).to(dev), torch.from_numpy(b).to(dev), 20, prec=api.FP64)
    res = lowest_eigenpairs(op, 15)
    assert res.change <= 1e-8, (res.iterations, res.change)
    want = oracle.lb_eigenvalues(val, col, 15)
    assert np.all(np.abs(res.values - want) <= 1e-6 * np.maximum(want, 1.0)), np.abs(res.values - want).max()
    exact = np.array([0.0, 2, 2, 6, 6, 6, 12, 12, 12, 12, 20, 20, 20, 20, 20])
    assert np.abs(res.values - exact).max() <= 0.1


def test_neumann_hemisphere_lambda182_on_the_device():
    # the table row lambda = 182 (l = 13, multiplicity 14) needs the 105 lowest
    # Neumann eigenvalues: a basis of 120 vectors
    dev = cuda_or_skip()
    from paper_1603_04100_gb300 import api
    from paper_1603_04100_gb300.eigs import lowest_eigenpairs
    from tests.test_gpu_eigs import _hemisphere_table
    n = 4000
    p, b = I.hemisphere(n, 3)
    _, _, _, _, _, _, val, col = _oracle(p, b, 20)
    op, _ = api.neumann_operator(torch.from_numpy(p).to(dev), torch.from_numpy(b).to(dev), 20, prec=api.FP64)
    res = lowest_eigenpairs(op, 105, maxit=600)
    assert res.change <= 1e-8, (res.iterations, res.change)
    want = oracle.lb_eigenvalues(val, col, 105)
    assert np.all(np.abs(res.values - want) <= 1e-6 * np.maximum(want, 1.0)), np.abs(res.values - want).max()
    mult = res.values[91:105]                      # l = 13: eigenvalues 91 .. 104
    einf = np.abs(mult - 182.0).max() / 182.0
    printed = _hemisphere_table("neumann_Einf_182")[n] * 1e-2
    assert 0.3 * printed <= einf <= 6.0 * printed, (einf, printed)
