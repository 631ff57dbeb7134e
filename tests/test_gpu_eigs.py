"""Lowest LB eigenvalues (Sec. 4.3) from the GPU subspace iteration against the
oracle's sparse eigensolver on the same operator, and the block kernels it
is built on against plain products."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1603_04100_gb300 import inputs as I
from tests.gpu_util import cuda_or_skip

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,p,q,w", [(1000, 8, 8, 8), (4097, 24, 16, 8), (70001, 40, 40, 8), (33, 6, 3, 3),
                                     (5003, 128, 96, 8)])
def test_block_gram_and_combine(n, p, q, w):
    dev = cuda_or_skip()
    from paper_1603_04100_gb300 import _lib as LB
    from paper_1603_04100_gb300 import api
    L = LB.load()
    g = np.random.default_rng(n)
    Xd = g.standard_normal((n, p))
    Yd = g.standard_normal((n, q))

    def blocked(a):  # column c of a at (c / w) n w + r w + c % w
        c = a.shape[1]
        return torch.from_numpy(np.ascontiguousarray(a.reshape(n, c // w, w).transpose(1, 0, 2))).to(dev)

    X, Y = blocked(Xd), blocked(Yd)
    G = torch.empty((p, q), dtype=torch.float64, device=dev)
    ws = torch.empty(L.mvgd_block_gram_workspace_bytes(p, q), dtype=torch.uint8, device=dev)
    LB.check("gram", L.mvgd_block_gram(api._vp(X), p, api._vp(Y), q, n, w, api._vp(G), api._vp(ws), ws.numel(),
                                        None))
    want = Xd.T @ Yd
    scale = np.sqrt((Xd ** 2).sum(0))[:, None] * np.sqrt((Yd ** 2).sum(0))[None, :]
    assert np.all(np.abs(G.cpu().numpy() - want) <= 1e-13 * scale)
    # the same call twice gives the same bits (fixed reduction order)
    G2 = torch.empty_like(G)
    L.mvgd_block_gram(api._vp(X), p, api._vp(Y), q, n, w, api._vp(G2), api._vp(ws), ws.numel(), None)
    assert torch.equal(G, G2)
    Cm = g.standard_normal((p, q))
    Z = torch.empty((q // w, n, w), dtype=torch.float64, device=dev)
    LB.check("combine", L.mvgd_block_combine(api._vp(X), p, api._vp(torch.from_numpy(Cm).to(dev)), q, n, w,
                                              api._vp(Z), None))
    got = Z.cpu().numpy().transpose(1, 0, 2).reshape(n, q)
    want = Xd @ Cm
    assert np.all(np.abs(got - want) <= 1e-13 * (np.abs(Xd) @ np.abs(Cm)))


@pytest.mark.parametrize("prec_name", ["FP64", "FP32_REFINE"])
def test_lowest_eigenvalues_match_oracle(prec_name):
    dev = cuda_or_skip()
    from paper_1603_04100_gb300 import api
    from paper_1603_04100_gb300.eigs import lowest_eigenpairs
    p = I.random_sphere(4000, 1)
    pt = torch.from_numpy(p).to(dev)
    nbr_t, ord_t = api.knn(pt, 20, want_order=True)
    op = api.assemble(pt, nbr_t, prec=getattr(api, prec_name), order=ord_t)
    res = lowest_eigenpairs(op, 25)
    assert res.change <= 1e-8, (res.iterations, res.change)
    val, _, _, _ = oracle.assemble(p, nbr_t.cpu().numpy())
    want = oracle.lb_eigenvalues(val, nbr_t.cpu().numpy(), 25)
    assert np.all(np.abs(res.values - want) <= 1e-6 * np.maximum(want, 1.0)), np.abs(res.values - want).max()
    # the sphere's spectrum: 0, then 2 (x3), 6 (x5), 12 (x7), 20 (x9) to discretisation accuracy
    assert abs(res.values[0]) <= 1e-8
    e2, _ = oracle.multiplet_errors(res.values, 4)
    assert e2 <= 0.02


def test_lambda8_multiplet_matches_oracle():
    # the 81 lowest eigenvalues (through lambda_8 = 72, eigenvalues 64 .. 80): a basis of 96 vectors
    dev = cuda_or_skip()
    from paper_1603_04100_gb300 import api
    from paper_1603_04100_gb300.eigs import lowest_eigenpairs
    p = I.random_sphere(4000, 1)
    pt = torch.from_numpy(p).to(dev)
    nbr_t, ord_t = api.knn(pt, 20, want_order=True)
    op = api.assemble(pt, nbr_t, prec=api.FP64, order=ord_t)
    res = lowest_eigenpairs(op, 81, maxit=400)
    assert res.vectors.shape[0] * res.vectors.shape[2] == 96
    assert res.change <= 1e-8, (res.iterations, res.change)
    val, _, _, _ = oracle.assemble(p, nbr_t.cpu().numpy())
    want = oracle.lb_eigenvalues(val, nbr_t.cpu().numpy(), 81)
    assert np.all(np.abs(res.values - want) <= 1e-6 * np.maximum(want, 1.0)), np.abs(res.values - want).max()
    e2, einf = oracle.multiplet_errors(res.values, 8)
    assert e2 <= 0.05 and einf <= 0.08


def test_dirichlet_hemisphere_eigenvalues_match_oracle():
    dev = cuda_or_skip()
    from paper_1603_04100_gb300 import api
    from paper_1603_04100_gb300.eigs import lowest_eigenpairs
    p, b = I.hemisphere(4000, 3)
    pt = torch.from_numpy(p).to(dev)
    bt = torch.from_numpy(b).to(dev)
    nbr_t, ord_t = api.knn(pt, 20, want_order=True)
    op = api.assemble(pt, nbr_t, prec=api.FP64, order=ord_t)
    api.dirichlet_rows(op, bt)
    res = lowest_eigenpairs(op, 10, boundary=bt)
    assert res.change <= 1e-8, (res.iterations, res.change)
    nbr = nbr_t.cpu().numpy()
    val, _, _, _ = oracle.assemble(p, nbr)
    want = oracle.lb_eigenvalues(oracle.dirichlet_rows(val, b), nbr, 10, boundary=b)
    assert np.all(np.abs(res.values - want) <= 1e-6 * want), np.abs(res.values - want).max()
    # l (l + 1) with multiplicity l
    assert np.abs(res.values - np.array([2.0, 6, 6, 12, 12, 12, 20, 20, 20, 20])).max() <= 0.1


def _hemisphere_table(row: str) -> dict:
    """Sec. 4.3's hemisphere tables (tests/golden/hemisphere_eigen_errors_sec4_3.txt):
    E^inf (x 1e-2) by sample size for the row named."""
    from pathlib import Path
    rows = {}
    for line in (Path(__file__).parent / "golden" / "hemisphere_eigen_errors_sec4_3.txt").read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            name, *vals = line.split()
            rows[name] = [float(v) for v in vals]
    return dict(zip([int(v) for v in rows["samples"]], rows[row]))


def test_dirichlet_hemisphere_lambda182_on_the_device():
    # the table row lambda = 182 (l = 13, multiplicity 13) needs the 91 lowest
    # Dirichlet eigenvalues: a basis of 104 vectors
    dev = cuda_or_skip()
    from paper_1603_04100_gb300 import api
    from paper_1603_04100_gb300.eigs import lowest_eigenpairs
    n = 4000
    p, b = I.hemisphere(n, 3)
    pt, bt = torch.from_numpy(p).to(dev), torch.from_numpy(b).to(dev)
    nbr_t, ord_t = api.knn(pt, 20, want_order=True)
    op = api.assemble(pt, nbr_t, prec=api.FP64, order=ord_t)
    api.dirichlet_rows(op, bt)
    res = lowest_eigenpairs(op, 91, boundary=bt, maxit=600)
    assert res.change <= 1e-8, (res.iterations, res.change)
    nbr = nbr_t.cpu().numpy()
    val, _, _, _ = oracle.assemble(p, nbr)
    want = oracle.lb_eigenvalues(oracle.dirichlet_rows(val, b), nbr, 91, boundary=b)
    assert np.all(np.abs(res.values - want) <= 1e-6 * want), np.abs(res.values - want).max()
    mult = res.values[78:91]                       # l = 13: eigenvalues 78 .. 90
    einf = np.abs(mult - 182.0).max() / 182.0
    printed = _hemisphere_table("dirichlet_Einf_182")[n] * 1e-2
    # the paper's samples are not ours (its hemisphere sampling is not stated): same order
    assert 0.3 * printed <= einf <= 6.0 * printed, (einf, printed)
