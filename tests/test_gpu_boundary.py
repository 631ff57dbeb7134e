"""Open surfaces with Dirichlet rows (Sec. 3.1) on the GPU against the FP64 oracle.

The cloud is the open upper hemisphere with a rim band of boundary points; the
problem is u = z, (I - L) u = 3z inside and u = z on the band.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1603_04100_gb300 import inputs as I
from tests.gpu_util import cuda_or_skip, row_relerr
from tests.oracle_util import backward_ok, reference_solution, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _problem(n, seed=3):
    p, b = I.hemisphere(n, seed)
    z = p[:, 2]
    f = np.where(b == 1, z, 3.0 * z)
    return p, b, z, f


@pytest.mark.parametrize("order", [False, True])
def test_dirichlet_rows_match_oracle(order):
    dev = cuda_or_skip()
    from paper_1603_04100_gb300 import api
    p, b, _, _ = _problem(12001)
    pt = torch.from_numpy(p).to(dev)
    nbr_t, ord_t = api.knn(pt, 20, want_order=True)
    op = api.assemble(pt, nbr_t, prec=api.FP64, order=ord_t if order else None)
    assert api.dirichlet_rows(op, torch.from_numpy(b).to(dev)) == int(b.sum())
    nbr = nbr_t.cpu().numpy()
    val, _, _, _ = oracle.assemble(p, nbr)
    want = oracle.dirichlet_rows(val, b)
    got = op.weights()  # rows in stored order
    rows = op.order.cpu().numpy() if order else np.arange(len(p))
    bd = b[rows] == 1
    assert np.all(got[bd] == 0.0)  # boundary rows: exactly zero
    err = row_relerr(got[~bd], want[rows][~bd])
    assert err.max() <= 1e-10, err.max()


@pytest.mark.parametrize("prec_name,precond", [("FP64", 1), ("FP32_REFINE", 2), ("FP64", 2)])
def test_dirichlet_solve_matches_oracle(prec_name, precond):
    dev = cuda_or_skip()
    from paper_1603_04100_gb300 import api
    prec = getattr(api, prec_name)
    p, b, z, f = _problem(16000)
    pt = torch.from_numpy(p).to(dev)
    nbr_t, ord_t = api.knn(pt, 20, want_order=True)
    op = api.assemble(pt, nbr_t, prec=prec, order=ord_t)
    api.dirichlet_rows(op, torch.from_numpy(b).to(dev))
    res = api.solve(op, torch.from_numpy(f).to(dev), rtol=1e-11, precond=precond)
    assert res.status == [0], res.status
    u = res.u.cpu().numpy()
    nbr = nbr_t.cpu().numpy()
    val, _, _, _ = oracle.assemble(p, nbr)
    v = oracle.dirichlet_rows(val, b)
    u_or, _, rels = reference_solution(p, nbr, v, f, rtol=1e-11)
    assert rels[0] <= 1e-11
    # backward error with the oracle's operator, forward error against its solution
    assert backward_ok(v, nbr, u, f, 1e-11)
    assert rel_l2(u, u_or) <= 1e-8, rel_l2(u, u_or)
    # the discretisation error against u = z is the oracle's (second order, Sec. 3.1)
    assert abs(np.abs(u - z).max() - np.abs(u_or - z).max()) <= 1e-3 * np.abs(u_or - z).max()
    # the boundary rows read u_i = z_i, to the solve's residual
    assert np.abs(u[b == 1] - z[b == 1]).max() <= 1e-9
