"""Power iteration on the Gauss-Seidel iteration matrix (Sec. 4.1) through
mvgd_gs_power against the oracle's power iteration on the same stored-order
system, step by step: the sequence of norms and the last iterate."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1603_04100_gb300 import inputs as I
from tests.gpu_util import cuda_or_skip

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _case(dev, n, k, prec_name, variant, reorder=True, seed=7):
    from paper_1603_04100_gb300 import api
    p = I.random_sphere(n, seed)
    pt = torch.from_numpy(p).to(dev)
    nbr_t, ord_t = api.knn(pt, k, want_order=True)
    op = api.assemble(pt, nbr_t, prec=getattr(api, prec_name), order=ord_t if reorder else None,
                      variant=variant)
    ovar = oracle.VARIANT_LS if variant == api.ROW_LS else oracle.VARIANT_MVGD
    val, _, _, _ = oracle.assemble(p, nbr_t.cpu().numpy(), variant=ovar)
    order = ord_t.cpu().numpy() if reorder else None
    return op, oracle.system_matrix(val, nbr_t.cpu().numpy(), 1.0, order)


@pytest.mark.parametrize("n,k,prec_name,ls,reorder",
                         [(3000, 20, "FP64", False, True), (3000, 20, "FP64", True, True),
                          (2017, 12, "FP32_REFINE", False, True), (1000, 16, "FP64", False, False),
                          (33, 6, "FP64", False, True)])
def test_power_sequence_matches_oracle(n, k, prec_name, ls, reorder):
    dev = cuda_or_skip()
    from paper_1603_04100_gb300 import api
    op, A = _case(dev, n, k, prec_name, api.ROW_LS if ls else api.ROW_MVGD, reorder)
    x0 = np.random.default_rng(n).standard_normal(n)
    iters = 60
    got = api.gs_power(op, torch.from_numpy(x0).to(dev), iters, sigma=1.0)
    assert got.status == 0
    nu, x = oracle.gs_power(A, x0, iters)
    # FP32 hi + lo weights equal the FP64 ones to ~2^-48 relative
    tol = 1e-10 if prec_name == "FP64" else 1e-9
    assert np.all(np.abs(got.nu - nu) <= tol * nu), np.abs(got.nu / nu - 1).max()
    xg = got.x.cpu().numpy()
    assert np.abs(xg - x).max() <= 10 * tol * np.abs(x).max()
    # the same call again gives the same bits
    again = api.gs_power(op, torch.from_numpy(x0).to(dev), iters, sigma=1.0)
    assert np.array_equal(again.nu, got.nu) and torch.equal(again.x, got.x)


def test_mvgd_converges_least_squares_does_not():
    # Sec. 4.1: the MVGD system's Gauss-Seidel iteration matrix has its spectrum in
    # the unit circle; the least-squares rows put eigenvalues far outside it
    dev = cuda_or_skip()
    from paper_1603_04100_gb300 import api
    rho = {}
    for variant in (api.ROW_MVGD, api.ROW_LS):
        op, A = _case(dev, 1000, 20, "FP64", variant, seed=5)
        x0 = np.random.default_rng(0).standard_normal(1000)
        got = api.gs_power(op, torch.from_numpy(x0).to(dev), 400)
        dense = float(np.abs(oracle.gs_eigenvalues(A)).max())
        assert abs(got.rho - dense) <= 1e-3 * dense, (variant, got.rho, dense)
        rho[variant] = got.rho
    assert rho[api.ROW_MVGD] < 1.0 < 5.0 < rho[api.ROW_LS], rho


def test_zero_start_reports_nonfinite():
    dev = cuda_or_skip()
    from paper_1603_04100_gb300 import api, _lib as LB
    op, _ = _case(dev, 500, 12, "FP64", api.ROW_MVGD)
    got = api.gs_power(op, torch.zeros(500, dtype=torch.float64, device=dev), 3)
    assert got.status == LB.ENONFINITE
