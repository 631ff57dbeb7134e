"""Pins of the oracle's Gauss-Seidel spectra (Sec. 4.1): the iteration matrix
M^-1 N of A = M + N, N the strictly upper triangle of A.

* a 2 x 2 matrix by hand: M^-1 N = [[0, b/a], [0, -bc/(ad)]];
* the 1-D Dirichlet Laplacian tridiag(-1, 2, -1) of order n: the nonzero
  eigenvalues are the squares cos^2(k pi / (n + 1)) of the Jacobi eigenvalues
  (a consistently ordered matrix), so the spectral radius is cos^2(pi / (n + 1));
* the stored-order system matrix against the oracle's own C product;
* the paper's finding on a sphere: every eigenvalue inside the unit circle for
  the MVGD rows, some far outside for the least-squares rows.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

import oracle
from paper_1603_04100_gb300 import inputs as I


def _tridiag(n):
    return sp.diags([-np.ones(n - 1), 2.0 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1], format="csr")


def test_two_by_two_by_hand():
    a, b, c, d = 2.0, -0.7, 0.3, 1.5
    A = np.array([[a, b], [c, d]])
    lam = oracle.gs_eigenvalues(A)
    want = -b * c / (a * d)
    assert sorted(np.abs(lam)) == sorted([0.0, abs(want)]) or np.allclose(sorted(lam.real), sorted([0.0, want]),
                                                                          atol=1e-16)
    assert np.isclose(lam.real[np.argmax(np.abs(lam))], want, rtol=1e-15, atol=0)
    nu, x = oracle.gs_power(A, np.array([0.6, -1.1]), 5)
    # after one step the iterate is the eigenvector of -bc/(ad); the norm ratio is then exact
    assert np.all(np.abs(nu[1:] - abs(want)) <= 4e-16 * abs(want))


def test_tridiagonal_spectrum_is_jacobi_squared():
    n = 12
    lam = oracle.gs_eigenvalues(_tridiag(n))
    top = np.sort(np.abs(lam))[::-1][: n // 2]
    want = np.sort(np.cos(np.arange(1, n // 2 + 1) * np.pi / (n + 1)) ** 2)[::-1]
    # the smallest nonzero one sits nearest the defective zero eigenvalue, whose
    # perturbation it shares: a looser bound there
    assert np.all(np.abs(top[:-1] - want[:-1]) <= 1e-12) and abs(top[-1] - want[-1]) <= 1e-9, (top, want)
    # the rest are zero: one defective eigenvalue, which rounding moves by about
    # eps^(1/m) for a Jordan block of size m (here m = n / 2 - 1)
    assert np.all(np.abs(np.sort(np.abs(lam))[: n // 2]) <= 2e-3)


def test_power_iteration_reaches_the_spectral_radius():
    n = 10
    nu, x = oracle.gs_power(_tridiag(n), np.random.default_rng(3).standard_normal(n), 300)
    rho = np.cos(np.pi / (n + 1)) ** 2
    assert abs(nu[-1] - rho) <= 1e-12
    # x is the dominant eigenvector: M^-1 N x = -rho x (the sweep x <- -M^-1 N x + M^-1 b
    # has the iteration matrix -M^-1 N, whose eigenvalues are the positive cos^2)
    A = _tridiag(n).toarray()
    Tx = np.linalg.solve(np.tril(A), np.triu(A, 1) @ x)
    assert np.abs(Tx + rho * x).max() <= 1e-10


def test_system_matrix_in_stored_order():
    p = I.random_sphere(900, 4)
    nbr = oracle.knn_grid(p, 12)
    val, _, _, _ = oracle.assemble(p, nbr)
    order = np.random.default_rng(5).permutation(900)
    A = oracle.system_matrix(val, nbr, 1.0, order)
    x = np.random.default_rng(6).standard_normal(900)
    want = oracle.spmv(val, nbr, x, sigma=1.0)[order]
    got = A @ x[order]
    scale = np.abs(val).sum(1)[order] * np.abs(x).max()
    assert np.all(np.abs(got - want) <= 1e-13 * scale)


def test_mvgd_inside_unit_circle_least_squares_outside():
    p = I.random_sphere(1000, 5)
    nbr = oracle.knn_grid(p, 20)
    rho = {}
    for variant in (oracle.VARIANT_MVGD, oracle.VARIANT_LS):
        val, st, _, _ = oracle.assemble(p, nbr, variant=variant)
        assert int(st.max()) == 0
        A = oracle.system_matrix(val, nbr, 1.0)
        lam = oracle.gs_eigenvalues(A)
        rho[variant] = float(np.abs(lam).max())
        nu, _ = oracle.gs_power(A, np.random.default_rng(0).standard_normal(1000), 400)
        # the geometric mean of the norm ratios settles on the spectral radius, also
        # when a complex pair is on top
        est = float(np.exp(np.mean(np.log(nu[200:]))))
        assert abs(est - rho[variant]) <= 1e-3 * rho[variant], (variant, est, rho[variant])
    assert rho[oracle.VARIANT_MVGD] < 1.0 < 5.0 < rho[oracle.VARIANT_LS], rho


def test_least_squares_system_is_indefinite_mvgd_is_not():
    # Sec. 4.1's conditioning contrast, on the system the solver sees, A = I - L:
    # on the Fibonacci sphere (2,562 points, K = 12) the MVGD rows give eigenvalues
    # of positive real part near the origin (the smallest is 1, the constants),
    # the least-squares rows eigenvalues of negative real part too -- an indefinite,
    # nonnormal system on which restarted GMRES stagnates and BiCGSTAB diverges
    import scipy.sparse.linalg as spl
    pts = I.fibonacci_sphere(2562)
    nbr = oracle.knn_grid(pts, 12)
    for variant, indefinite in ((oracle.VARIANT_MVGD, False), (oracle.VARIANT_LS, True)):
        val, st, _, _ = oracle.assemble(pts, nbr, variant=variant)
        A = oracle.system_matrix(val, nbr, 1.0).tocsc()
        ev = spl.eigs(A, k=6, sigma=0.0, which="LM", return_eigenvectors=False)
        assert (ev.real.min() < 0.0) == indefinite, (variant, np.sort_complex(ev))
        if not indefinite:
            assert abs(ev.real.min() - 1.0) < 1e-8   # the constant vector: (I - L) 1 = 1
    # the oracle's GMRES(30) on the least-squares system: the residual stalls far above 1e-8
    val, _, _, _ = oracle.assemble(pts, nbr, variant=oracle.VARIANT_LS)
    _, it, rel, status = oracle.gmres(val, nbr, 3.0 * pts[:, 0], rtol=1e-8, maxit=3000, restart=30)
    assert status != 0 and 1e-6 < rel < 1e-2, (it, rel)
