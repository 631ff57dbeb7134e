"""Pins of the FP64 aggregation-multigrid oracle (oracle/amg.py).

Each expected value is fixed outside the code under test: a dense product
built from explicit matrices, the textbook two-grid error-propagation
operator, exactness when the coarse space is the whole space, linearity, and
the plain (unpreconditioned) solver's solution.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import amg
from paper_1603_04100_gb300 import inputs as I


def _operator(n, k, seed, morton=True):
    pts = I.random_sphere(n, seed)
    if morton:
        pts = I.morton_sorted(pts)
    nbr = oracle.knn_grid(pts, k)
    val, st, _, _ = oracle.assemble(pts, nbr)
    assert int(st.max()) == 0
    return pts, nbr, val


def _dense_P(n, agg):
    nc = (n + agg - 1) // agg
    P = np.zeros((n, nc))
    P[np.arange(n), np.arange(n) // agg] = 1.0
    return P


@pytest.mark.parametrize("agg", [2, 8])
def test_galerkin_equals_dense_triple_product(agg):
    _, nbr, val = _operator(301, 12, 11)  # 301: the last aggregate is ragged
    A = amg.fine_level(val, nbr, 1.0)
    # the fine level itself is sigma I - L as a dense matrix
    Ld = oracle.to_csr(val, nbr).toarray()
    np.testing.assert_allclose(A.dense(), np.eye(301) - Ld, rtol=0, atol=1e-12 * np.abs(Ld).max())
    Ac = amg.galerkin(A, agg)
    P = _dense_P(301, agg)
    want = P.T @ A.dense() @ P
    assert Ac.n == P.shape[1]
    np.testing.assert_allclose(Ac.dense(), want, rtol=0, atol=1e-12 * np.abs(want).max())


def test_smoother_scaling_by_hand():
    # a 3x3 matrix written out: row 0 diagonally strong (4 > 0.3 * 6), row 1 weak
    # (0.5 < 0.3 * 3.5), row 2 with a negative diagonal
    A = amg.Level(3, [0, 0, 0, 1, 1, 1, 2, 2], [0, 1, 2, 0, 1, 2, 1, 2], [4, -1, -1, 2, 0.5, -1, 3, -2])
    assert amg.THETA == 0.3 and amg.OMEGA == 0.9
    np.testing.assert_array_equal(A.diag, [4.0, 0.5, -2.0])
    np.testing.assert_array_equal(A.l1, [6.0, 3.5, 5.0])
    np.testing.assert_allclose(A.d, [0.9 / 4.0, 1.0 / 3.5, 1.0 / 5.0], rtol=1e-15)


def test_coarse_row_sums_are_aggregated_fine_row_sums():
    _, nbr, val = _operator(2000, 16, 12)
    levels = amg.hierarchy(val, nbr, 1.0, coarsest=40)
    for fine, coarse in zip(levels[:-1], levels[1:]):
        rs_f = fine.matvec(np.ones(fine.n))
        rs_c = coarse.matvec(np.ones(coarse.n))
        want = np.zeros(coarse.n)
        np.add.at(want, np.arange(fine.n) // amg.AGG, rs_f)
        scale = np.abs(fine.vals).sum()
        np.testing.assert_allclose(rs_c, want, rtol=0, atol=1e-12 * scale / coarse.n)
    assert levels[-1].n <= 40 < levels[-2].n


def test_vcycle_is_exact_when_the_coarse_space_is_everything():
    # agg = 1: P = I and the coarse level is A itself, solved exactly, so the
    # cycle returns A^-1 b whatever the smoother does
    _, nbr, val = _operator(200, 12, 13)
    A = amg.fine_level(val, nbr, 1.0)
    levels = [A, amg.galerkin(A, 1)]
    b = np.random.default_rng(0).standard_normal(200)
    x = amg.vcycle(levels, b, agg=1)
    want = np.linalg.solve(A.dense(), b)
    np.testing.assert_allclose(x, want, rtol=0, atol=1e-10 * np.abs(want).max())


def test_two_grid_error_propagation_operator():
    # one V(1,1)-cycle M on two levels with an exact coarse solve has
    # I - M A = (I - D^-1 A)(I - P Ac^-1 P^T A)(I - D^-1 A)
    n, agg = 240, 8
    _, nbr, val = _operator(n, 12, 14)
    A = amg.fine_level(val, nbr, 1.0)
    levels = [A, amg.galerkin(A, agg)]
    Ad = A.dense()
    P = _dense_P(n, agg)
    Ac = P.T @ Ad @ P
    # the smoother's D from the dense matrix: omega / a_ii on diagonally strong rows, l1 elsewhere
    l1, dg = np.abs(Ad).sum(axis=1), np.diag(Ad)
    strong = dg > amg.THETA * l1
    assert strong.any() and not strong.all()  # both branches of the choice occur here
    Dinv = np.diag(np.where(strong, amg.OMEGA / np.where(strong, dg, 1.0), 1.0 / l1))
    S = np.eye(n) - Dinv @ Ad
    E = S @ (np.eye(n) - P @ np.linalg.solve(Ac, P.T @ Ad)) @ S
    M = np.stack([amg.vcycle(levels, e, agg) for e in np.eye(n)], axis=1)
    np.testing.assert_allclose(np.eye(n) - M @ Ad, E, rtol=0, atol=1e-9)


def test_vcycle_is_linear():
    _, nbr, val = _operator(3000, 20, 15)
    levels = amg.hierarchy(val, nbr, 1.0, coarsest=64)
    assert len(levels) >= 3
    g = np.random.default_rng(1)
    x, y = g.standard_normal(3000), g.standard_normal(3000)
    lhs = amg.vcycle(levels, 2.5 * x - 0.75 * y)
    rhs = 2.5 * amg.vcycle(levels, x) - 0.75 * amg.vcycle(levels, y)
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-11 * np.abs(rhs).max())


def test_preconditioned_solve_matches_plain_solve_in_fewer_iterations():
    pts, nbr, val = _operator(16384, 20, 16)
    z = pts[:, 2]
    f = 13.0 * (5 * z ** 3 - 3 * z)
    u_plain, it_plain, rel_plain, st = oracle.bicgstab(val, nbr, f, 1.0, rtol=1e-12)
    assert st == 0 and rel_plain <= 1e-12
    levels = amg.hierarchy(val, nbr, 1.0)
    assert [lv.n for lv in levels] == [16384, 2048, 256]
    u, its, rel = amg.bicgstab_right(levels, f, rtol=1e-10)
    assert rel <= 1e-10
    np.testing.assert_allclose(u, u_plain, rtol=0, atol=1e-8 * np.abs(u_plain).max())
    # the point of the preconditioner: far fewer iterations than the plain solve
    assert its * 4 < it_plain, (its, it_plain)
