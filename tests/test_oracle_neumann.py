"""Pins of the oracle's Neumann reflection (Sec. 3.1) and of the open-surface
spectra of Sec. 4.3.

* A planar half-disk, moved by a rigid motion: the boundary is a straight line
  in a plane, so the frame is exact and every ghost is the mirror image of its
  point through that line, to rounding.
* The upper hemisphere: the reflection through the rim plane z = 0 maps
  (x, y, z) to (x, y, -z); the estimated frames reach it as the sampling gets
  denser.
* Folded rows still sum to zero (constants are Neumann eigenfunctions, lambda = 0).
* The Neumann hemisphere spectrum l (l + 1) with multiplicity l + 1, and the
  two printed tables (tests/golden/hemisphere_eigen_errors_sec4_3.txt): our
  random samples are not the paper's, so the tables pin the size and the decay
  of the errors, not their digits.
"""
from __future__ import annotations

from pathlib import Path

import numpy as np

import oracle
from paper_1603_04100_gb300 import inputs as I

GOLDEN = Path(__file__).parent / "golden" / "hemisphere_eigen_errors_sec4_3.txt"


def _half_disk(n, nb, seed):
    g = np.random.default_rng(seed)
    r = np.sqrt(g.uniform(size=n - nb))
    t = g.uniform(0.0, np.pi, size=n - nb)
    inner = np.stack([r * np.cos(t), r * np.sin(t), np.zeros(n - nb)], axis=1)
    rim = np.stack([np.linspace(-1.0, 1.0, nb), np.zeros(nb), np.zeros(nb)], axis=1)
    b = np.zeros(n, dtype=np.uint8)
    b[:nb] = 1
    return np.concatenate([rim, inner]), b


def _rotation(seed):
    q, r = np.linalg.qr(np.random.default_rng(seed).standard_normal((3, 3)))
    return q * np.sign(np.diag(r))


def test_half_disk_ghosts_are_mirror_images():
    p, b = _half_disk(3000, 60, 1)
    R, t = _rotation(2), np.array([0.3, -1.2, 2.0])
    pm = p @ R.T + t
    nbr = oracle.knn_grid(pm, 16)
    g = oracle.neumann_ghosts(pm, b, nbr)
    assert g.pts.shape[0] > 60
    src = p[g.interior[g.src]]
    want = (src * np.array([1.0, -1.0, 1.0])) @ R.T + t
    assert np.abs(g.pts - want).max() <= 1e-12
    assert np.abs(g.dist - 2.0 * src[:, 1]).max() <= 1e-12
    # every ghost belongs to an interior point with a boundary neighbour, and to no other
    flagged = np.flatnonzero(b[nbr].any(axis=1) & (b == 0))
    assert np.array_equal(g.interior[g.src], flagged)
    # the boundary point used is the closest one (key: squared distance, then index)
    for s, bb in zip(g.src[:50], g.bnd[:50]):
        d2 = ((pm[b == 1] - pm[g.interior[s]]) ** 2).sum(1)
        assert bb == np.flatnonzero(b)[np.argmin(d2)]


def test_hemisphere_reflection_approaches_the_rim_plane():
    errs = []
    for n in (2000, 8000):
        p, b = I.hemisphere(n, 3)
        g = oracle.neumann_ghosts(p, b, oracle.knn_grid(p, 20))
        src = p[g.interior[g.src]]
        errs.append(np.abs(g.pts - src * np.array([1.0, 1.0, -1.0])).max())
    # second order in the spacing h ~ n^(-1/2): a factor of about 4 from 2000 to 8000
    assert errs[0] < 0.05 and errs[1] < errs[0] / 3, errs


def _neumann(p, b, k=20):
    nbr = oracle.knn_grid(p, k)
    g = oracle.neumann_ghosts(p, b, nbr)
    q, q_src = g.cloud(p)
    nq = oracle.knn_grid(q, k)
    vq, st, _, _ = oracle.assemble(q, nq)
    assert int(st[:g.interior.size].max()) == 0
    return oracle.neumann_fold(vq, nq, g.interior.size, q_src)


def test_folded_rows_sum_to_zero():
    p, b = I.hemisphere(3000, 4)
    val, col = _neumann(p, b)
    assert col.max() < val.shape[0]
    ones = np.ones(val.shape[0])
    Lx = oracle.to_csr(val, col) @ ones
    assert np.all(np.abs(Lx) <= 1e-12 * np.abs(val).sum(1))
    # some rows see their own ghost: the column equals the row
    assert np.any(col == np.arange(val.shape[0])[:, None])


def test_inhomogeneous_condition_is_exact_for_quadratic_data_on_a_plane():
    # half-disk y >= 0 with the rim on y = 0: the outward normal is -y, so for
    # u = 3y + y^2 - x^2 / 2 the condition is g = -du/dy = -3 on the rim, and the
    # ghost values U(p) + 2 y g = -3y + y^2 - x^2 / 2 are u's own values there: the
    # extended data is one quadratic, which the MVGD rows differentiate exactly
    p, b = _half_disk(3000, 60, 1)
    R, t = _rotation(2), np.array([0.3, -1.2, 2.0])
    pm = p @ R.T + t
    nbr = oracle.knn_grid(pm, 16)
    g = oracle.neumann_ghosts(pm, b, nbr)
    q, q_src = g.cloud(pm)
    nq = oracle.knn_grid(q, 16)
    vq, st, _, _ = oracle.assemble(q, nq)
    n_i = g.interior.size
    val, col = oracle.neumann_fold(vq, nq, n_i, q_src)
    x, y = p[g.interior, 0], p[g.interior, 1]
    u = 3.0 * y + y * y - 0.5 * x * x
    c = oracle.neumann_rhs(vq, nq, n_i, g, np.full(pm.shape[0], -3.0))
    lap = oracle.to_csr(val, col) @ u + c          # L applied to the extended data
    scale = np.abs(val).sum(1) * np.abs(u).max()
    assert np.all(np.abs(lap - 1.0) <= 1e-10 * scale), np.abs(lap - 1.0).max()
    # without the condition's term the rows near the rim are wrong
    assert np.abs(oracle.to_csr(val, col) @ u - 1.0).max() > 1.0


def test_inhomogeneous_hemisphere_converges_to_the_exact_solution():
    # u = z on the upper hemisphere: the rim's outward normal in the tangent plane is
    # -z, so dU/dn = -1; -Delta z = 2 z, so (I - L) u = 3 z with the condition's term
    import scipy.sparse.linalg as spl
    errs = []
    for n in (4000, 16000):
        p, b = I.hemisphere(n, 3)
        nbr = oracle.knn_grid(p, 20)
        g = oracle.neumann_ghosts(p, b, nbr)
        q, q_src = g.cloud(p)
        nq = oracle.knn_grid(q, 20)
        vq, _, _, _ = oracle.assemble(q, nq)
        val, col = oracle.neumann_fold(vq, nq, g.interior.size, q_src)
        z = p[g.interior, 2]
        A = oracle.system_matrix(val, col, 1.0).tocsc()
        c = oracle.neumann_rhs(vq, nq, g.interior.size, g, np.full(n, -1.0))
        errs.append(np.abs(spl.spsolve(A, 3.0 * z + c) - z).max())
        if n == 4000:  # without the term the rim condition is dU/dn = 0: far from z
            assert np.abs(spl.spsolve(A, 3.0 * z) - z).max() > 0.5
    assert errs[0] < 0.01 and errs[1] < errs[0] / 3, errs


def test_neumann_hemisphere_spectrum():
    want = np.array([0.0, 2, 2, 6, 6, 6, 12, 12, 12, 12, 20, 20, 20, 20, 20])
    errs = []
    for n in (2000, 8000):
        p, b = I.hemisphere(n, 3)
        val, col = _neumann(p, b)
        lam = oracle.lb_eigenvalues(val, col, 15)
        assert abs(lam[0]) <= 1e-9
        errs.append(np.abs(lam - want).max() / 20.0)
    assert errs[0] < 0.02 and errs[1] < errs[0] / 3, errs


def _golden():
    rows = {}
    for line in GOLDEN.read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            key, *vals = line.split()
            rows[key] = [float(v) for v in vals]
    return rows


def test_hemisphere_tables_size_and_decay():
    g = _golden()
    sizes = [2000, 4000, 8000]
    cols = [g["samples"].index(s) for s in sizes]
    ours = {key: [] for key in ("dirichlet_Einf_30", "dirichlet_Einf_182", "neumann_Einf_30", "neumann_Einf_182")}
    for n, c in zip(sizes, cols):
        nb = int(g["boundary_points"][c])
        p, b = I.hemisphere(n, 3, nb=nb)
        nbr = oracle.knn_grid(p, 20)
        val, _, _, _ = oracle.assemble(p, nbr)
        # Dirichlet: l (l + 1) with multiplicity l, so 30 is eigenvalues 10..14, 182 is 78..90
        lam = oracle.lb_eigenvalues(oracle.dirichlet_rows(val, b), nbr, 91, boundary=b)
        ours["dirichlet_Einf_30"].append(100 * np.abs(lam[10:15] / 30.0 - 1).max())
        ours["dirichlet_Einf_182"].append(100 * np.abs(lam[78:91] / 182.0 - 1).max())
        # Neumann: multiplicity l + 1, from l = 0: 30 is eigenvalues 15..20, 182 is 91..104
        v2, c2 = _neumann(p, b)
        lam = oracle.lb_eigenvalues(v2, c2, 105)
        ours["neumann_Einf_30"].append(100 * np.abs(lam[15:21] / 30.0 - 1).max())
        ours["neumann_Einf_182"].append(100 * np.abs(lam[91:105] / 182.0 - 1).max())
    for key, vals in ours.items():
        paper = np.array([g[key][c] for c in cols])
        ratio = np.array(vals) / paper
        assert np.all((ratio > 0.3) & (ratio < 6.0)), (key, vals, paper.tolist())
        assert vals[-1] < vals[0] / 3, (key, vals)
