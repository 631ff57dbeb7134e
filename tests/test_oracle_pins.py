"""Pins of the FP64 oracle to facts fixed outside the oracle itself.

Each test states what fixes the expected value: a number printed in the paper
(tests/golden), a closed form of the continuous operator, an algebraic
identity of the method, an invariance, or an independent library routine.
"""
from __future__ import annotations

import math
from fractions import Fraction
from pathlib import Path

import numpy as np
import pytest

import oracle
from paper_1603_04100_gb300 import inputs as I

GOLDEN = Path(__file__).parent / "golden" / "line_example_sec3_2.txt"


def _golden():
    rows = {}
    for line in GOLDEN.read_text().splitlines():
        if not line.strip() or line.startswith("#"):
            continue
        key, rest = line.split(None, 1)
        rows[key] = [[Fraction(t) for t in part.split()] for part in rest.split(";")]
    return rows


# ---------------------------------------------------------------------------
# Sec. 3.2: the 1-D worked example, exact numbers printed in the paper
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("k", [1.0, 0.5, 3.0, 0.01])
def test_line_least_squares_weights_printed(k):
    g = _golden()["ls"][0]
    want = np.array([float(v) for v in g[:5]]) / (float(g[5]) * k * k)
    xs = k * np.arange(-2, 3, dtype=np.float64)
    got = oracle.line_weights(xs, 2, h=k, variant=oracle.VARIANT_LS)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())


@pytest.mark.parametrize("k", [1.0, 0.25, 2.0])
@pytest.mark.parametrize("r", [0.3, 0.6, 1.0, 2.0, 4.8, 6.0])
def test_line_mvgd_weights_printed(k, r):
    g = _golden()["mvgd"]
    pref = float(g[5][0]) / float(g[5][1])
    h = k * math.sqrt(r)
    want = pref / (h * h) * np.array([float(a) + float(b) * r for a, b in g[:5]])
    xs = k * np.arange(-2, 3, dtype=np.float64)
    got = oracle.line_weights(xs, 2, h=h, variant=oracle.VARIANT_MVGD)
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-12 * np.abs(want).max())
    # consistency: the row sums to zero (Sec. 3.2)
    assert abs(got.sum()) <= 1e-12 * np.abs(got).sum()
    # Eq. 8: M-matrix sign pattern iff 3/5 <= r <= 24/5
    lo_n, lo_d, hi_n, hi_d = [float(v) for v in _golden()["mmatrix_interval"][0]]
    mmatrix = got[2] < 0 and np.all(np.delete(got, 2) >= -1e-12 * np.abs(got).max())
    assert mmatrix == (lo_n / lo_d - 1e-12 <= r <= hi_n / hi_d + 1e-12)


def test_line_mvgd_at_h_equal_k():
    """Sec. 3.2: the quarter-range rule gives h = k and weights (2/70k^2)(4,19,-46,19,4)."""
    xs = np.arange(-2, 3, dtype=np.float64)
    h = 0.25 * (xs.max() - xs.min())
    assert h == 1.0
    got = oracle.line_weights(xs, 2, h=h)
    np.testing.assert_allclose(got, np.array([4, 19, -46, 19, 4]) * 2 / 70, rtol=1e-12)


def test_line_fit_coefficient_rows_printed():
    """The three rows (1/70k^2)[...] giving a0, a1, a2 (Sec. 3.2), via a = A^{-1} B."""
    g = _golden()
    k = 0.7
    xs = k * np.arange(-2, 3, dtype=np.float64)
    A = np.array([[float(v) for v in row] for row in g["normal_matrix"]])
    A = A * np.array([[1, k ** 2, k ** 2], [k ** 2, k ** 2, k ** 4], [k ** 2, k ** 4, k ** 4]])
    A[0, 0], A[0, 1], A[1, 0] = 5.0, 0.0, 0.0
    np.testing.assert_allclose(A, np.vander(xs, 3, increasing=True).T @ np.vander(xs, 3, increasing=True),
                               rtol=1e-14, atol=1e-14)
    B = np.vander(xs, 3, increasing=True).T
    a = np.linalg.solve(A, B)
    for name, row, scale in (("a0", 0, k ** 2), ("a1", 1, k), ("a2", 2, 1.0)):
        gr = g[name][0]
        want = np.array([float(v) for v in gr[:5]]) * scale / (float(gr[5]) * k ** 2)
        np.testing.assert_allclose(a[row], want, rtol=1e-12, atol=1e-14)
    # LS second derivative 2 a2 from the oracle equals the printed a2 row times 2
    np.testing.assert_allclose(oracle.line_weights(xs, 2, h=k, variant=oracle.VARIANT_LS), 2 * a[2],
                               rtol=1e-12)


# ---------------------------------------------------------------------------
# Sec. 2: the normal-equation matrix as printed (typo at [4][5] read as x y^3)
# ---------------------------------------------------------------------------

def test_normal_matrix_equals_vtv():
    rng = np.random.default_rng(5)
    x, y = rng.normal(size=13), rng.normal(size=13)
    V = np.stack([np.ones_like(x), x, y, x * x, x * y, y * y], axis=1)
    A = oracle.normal_matrix(x, y)
    np.testing.assert_allclose(A, V.T @ V, rtol=1e-13, atol=1e-13)
    assert np.allclose(A, A.T)
    np.testing.assert_allclose(A[4, 5], np.sum(x * y ** 3), rtol=1e-13)


# ---------------------------------------------------------------------------
# kNN (Sec. 2): brute force is the definition; scipy's kd-tree is independent
# ---------------------------------------------------------------------------

def test_knn_brute_matches_kdtree():
    from scipy.spatial import cKDTree
    p = I.random_sphere(3000, 11)
    k = 16
    nb = oracle.knn_brute(p, k)
    d, j = cKDTree(p).query(p, k + 1)
    assert np.all(j[:, 0] == np.arange(len(p)))
    np.testing.assert_array_equal(nb, j[:, 1:])


def test_knn_tie_break_by_index():
    """Integer lattice: many exact distance ties, broken by the lower index."""
    g = np.stack(np.meshgrid(np.arange(5), np.arange(4), np.arange(3), indexing="ij"), -1)
    p = g.reshape(-1, 3).astype(np.float64)
    perm = np.random.default_rng(3).permutation(len(p))
    p = p[perm]
    k = 10
    nb = oracle.knn_brute(p, k)
    for i in range(len(p)):
        d2 = ((p - p[i]) ** 2).sum(1)
        keys = sorted((d2[j], j) for j in range(len(p)) if j != i)
        assert list(nb[i]) == [j for _, j in keys[:k]]


@pytest.mark.parametrize("maker", [
    lambda: I.random_sphere(5000, 1),
    lambda: I.fibonacci_sphere(4000),
    lambda: I.torus(6000, 2),
    lambda: np.concatenate([I.random_sphere(800, 4), I.random_sphere(800, 4)[:300]]),  # duplicates
    lambda: np.concatenate([I.random_sphere(2000, 5) * 1e-3, I.random_sphere(500, 6) + 3.0]),
])
def test_knn_grid_equals_brute(maker):
    p = maker()
    for k in (12, 20):
        np.testing.assert_array_equal(oracle.knn_grid(p, k), oracle.knn_brute(p, k))


def test_row_sign_counts_on_the_line_example():
    # the 1-D rows of Sec. 3.2 laid out as [self, neighbours]: the MVGD row has the
    # M-matrix sign pattern exactly for 3/5 <= r <= 24/5 (Eq. 8), the least-squares
    # row (2, -1, -2, -1, 2) never (two negative neighbour weights)
    xs = np.arange(-2, 3, dtype=np.float64)
    rs = [0.3, 0.6, 1.0, 2.0, 4.8, 6.0]
    rows = []
    for r in rs:
        w = oracle.line_weights(xs, 2, h=math.sqrt(r), variant=oracle.VARIANT_MVGD)
        w[np.abs(w) <= 1e-12 * np.abs(w).max()] = 0.0  # the interval's ends hold exact zeros
        rows.append(np.concatenate([[w[2]], np.delete(w, 2)]))
    m_rows, neg, self_nonneg = oracle.row_sign_counts(np.array(rows))
    assert m_rows == sum(1 for r in rs if 0.6 <= r <= 4.8) == 4
    assert self_nonneg == 0
    ls = oracle.line_weights(xs, 2, h=1.0, variant=oracle.VARIANT_LS)
    assert oracle.row_sign_counts(np.array([np.concatenate([[ls[2]], np.delete(ls, 2)])])) == (0, 2, 0)
    # by hand: one row of each kind
    assert oracle.row_sign_counts(np.array([[-3.0, 1, 2, 0], [-1.0, 2, -1, 0], [0.5, -1, 0.5, 0]])) == (1, 2, 1)


# ---------------------------------------------------------------------------
# Structural invariants of the MVGD rows
# ---------------------------------------------------------------------------

def _rows(p, k, **kw):
    nb = oracle.knn_grid(p, k)
    val, st, dg, p00 = oracle.assemble(p, nb, **kw)
    return nb, val, st, dg, p00


@pytest.mark.parametrize("shape", I.SHAPES, ids=lambda s: s.kind)
@pytest.mark.parametrize("k", [12, 20])
def test_row_sums_vanish(shape, k):
    """Consistency (Sec. 2, Sec. 3.2): every row of L sums to zero."""
    p = shape.sample(4000, 7)
    nb, val, st, dg, _ = _rows(p, k)
    assert st.max() == 0
    eps = np.finfo(np.float64).eps
    assert np.all(np.abs(val.sum(1)) <= 1e3 * eps * np.abs(val).sum(1))


def _plane_cloud(n, seed):
    rng = np.random.default_rng(seed)
    uv = rng.uniform(-1, 1, size=(n, 2))
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    origin = rng.normal(size=3)
    p = origin + uv[:, :1] * Q[:, 0] + uv[:, 1:] * Q[:, 1]
    return p, uv


@pytest.mark.parametrize("delta_kind", [oracle.DELTA_MEAN_NN, oracle.DELTA_QUARTER_RANGE])
def test_planar_exactness(delta_kind):
    """On a plane the fits reproduce quadratics exactly, so L u equals the
    plane Laplacian of u (quadratic: a constant; linear and constant: zero)."""
    p, uv = _plane_cloud(3000, 9)
    nb, val, st, dg, _ = _rows(p, 16, delta_kind=delta_kind)
    assert st.max() == 0
    L = oracle.to_csr(val, nb)
    s, t = uv[:, 0], uv[:, 1]
    scale = np.abs(val).sum(1)
    for u, lap in ((np.ones_like(s), 0.0), (0.3 + 2 * s - 5 * t, 0.0),
                   (1.5 * s * s - 0.7 * s * t + 4.0 * t * t + s, 2 * 1.5 + 2 * 4.0)):
        r = L @ u - lap
        assert np.all(np.abs(r) <= 1e-9 * scale), np.abs(r / scale).max()


def test_identity_mvgd_minus_ls():
    """Eq. 9 generalised to 2-D: MVGD = LS + 2 tr(g^-1)/h^2 (U^{(i)}(0) - U_i),
    i.e. w_MVGD - w_LS = 2 (A3 + A5)/h^2 (P00 - e_self), row by row."""
    p = I.torus(3000, 3)
    nb = oracle.knn_grid(p, 16)
    w_m, _, dg, p00 = oracle.assemble(p, nb, variant=oracle.VARIANT_MVGD, want_p00=True)
    w_l, _, _, _ = oracle.assemble(p, nb, variant=oracle.VARIANT_LS)
    A3, A5, h = dg[:, 2], dg[:, 4], dg[:, 5]
    e = np.zeros_like(p00)
    e[:, 0] = 1.0
    want = (2 * (A3 + A5) / h ** 2)[:, None] * (p00 - e)
    scale = np.abs(w_m).max(1, keepdims=True)
    assert np.all(np.abs((w_m - w_l) - want) <= 1e-10 * scale)


def test_rigid_motion_and_scaling_invariance():
    """LB is intrinsic (Sec. 2): rows are unchanged by rotation and translation,
    and scale as 1/s^2 under p -> s p."""
    p = I.ellipsoid(3000, 8)
    nb, val, _, _, _ = _rows(p, 20)
    Q, _ = np.linalg.qr(np.random.default_rng(2).normal(size=(3, 3)))
    for s in (1.0, 3.7, 1e-3):
        q = s * (p @ Q.T) + np.array([0.4, -1.0, 2.0]) * s
        nb2 = oracle.knn_brute(q, 20)
        np.testing.assert_array_equal(nb2, nb)
        val2, _, _, _ = oracle.assemble(q, nb2)
        scale = np.abs(val).max(1, keepdims=True)
        assert np.all(np.abs(val2 * s * s - val) <= 1e-8 * scale)


def test_degenerate_neighbourhood_flagged():
    """Collinear samples cannot carry a quadratic surface fit: status 1."""
    t = np.linspace(0, 1, 50)
    p = np.stack([t, 2 * t, -t], axis=1) + 1e-300
    nb = oracle.knn_brute(p, 8)
    _, st, _, _ = oracle.assemble(p, nb)
    assert np.all(st > 0)


# ---------------------------------------------------------------------------
# Closed forms of the continuous operator (Sec. 4.2, Sec. 4.3)
# ---------------------------------------------------------------------------

def test_sphere_coordinates_converge():
    """-Delta p = 2 H p, on the unit sphere Delta x_i = -2 x_i (Eq. 11)."""
    errs = []
    for n in (642, 2562, 10242):
        p = I.fibonacci_sphere(n)
        nb, val, _, _, _ = _rows(p, 12, delta_m=6)
        L = oracle.to_csr(val, nb)
        errs.append(np.abs(L @ p + 2 * p).max())
    assert errs[0] < 0.05
    assert errs[1] < errs[0] / 3 and errs[2] < errs[1] / 3, errs


@pytest.mark.parametrize("l", [1, 2, 3, 4])
def test_spherical_harmonics_eigenvalues(l):
    """-Delta Y_l = l(l+1) Y_l on the unit sphere (Sec. 4.3).  The local
    truncation error is at least first order in h (Sec. 3.2), and h halves
    between the two clouds."""
    errs = []
    for n in (2562, 10242):
        p = I.fibonacci_sphere(n)
        nb, val, _, _, _ = _rows(p, 12)
        L = oracle.to_csr(val, nb)
        y = I.zonal_legendre(l, p[:, 2])
        errs.append(np.abs(L @ y + l * (l + 1) * y).max() / (l * (l + 1)))
    assert errs[1] < errs[0] / 1.8 and errs[1] < 5e-3, errs


def test_implicit_formula_pins_inputs():
    """The exact right-hand sides: the level-set formula agrees with the sphere
    closed forms and with the torus parametric formula."""
    p = I.random_sphere(500, 1)
    _, lap = I.surface_laplacian(I.SPHERE, p, "x")
    np.testing.assert_allclose(lap, -2 * p[:, 0], atol=1e-12)
    F, lap = I.surface_laplacian(I.SPHERE, p, "p3")
    np.testing.assert_allclose(lap, -12 * F, atol=1e-11)
    F, lap = I.surface_laplacian(I.SPHERE, p, "xy")
    np.testing.assert_allclose(lap, -6 * F, atol=1e-11)   # degree-2 harmonic
    th, ph = I.torus_params(400, 5)
    q = I.torus_points(th, ph)
    u, lap_param = I.torus_u_lap(th, ph)
    # sin(2 th) cos(3 ph) as an ambient function: use the parametric value and
    # check the level-set formula on the ambient functions it can represent
    th2, ph2 = I.torus_angles(q)
    np.testing.assert_allclose(np.sin(2 * th2) * np.cos(3 * ph2), u, atol=1e-12)
    # z = r sin(th): parametric LB from the torus formula vs level-set formula
    R, r = 1.0, 0.4
    rho = R + r * np.cos(th)
    lap_z_param = (1 / (r * r * rho)) * (-r * np.sin(th) * r * np.cos(th) - rho * r * np.sin(th))
    _, lap_z = I.surface_laplacian(I.TORUS, q, "z")
    np.testing.assert_allclose(lap_z, lap_z_param, atol=1e-11)


def test_torus_closed_form_converges():
    errs = []
    for n in (8000, 32000):
        th, ph = I.torus_params(n, 1)
        p = I.torus_points(th, ph)
        u, lap = I.torus_u_lap(th, ph)
        nb, val, st, _, _ = _rows(p, 16)
        assert st.max() == 0
        L = oracle.to_csr(val, nb)
        e = L @ u - lap
        errs.append(math.sqrt(np.mean(e * e) / np.mean(lap * lap)))
    # random sampling: the RMS truncation error decays at least at first order
    # in h (Sec. 3.2); h halves between the two clouds
    assert errs[1] < errs[0] / 1.8 and errs[1] < 0.06, errs


def test_solution_converges_second_order():
    """Sec. 4.2: roughly second-order L-infinity convergence on Fibonacci spheres."""
    hs, errs = [], []
    for n in (2562, 10242, 40962):
        pr = I.fibonacci_problem(n, 12)
        nb, val, _, dg, _ = _rows(pr.pts, pr.k)
        u, it, rr, st = oracle.bicgstab(val, nb, pr.f[:, 0], rtol=1e-12)
        assert st == 0 and rr <= 1e-12
        hs.append(math.sqrt(4 * math.pi / n))
        errs.append(np.abs(u - pr.u_exact[:, 0]).max())
    orders = [math.log(errs[i] / errs[i + 1]) / math.log(hs[i] / hs[i + 1]) for i in range(2)]
    assert min(orders) >= 1.5, (errs, orders)


# ---------------------------------------------------------------------------
# Operator application and solvers against independent library routines
# ---------------------------------------------------------------------------

def test_spmv_matches_scipy():
    p = I.torus(2000, 4)
    nb, val, _, _, _ = _rows(p, 16)
    L = oracle.to_csr(val, nb)
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2000, 3))
    y = rng.normal(size=(2000, 3))
    got = oracle.spmv(val, nb, x, sigma=1.7, alpha=-0.3, beta=2.0, y=y)
    want = -0.3 * (1.7 * x - L @ x) + 2.0 * y
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-10)


@pytest.mark.parametrize("solver", ["bicgstab", "gmres"])
def test_solvers_match_direct(solver):
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    pr = I.fibonacci_problem(2562, 12)
    nb, val, _, _, _ = _rows(pr.pts, pr.k)
    A = sp.identity(pr.n) - oracle.to_csr(val, nb)
    want = spla.spsolve(A.tocsc(), pr.f[:, 0])
    if solver == "bicgstab":
        u, it, rr, st = oracle.bicgstab(val, nb, pr.f[:, 0], rtol=1e-13)
    else:
        u, it, rr, st = oracle.gmres(val, nb, pr.f[:, 0], rtol=1e-13, restart=60)
    assert st == 0 and rr <= 1e-13
    assert np.linalg.norm(u - want) <= 1e-10 * np.linalg.norm(want)


# ---------------------------------------------------------------------------
# Open surfaces: Dirichlet rows (Sec. 3.1)
# ---------------------------------------------------------------------------

def test_dirichlet_hemisphere_converges_at_second_order():
    # u = z on the upper hemisphere: Delta_S z = -2z, so (I - L) u = 3z inside and
    # u = z is enforced on the rim band; the error against z falls like h^2
    errs = []
    for n in (4000, 16000):
        p, b = I.hemisphere(n, 3)
        nbr = oracle.knn_grid(p, 20)
        val, st, _, _ = oracle.assemble(p, nbr)
        assert int(st.max()) == 0
        v = oracle.dirichlet_rows(val, b)
        assert np.all(v[b == 1] == 0.0) and np.array_equal(v[b == 0], val[b == 0])
        z = p[:, 2]
        f = np.where(b == 1, z, 3.0 * z)
        u, _, rel, s = oracle.bicgstab(v, nbr, f, 1.0, rtol=1e-12, maxit=20000)
        assert s == 0 and rel <= 1e-12
        # the boundary rows read u_i = g_i, to the solver's tolerance
        assert np.abs(u[b == 1] - z[b == 1]).max() <= 1e-10
        errs.append(np.abs(u - z).max())
    assert errs[1] < 1e-4 and errs[0] / errs[1] > 3.0, errs  # observed order in h above 1.58
