"""Neumann boundary by reflection (Sec. 3.1) -- TEST INFRASTRUCTURE ONLY.

Plain numpy, FP64, in the order the paper takes the steps:

1. An interior point whose K nearest neighbours include a boundary point gets
   a ghost.  Its closest boundary point p_b (key: squared distance, then index)
   carries a local frame:
   * e2, the surface normal at p_b: the eigenvector of the smallest eigenvalue
     of the covariance of p_b's K nearest neighbours in the whole cloud;
   * e1, the boundary tangent: p_b and its kb nearest boundary points give a
     principal axis t (largest covariance eigenvalue) and two others u, v; the
     curve through them is fitted as (xi, eta(xi), zeta(xi)), eta and zeta
     quadratics in xi = (p - p_b).t by least squares, and its tangent at p_b is
     t + eta'(0) u + zeta'(0) v;
   * e3 = e1 x e2, the normal of the boundary in the tangent plane (e1 is first
     made orthogonal to e2, so that the frame is orthonormal).
   The ghost is the point mirrored through the plane of e1, e2 at p_b:
   p^R = p - 2 ((p - p_b).e3) e3.
2. The unknowns are the interior points; the cloud Q = interior points (in
   point order) followed by the ghosts; each interior point's K nearest
   neighbours are taken in Q, its MVGD row assembled there, and every ghost
   column then points at the interior point it mirrors: with a homogeneous
   condition U(p^R) = U(p), so the weights of a point and of its ghost add up.
3. An inhomogeneous condition dU/dn = g sets U(p^R) = U(p) + |p - p^R| g(p_b);
   the known part moves to the right-hand side: row i of L U gains
   c_i = sum over its ghost neighbours of w_ij |p - p^R| g(p_b), and
   (sigma I - L) u = f becomes (sigma I - L_folded) u = f + c.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Ghosts:
    interior: np.ndarray    # [n_I] point index of interior position i (ascending)
    pts: np.ndarray         # [n_G][3] ghost coordinates
    src: np.ndarray         # [n_G] interior position of the mirrored point
    bnd: np.ndarray         # [n_G] point index of the boundary point used
    dist: np.ndarray        # [n_G] |p - p^R|

    def cloud(self, pts) -> tuple:
        """(Q [n_I + n_G][3], q_src [n_I + n_G]): interior points, then ghosts; q_src maps
        every point of Q to the interior position it stands for."""
        q = np.concatenate([np.asarray(pts, dtype=np.float64)[self.interior], self.pts])
        q_src = np.concatenate([np.arange(self.interior.size), self.src]).astype(np.int64)
        return np.ascontiguousarray(q), q_src


def _d2(a, b):
    d = a - b
    return (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]


def surface_normal(pts, nbr, b) -> np.ndarray:
    """PCA normal at point b from its K nearest neighbours (barycentre of the K)."""
    d = pts[nbr[b]] - pts[b]
    c = d - d.mean(axis=0)
    w, v = np.linalg.eigh(c.T @ c)
    return v[:, 0]


def boundary_tangent(pts, bidx, b, kb) -> np.ndarray:
    """Tangent of the boundary curve at boundary point b (a point index) from its kb
    nearest boundary points (bidx: every boundary point index, ascending)."""
    others = bidx[bidx != b]
    d2 = _d2(pts[others], pts[b])
    near = others[np.lexsort((others, d2))][:kb]
    d = pts[np.concatenate([[b], near])] - pts[b]
    c = d - d.mean(axis=0)
    w, v = np.linalg.eigh(c.T @ c)
    t, u, s = v[:, 2], v[:, 1], v[:, 0]
    xi = d @ t
    V = np.stack([np.ones_like(xi), xi, xi * xi], axis=1)
    coef, *_ = np.linalg.lstsq(V, np.stack([d @ u, d @ s], axis=1), rcond=None)
    tan = t + coef[1, 0] * u + coef[1, 1] * s
    return tan / np.linalg.norm(tan)


def boundary_normal(pts, nbr, bidx, b, kb) -> np.ndarray:
    """e3 at boundary point b: the unit normal of the boundary in the tangent plane."""
    e2 = surface_normal(pts, nbr, b)
    e1 = boundary_tangent(pts, bidx, b, kb)
    e1 = e1 - (e1 @ e2) * e2
    e1 /= np.linalg.norm(e1)
    e3 = np.cross(e1, e2)
    return e3 / np.linalg.norm(e3)


def neumann_ghosts(pts, boundary, nbr, kb: int = 6) -> Ghosts:
    """Step 1: the ghosts of the interior points next to the boundary."""
    pts = np.asarray(pts, dtype=np.float64)
    bmask = np.asarray(boundary).astype(bool)
    interior = np.flatnonzero(~bmask)
    bidx = np.flatnonzero(bmask)
    kb = min(kb, bidx.size - 1)
    e3 = {}
    g_pts, g_src, g_bnd, g_dist = [], [], [], []
    for pos, i in enumerate(interior):
        if not bmask[nbr[i]].any():
            continue
        d2 = _d2(pts[bidx], pts[i])
        b = int(bidx[np.lexsort((bidx, d2))[0]])
        if b not in e3:
            e3[b] = boundary_normal(pts, nbr, bidx, b, kb)
        s = (pts[i] - pts[b]) @ e3[b]
        g_pts.append(pts[i] - 2.0 * s * e3[b])
        g_src.append(pos)
        g_bnd.append(b)
        g_dist.append(2.0 * abs(s))
    return Ghosts(interior=interior, pts=np.array(g_pts).reshape(-1, 3), src=np.array(g_src, dtype=np.int64),
                  bnd=np.array(g_bnd, dtype=np.int64), dist=np.array(g_dist))


def fold(val_q, nbr_q, n_interior: int, q_src) -> tuple:
    """Step 2's last part: the rows of the interior points (the first n_interior of Q)
    with every column mapped to the interior position it stands for.  Returns
    (val [n_I][k+1], col [n_I][k]); a column may repeat or equal the row itself."""
    q_src = np.asarray(q_src)
    return np.array(val_q[:n_interior], copy=True), q_src[np.asarray(nbr_q[:n_interior])]


def neumann_rhs(val_q, nbr_q, n_interior: int, ghosts: Ghosts, g) -> np.ndarray:
    """Step 3: c [n_I] for dU/dn = g, g given at every point of the original cloud
    (read at the boundary points), the outward normal of the boundary."""
    val_q = np.asarray(val_q, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    c = np.zeros(n_interior)
    for i in range(n_interior):
        for s, j in enumerate(nbr_q[i]):
            if j >= n_interior:
                t = j - n_interior
                c[i] += val_q[i, s + 1] * ghosts.dist[t] * g[ghosts.bnd[t]]
    return c
