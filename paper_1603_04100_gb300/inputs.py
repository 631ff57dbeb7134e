"""Seeded synthetic point clouds and exact continuous solutions.

This module is shared by the CUDA path, its tests, the benchmark and the FP64
oracle's tests.  It holds none of the discretisation's arithmetic: it only
samples surfaces and evaluates closed-form functions and their exact
Laplace-Beltrami values, so that both sides of a parity test receive the same
FP64 inputs and the same exact answers.

Surfaces (Sec. 4.2 uses spheres sampled uniformly and at random; the torus and
ellipsoid stand in for the paper's public clouds, which are not available):

* ``fibonacci_sphere(N)``: z_i = 1 - (2i+1)/N, phi_i = 2 pi i / Phi with the
  golden ratio Phi, i = 0..N-1 (the Fibonacci lattice of Sec. 4.2, written for
  any N, odd or even).
* ``random_sphere(N, seed)``: rows of a PCG64 standard normal N x 3 draw,
  each divided by its norm.
* ``ellipsoid(N, seed, axes)``: a random sphere scaled by its semi-axes.
* ``torus(N, seed, R, r)``: (theta, phi) uniform on [0, 2pi)^2, accepted when
  1.75 U < 1 + 0.75 cos(theta), i.e. a parameter-space density proportional
  to 1 + 0.75 cos(theta).

Exact Laplace-Beltrami values (Eq. 1 of Sec. 2, with the paper's sign
convention that the operator is negative semi-definite):

* on a level set phi = 0 with unit normal n = grad phi / |grad phi| and total
  curvature kappa = div n, the surface Laplacian of an ambient function F is
  Delta F - n^T (Hess F) n - kappa (n . grad F);
* on the torus the parametric form with metric r^2 dtheta^2 + rho^2 dphi^2,
  rho = R + r cos(theta), is used as an independent check of the above.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GOLDEN = (1.0 + math.sqrt(5.0)) / 2.0


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ----------------------------------------------------------------------------
# Samplers
# ----------------------------------------------------------------------------

def fibonacci_sphere(n: int) -> np.ndarray:
    """Fibonacci lattice on the unit sphere, FP64 [n][3]."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    phi = 2.0 * math.pi * i / GOLDEN
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.ascontiguousarray(np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1))


def random_sphere(n: int, seed: int) -> np.ndarray:
    """Uniform random points on the unit sphere (normalised Gaussian rows)."""
    g = _rng(seed).standard_normal((n, 3))
    return np.ascontiguousarray(g / np.linalg.norm(g, axis=1, keepdims=True))


def hemisphere(n: int, seed: int, nb: int | None = None) -> tuple[np.ndarray, np.ndarray]:
    """n points of the upper unit hemisphere and its boundary mask: nb points (default
    round(sqrt(2 pi n) / 2), about the interior spacing apart) evenly spaced on the rim
    circle z = 0 with a random phase, flagged 1, then n - nb uniform random points with
    z > 0, flagged 0."""
    rng = _rng(seed)
    if nb is None:
        nb = int(round(math.sqrt(2.0 * math.pi * n) / 2.0))
    out, have = [], 0
    while have < n - nb:
        g = rng.standard_normal((2 * (n - nb - have) + 64, 3))
        g /= np.linalg.norm(g, axis=1, keepdims=True)
        g = g[g[:, 2] > 0.0]
        out.append(g)
        have += g.shape[0]
    inner = np.concatenate(out)[:n - nb]
    t = (np.arange(nb) + rng.uniform()) * (2.0 * math.pi / nb)
    rim = np.stack([np.cos(t), np.sin(t), np.zeros(nb)], axis=1)
    pts = np.ascontiguousarray(np.concatenate([rim, inner]))
    boundary = np.zeros(n, dtype=np.uint8)
    boundary[:nb] = 1
    return pts, boundary


def morton_permutation(pts: np.ndarray, bits: int = 10) -> np.ndarray:
    """Indices that order the points along a Z-order curve of their bounding
    cube (`bits` per axis, stable in the original index): consecutive points
    are then spatial neighbours, as in the stored order the kNN step produces."""
    lo = pts.min(axis=0)
    span = float((pts.max(axis=0) - lo).max()) or 1.0
    q = np.minimum(((pts - lo) / span * (1 << bits)).astype(np.int64), (1 << bits) - 1)
    code = np.zeros(pts.shape[0], dtype=np.int64)
    for b in range(bits):
        for d in range(3):
            code |= ((q[:, d] >> b) & 1) << (3 * b + d)
    return np.argsort(code, kind="stable")


def morton_sorted(pts: np.ndarray, bits: int = 10) -> np.ndarray:
    """The same points reordered along a Z-order curve (morton_permutation)."""
    return np.ascontiguousarray(pts[morton_permutation(pts, bits)])


def ellipsoid(n: int, seed: int, axes=(1.0, 0.7, 0.4)) -> np.ndarray:
    """Random sphere points scaled by the semi-axes (a, b, c)."""
    return np.ascontiguousarray(random_sphere(n, seed) * np.asarray(axes, dtype=np.float64))


def torus_params(n: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Rejection-sampled (theta, phi) with density proportional to 1 + 0.75 cos(theta)."""
    rng = _rng(seed)
    th_out, ph_out, have = [], [], 0
    while have < n:
        m = max(1024, int(1.5 * (n - have)) + 16)
        th = rng.uniform(0.0, 2.0 * math.pi, m)
        ph = rng.uniform(0.0, 2.0 * math.pi, m)
        u = rng.uniform(0.0, 1.0, m)
        keep = 1.75 * u < 1.0 + 0.75 * np.cos(th)
        th_out.append(th[keep])
        ph_out.append(ph[keep])
        have += int(keep.sum())
    return np.concatenate(th_out)[:n], np.concatenate(ph_out)[:n]


def torus_points(theta: np.ndarray, phi: np.ndarray, R: float = 1.0, r: float = 0.4) -> np.ndarray:
    rho = R + r * np.cos(theta)
    return np.ascontiguousarray(
        np.stack([rho * np.cos(phi), rho * np.sin(phi), r * np.sin(theta)], axis=1))


def torus(n: int, seed: int, R: float = 1.0, r: float = 0.4) -> np.ndarray:
    th, ph = torus_params(n, seed)
    return torus_points(th, ph, R, r)


# ----------------------------------------------------------------------------
# Level-set descriptions (phi, grad phi, Hess phi) of the three surfaces
# ----------------------------------------------------------------------------

@dataclass(frozen=True)
class Shape:
    kind: str                      # "sphere" | "ellipsoid" | "torus"
    axes: tuple = (1.0, 1.0, 1.0)  # ellipsoid semi-axes
    R: float = 1.0                 # torus radii
    r: float = 0.4

    def sample(self, n: int, seed: int) -> np.ndarray:
        if self.kind == "sphere":
            return random_sphere(n, seed)
        if self.kind == "ellipsoid":
            return ellipsoid(n, seed, self.axes)
        if self.kind == "torus":
            return torus(n, seed, self.R, self.r)
        raise ValueError(self.kind)

    def grad_hess(self, p: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
        """Gradient [n][3] and Hessian [n][3][3] of the level-set function."""
        x, y, z = p[:, 0], p[:, 1], p[:, 2]
        n = p.shape[0]
        if self.kind in ("sphere", "ellipsoid"):
            a, b, c = self.axes if self.kind == "ellipsoid" else (1.0, 1.0, 1.0)
            w = np.array([1.0 / a ** 2, 1.0 / b ** 2, 1.0 / c ** 2])
            g = 2.0 * p * w
            H = np.zeros((n, 3, 3))
            H[:, 0, 0], H[:, 1, 1], H[:, 2, 2] = 2 * w[0], 2 * w[1], 2 * w[2]
            return g, H
        # torus: phi = (s - R)^2 + z^2 - r^2 with s = sqrt(x^2 + y^2)
        s = np.sqrt(x * x + y * y)
        f = (s - self.R) / s
        g = np.stack([2 * x * f, 2 * y * f, 2 * z], axis=1)
        H = np.zeros((n, 3, 3))
        # d/dx_i of 2 x_j (1 - R/s) = 2 delta_ij (1 - R/s) + 2 x_j R x_i / s^3
        c3 = 2.0 * self.R / s ** 3
        H[:, 0, 0] = 2 * f + c3 * x * x
        H[:, 1, 1] = 2 * f + c3 * y * y
        H[:, 0, 1] = H[:, 1, 0] = c3 * x * y
        H[:, 2, 2] = 2.0
        return g, H


SPHERE = Shape("sphere")
ELLIPSOID = Shape("ellipsoid", axes=(1.0, 0.7, 0.4))
TORUS = Shape("torus", R=1.0, r=0.4)
SHAPES = (SPHERE, ELLIPSOID, TORUS)


# ----------------------------------------------------------------------------
# Ambient test functions with exact gradient and Hessian
# ----------------------------------------------------------------------------

def _fn_x(p):
    n = p.shape[0]
    g = np.zeros((n, 3)); g[:, 0] = 1.0
    return p[:, 0].copy(), g, np.zeros((n, 3, 3))


def _fn_z(p):
    n = p.shape[0]
    g = np.zeros((n, 3)); g[:, 2] = 1.0
    return p[:, 2].copy(), g, np.zeros((n, 3, 3))


def _fn_yz(p):
    n = p.shape[0]
    y, z = p[:, 1], p[:, 2]
    g = np.zeros((n, 3)); g[:, 1] = z; g[:, 2] = y
    H = np.zeros((n, 3, 3)); H[:, 1, 2] = H[:, 2, 1] = 1.0
    return y * z, g, H


def _fn_xy(p):
    n = p.shape[0]
    x, y = p[:, 0], p[:, 1]
    g = np.zeros((n, 3)); g[:, 0] = y; g[:, 1] = x
    H = np.zeros((n, 3, 3)); H[:, 0, 1] = H[:, 1, 0] = 1.0
    return x * y, g, H


def _fn_x2my2(p):
    n = p.shape[0]
    x, y = p[:, 0], p[:, 1]
    g = np.zeros((n, 3)); g[:, 0] = 2 * x; g[:, 1] = -2 * y
    H = np.zeros((n, 3, 3)); H[:, 0, 0] = 2.0; H[:, 1, 1] = -2.0
    return x * x - y * y, g, H


def _fn_sinx_expy(p):
    n = p.shape[0]
    x, y = p[:, 0], p[:, 1]
    sx, cx, ey = np.sin(x), np.cos(x), np.exp(y)
    g = np.zeros((n, 3)); g[:, 0] = cx * ey; g[:, 1] = sx * ey
    H = np.zeros((n, 3, 3))
    H[:, 0, 0] = -sx * ey; H[:, 1, 1] = sx * ey; H[:, 0, 1] = H[:, 1, 0] = cx * ey
    return sx * ey, g, H


def _fn_p3(p):
    """5 z^3 - 3 z: on the unit sphere twice the degree-3 zonal Legendre polynomial."""
    n = p.shape[0]
    z = p[:, 2]
    g = np.zeros((n, 3)); g[:, 2] = 15 * z * z - 3
    H = np.zeros((n, 3, 3)); H[:, 2, 2] = 30 * z
    return 5 * z ** 3 - 3 * z, g, H


FUNCTIONS = {
    "x": _fn_x, "z": _fn_z, "yz": _fn_yz, "xy": _fn_xy, "x2-y2": _fn_x2my2,
    "sinx_expy": _fn_sinx_expy, "p3": _fn_p3,
}
BATCH_RHS = ("x", "yz", "x2-y2", "sinx_expy")


def surface_laplacian(shape: Shape, p: np.ndarray, fname: str) -> tuple[np.ndarray, np.ndarray]:
    """(F, Delta_Sigma F) at points p on the level set of ``shape``."""
    F, gF, HF = FUNCTIONS[fname](p)
    gphi, Hphi = shape.grad_hess(p)
    gn = np.linalg.norm(gphi, axis=1)
    nrm = gphi / gn[:, None]
    lap_phi = np.trace(Hphi, axis1=1, axis2=2)
    nHn_phi = np.einsum("ni,nij,nj->n", nrm, Hphi, nrm)
    kappa = (lap_phi - nHn_phi) / gn
    lapF = np.trace(HF, axis1=1, axis2=2)
    nHn_F = np.einsum("ni,nij,nj->n", nrm, HF, nrm)
    dnF = np.einsum("ni,ni->n", nrm, gF)
    return F, lapF - nHn_F - kappa * dnF


def zonal_legendre(l: int, z: np.ndarray) -> np.ndarray:
    """Legendre polynomial P_l(z); on the unit sphere Delta P_l(z) = -l(l+1) P_l(z)."""
    p0, p1 = np.ones_like(z), z.copy()
    if l == 0:
        return p0
    for k in range(1, l):
        p0, p1 = p1, ((2 * k + 1) * z * p1 - k * p0) / (k + 1)
    return p1


def torus_u_lap(theta: np.ndarray, phi: np.ndarray, R: float = 1.0, r: float = 0.4):
    """u = sin(2 theta) cos(3 phi) and its exact LB for the metric r^2 dth^2 + rho^2 dph^2."""
    rho = R + r * np.cos(theta)
    u = np.sin(2 * theta) * np.cos(3 * phi)
    lap = np.cos(3 * phi) * (-2.0 * np.sin(theta) * np.cos(2 * theta) / (r * rho)
                             - 4.0 * np.sin(2 * theta) / r ** 2
                             - 9.0 * np.sin(2 * theta) / rho ** 2)
    return u, lap


def torus_angles(p: np.ndarray, R: float = 1.0) -> tuple[np.ndarray, np.ndarray]:
    phi = np.mod(np.arctan2(p[:, 1], p[:, 0]), 2 * math.pi)
    s = np.sqrt(p[:, 0] ** 2 + p[:, 1] ** 2)
    theta = np.mod(np.arctan2(p[:, 2], s - R), 2 * math.pi)
    return theta, phi


# ----------------------------------------------------------------------------
# Workloads: one cloud + right-hand sides for (sigma I - L) u = f, sigma = 1
# ----------------------------------------------------------------------------

@dataclass
class Problem:
    name: str
    pts: np.ndarray            # [n][3] FP64
    k: int
    u_exact: np.ndarray        # [n][r] FP64
    f: np.ndarray              # [n][r] FP64, f = sigma u - Delta u
    sigma: float = 1.0
    delta_m: int = 6           # mean distance to the delta_m nearest neighbours
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.pts.shape[0]

    @property
    def nrhs(self) -> int:
        return self.u_exact.shape[1]


def fibonacci_problem(n: int = 2562, k: int = 12) -> Problem:
    """Unit Fibonacci sphere; u = x (Delta x = -2x), f = 3x."""
    p = fibonacci_sphere(n)
    u = p[:, 0:1].copy()
    return Problem(f"fibonacci_sphere_n{n}_k{k}", p, k, u, 3.0 * u)


def random_sphere_problem(n: int = 1_048_576, k: int = 20, seed: int = 0) -> Problem:
    """Random unit sphere; u = 5z^3 - 3z (degree-3 zonal harmonic), f = 13 u."""
    p = random_sphere(n, seed)
    z = p[:, 2]
    u = (5 * z ** 3 - 3 * z)[:, None]
    return Problem(f"random_sphere_n{n}_k{k}", p, k, u, 13.0 * u)


def torus_problem(n: int = 524_288, k: int = 16, seed: int = 1) -> Problem:
    """Rejection-sampled torus; u = sin(2 theta) cos(3 phi), f = u - Delta u."""
    th, ph = torus_params(n, seed)
    p = torus_points(th, ph)
    u, lap = torus_u_lap(th, ph)
    return Problem(f"torus_n{n}_k{k}", p, k, u[:, None], (u - lap)[:, None])


def shape_problem(shape: Shape, n: int, k: int, seed: int, fnames) -> Problem:
    p = shape.sample(n, seed)
    us, fs = [], []
    for fn in fnames:
        F, lap = surface_laplacian(shape, p, fn)
        us.append(F)
        fs.append(F - lap)
    return Problem(f"{shape.kind}_n{n}_k{k}_s{seed}", p, k,
                   np.ascontiguousarray(np.stack(us, axis=1)),
                   np.ascontiguousarray(np.stack(fs, axis=1)), meta={"shape": shape.kind})


@dataclass(frozen=True)
class CloudSpec:
    shape: Shape
    n: int
    k: int
    seed: int
    rhs: tuple

    def build(self) -> Problem:
        return shape_problem(self.shape, self.n, self.k, self.seed, self.rhs)


def batched_specs(count: int = 256, seed: int = 2, n_lo: int = 2000, n_hi: int = 262_144):
    """Uneven clouds: N log-uniform in [n_lo, n_hi], shape uniform over the three
    families, K uniform over {12, 20}, four smooth right-hand sides each."""
    rng = _rng(seed)
    specs = []
    for c in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        shape = SHAPES[int(rng.integers(0, 3))]
        k = (12, 20)[int(rng.integers(0, 2))]
        specs.append(CloudSpec(shape, n, k, seed * 1_000_003 + c, BATCH_RHS))
    return specs


@dataclass(frozen=True)
class RequestSpec:
    rid: int
    arrival_s: float
    cloud: CloudSpec


def serving_trace(count: int = 4000, seed: int = 3, rate_per_s: float = 200.0,
                  n_lo: int = 1000, n_hi: int = 1_048_576, k: int = 20):
    """Poisson arrivals; N log-uniform in [n_lo, n_hi]; 1..8 right-hand sides."""
    rng = _rng(seed)
    names = tuple(FUNCTIONS.keys())
    t = 0.0
    out = []
    for rid in range(count):
        t += rng.exponential(1.0 / rate_per_s)
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        shape = SHAPES[int(rng.integers(0, 3))]
        nr = int(rng.integers(1, 9))
        rhs = tuple(names[(rid + j) % len(names)] for j in range(nr))
        out.append(RequestSpec(rid, t, CloudSpec(shape, n, k, seed * 1_000_003 + rid, rhs)))
    return out
