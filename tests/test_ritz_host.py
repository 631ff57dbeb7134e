"""The eigensolver's host-side p x p steps in the library (no GPU needed):
mvgd_block_chol_inverse against a Cholesky factorisation by numpy, and
mvgd_ritz_values (Hessenberg reduction + Francis double-shift QR) against the
eigenvalues numpy's LAPACK finds, on matrices with real, complex, repeated and
clustered eigenvalues."""
import ctypes as C

import numpy as np
import pytest


@pytest.fixture(scope="module")
def L():
    from paper_1603_04100_gb300 import _lib as LB, build
    build.build()
    return LB.load()


def _ritz(L, H):
    from paper_1603_04100_gb300 import _lib as LB
    H = np.ascontiguousarray(H, dtype=np.float64)
    p = H.shape[0]
    re, im = np.empty(p), np.empty(p)
    st = L.mvgd_ritz_values(H.ctypes.data_as(C.c_void_p), p, re.ctypes.data_as(C.c_void_p),
                            im.ctypes.data_as(C.c_void_p))
    assert st == LB.OK, LB.status_string(st)
    return re + 1j * im


def _match(got, want, tol):
    # every eigenvalue of `want` has a distinct partner in `got` within tol (greedy on sorted order)
    got, want = list(got), list(want)
    for w in sorted(want, key=lambda z: (z.real, z.imag)):
        j = int(np.argmin([abs(g - w) for g in got]))
        assert abs(got[j] - w) <= tol, (w, got[j])
        got.pop(j)


@pytest.mark.parametrize("p,seed", [(1, 0), (2, 1), (3, 2), (8, 3), (33, 4), (96, 5), (128, 6)])
def test_ritz_values_random(L, p, seed):
    H = np.random.default_rng(seed).standard_normal((p, p))
    want = np.linalg.eigvals(H)
    got = _ritz(L, H)
    scale = max(1.0, np.abs(want).max())
    _match(got, want, 1e-9 * scale)
    # complex eigenvalues come in conjugate pairs; real ones have im == 0 exactly
    assert np.isclose(np.sum(got.imag), 0.0, atol=1e-9 * scale)


def test_ritz_values_of_a_nearly_symmetric_projected_operator(L):
    # the shape of X^T L X on the sphere: multiplets -l(l+1) of sizes 2l+1, a small
    # nonsymmetric perturbation, in a random orthonormal basis
    rng = np.random.default_rng(7)
    lam = np.concatenate([np.full(2 * l + 1, -l * (l + 1.0)) for l in range(7)])[:48]
    Q, _ = np.linalg.qr(rng.standard_normal((48, 48)))
    H = Q @ np.diag(lam) @ Q.T + 1e-6 * rng.standard_normal((48, 48))
    got = np.sort(_ritz(L, H).real)
    want = np.sort(np.linalg.eigvals(H).real)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-8 * 42)


def test_ritz_values_exact_cases(L):
    # a rotation block (eigenvalues +-i), a Jordan-free triangular matrix, a zero matrix
    got = _ritz(L, np.array([[0.0, -1.0], [1.0, 0.0]]))
    _match(got, [1j, -1j], 1e-15)
    T = np.triu(np.arange(1.0, 26.0).reshape(5, 5))
    _match(_ritz(L, T), np.diag(T).astype(complex), 1e-12)
    _match(_ritz(L, np.zeros((4, 4))), np.zeros(4, complex), 0.0)
    # companion matrix of (x-1)(x-2)(x-3)(x-4)(x-5)
    c = np.poly([1, 2, 3, 4, 5])
    Cm = np.zeros((5, 5))
    Cm[0] = -c[1:]
    Cm[1:, :-1] = np.eye(4)
    _match(_ritz(L, Cm), np.arange(1.0, 6.0).astype(complex), 1e-8)


@pytest.mark.parametrize("p", [1, 8, 64, 128])
def test_block_chol_inverse(L, p):
    from paper_1603_04100_gb300 import _lib as LB
    rng = np.random.default_rng(p)
    Y = rng.standard_normal((3 * p + 5, p))
    G = Y.T @ Y
    G[0, -1] += 1e-13  # slightly unsymmetric, as a computed Gram matrix is
    Rinv = np.empty((p, p))
    st = L.mvgd_block_chol_inverse(np.ascontiguousarray(G).ctypes.data_as(C.c_void_p), p,
                                   Rinv.ctypes.data_as(C.c_void_p))
    assert st == LB.OK
    R = np.linalg.cholesky(0.5 * (G + G.T)).T
    np.testing.assert_allclose(Rinv, np.linalg.inv(R), rtol=0, atol=1e-10 * np.abs(np.linalg.inv(R)).max())
    assert np.all(np.tril(Rinv, -1) == 0.0)
    # Y R^-1 has orthonormal columns
    Qm = Y @ Rinv
    np.testing.assert_allclose(Qm.T @ Qm, np.eye(p), atol=1e-10)


def test_block_chol_inverse_rejects_indefinite(L):
    from paper_1603_04100_gb300 import _lib as LB
    G = np.array([[1.0, 2.0], [2.0, 1.0]])
    out = np.empty((2, 2))
    assert L.mvgd_block_chol_inverse(G.ctypes.data_as(C.c_void_p), 2, out.ctypes.data_as(C.c_void_p)) == LB.EDEGENERATE
    assert L.mvgd_ritz_values(G.ctypes.data_as(C.c_void_p), 0, out.ctypes.data_as(C.c_void_p),
                              out.ctypes.data_as(C.c_void_p)) == LB.EINVAL
