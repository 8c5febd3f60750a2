"""The FP64 recompute identities of the mixed paths, checked in numpy.

The pivot of index g given the decisions on P is d_g = K_gg - b^T A^{-1} a
(A = K_P - 1_G, a = K[P, g], b = K[g, P]^T; Props. 3-5). The mixed paths
recompute it from approximate factors of A with
    real Hermitian : d = K_gg - a^T x0 - x0^T r - r^T A^{-1} r,
    LU             : d = K_gg - b^T x0 - y0^T r - s^T A^{-1} r,
    complex Herm.  : d = Re K_gg - Re(a^H x0) - Re(x0^H r) - r^H A^{-1} r,
exact for any x0 (and y0), with r = a - A x0, s = b - A^T y0, and the last
term taken from the approximate factors. With factors perturbed by eps the
result must be exact to second order in eps, while the pivot read off the
perturbed factors is off at first order.
"""
import numpy as np
import pytest

EPS = 1e-5


def _unit_lower(M):
    return np.tril(M, -1) + np.eye(M.shape[0])


def _perturbed_ldl(A, rng, complex_=False):
    """L, d with L D L^H ~ A to relative eps."""
    n = A.shape[0]
    E = rng.standard_normal((n, n))
    if complex_:
        E = E + 1j * rng.standard_normal((n, n))
    E = EPS * (E + E.conj().T) / 2 * np.abs(A).max()
    B = A + E
    L = np.eye(n, dtype=B.dtype)
    d = np.zeros(n)
    W = B.copy()
    for j in range(n):
        d[j] = W[j, j].real
        L[j + 1:, j] = W[j + 1:, j] / d[j]
        W[j + 1:, j + 1:] -= np.outer(L[j + 1:, j], W[j, j + 1:])
    return L, d


def _perturbed_lu(A, rng):
    """L, d, M (unit lower) with L D M^T ~ A to relative eps."""
    n = A.shape[0]
    B = A + EPS * rng.standard_normal((n, n)) * np.abs(A).max()
    L = np.eye(n)
    M = np.eye(n)
    d = np.zeros(n)
    W = B.copy()
    for j in range(n):
        d[j] = W[j, j]
        L[j + 1:, j] = W[j + 1:, j] / d[j]
        M[j + 1:, j] = W[j, j + 1:] / d[j]
        W[j + 1:, j + 1:] -= np.outer(W[j + 1:, j], W[j, j + 1:]) / d[j]
    return L, d, M


def _spd_like(n, rng, complex_=False):
    G = rng.standard_normal((n, n))
    if complex_:
        G = G + 1j * rng.standard_normal((n, n))
    Q, _ = np.linalg.qr(G)
    lam = rng.uniform(0.2, 0.9, n)
    return (Q * lam) @ Q.conj().T


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_hermitian_real_identity_second_order(seed):
    rng = np.random.default_rng(seed)
    n = 40
    K = _spd_like(n + 1, rng)
    keep = rng.random(n) < 0.5
    A = K[:n, :n] - np.diag(~keep * 1.0)
    a, kgg = K[:n, n], K[n, n]
    exact = kgg - a @ np.linalg.solve(A, a)
    L, d = _perturbed_ldl(A, rng)
    l = np.linalg.solve(L, a) / d                 # row g of the mixed L
    x0 = np.linalg.solve(L.T, l)
    r = a - A @ x0
    v = np.linalg.solve(L, r)
    d2 = kgg - a @ x0 - x0 @ r - np.sum(v * v / d)
    naive = kgg - l @ (d * l)
    assert abs(d2 - exact) < 50 * EPS ** 2 * (1 + abs(exact)), (d2, exact)
    assert abs(naive - exact) > abs(d2 - exact)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_lu_two_sided_identity_second_order(seed):
    rng = np.random.default_rng(seed)
    n = 40
    S = _spd_like(n + 1, rng)
    D = np.exp(0.5 * rng.standard_normal(n + 1))
    K = S * (D[None, :] / D[:, None])             # non-symmetric, same minors as S
    keep = rng.random(n) < 0.5
    A = K[:n, :n] - np.diag(~keep * 1.0)
    a, b, kgg = K[:n, n], K[n, :n], K[n, n]
    exact = kgg - b @ np.linalg.solve(A, a)
    L, d, M = _perturbed_lu(A, rng)
    m = np.linalg.solve(L, a) / d                 # row g of M
    l = np.linalg.solve(M, b) / d                 # row g of L
    x0 = np.linalg.solve(M.T, m)
    y0 = np.linalg.solve(L.T, l)
    r = a - A @ x0
    s = b - A.T @ y0
    v1 = np.linalg.solve(L, r)
    v2 = np.linalg.solve(M, s)
    d2 = kgg - b @ x0 - y0 @ r - np.sum(v1 * v2 / d)
    naive = kgg - l @ (d * m)
    assert abs(d2 - exact) < 50 * EPS ** 2 * (1 + abs(exact)), (d2, exact)
    assert abs(naive - exact) > abs(d2 - exact)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_hermitian_complex_identity_second_order(seed):
    rng = np.random.default_rng(seed)
    n = 40
    K = _spd_like(n + 1, rng, complex_=True)
    keep = rng.random(n) < 0.5
    A = K[:n, :n] - np.diag(~keep * 1.0)
    a, kgg = K[:n, n], K[n, n].real
    exact = kgg - (a.conj() @ np.linalg.solve(A, a)).real
    L, d = _perturbed_ldl(A, rng, complex_=True)
    lrow = (np.linalg.solve(L, a) / d).conj()     # row g of L: conj(D^-1 L^-1 a)
    x0 = np.linalg.solve(L.conj().T, lrow.conj())
    r = a - A @ x0
    v = np.linalg.solve(L, r)
    d2 = kgg - (a.conj() @ x0).real - (x0.conj() @ r).real - np.sum(np.abs(v) ** 2 / d)
    naive = kgg - np.sum(np.abs(lrow) ** 2 * d)
    assert abs(d2 - exact) < 50 * EPS ** 2 * (1 + abs(exact)), (d2, exact)
    assert abs(naive - exact) > abs(d2 - exact)


def test_fp32_decision_outside_the_band_equals_fp64():
    """The mixed chains decide in FP32 outside the borderline band: u (FP64) and
    the pivot's FP32 high part are each rounded to FP32. Every |u - d| > 2^-22
    (the band's floor) gives the same decision in FP32 as in FP64, since each
    rounding moves a value in (0, 2) by at most 2^-24; checked on a grid that
    crowds the band's edge."""
    import numpy as np
    rng = np.random.default_rng(0)
    u = rng.uniform(0.0, 1.0, 200000)
    for scale in (1.0, 1.000001, 0.999999):
        off = np.where(rng.random(u.size) < 0.5, 1.0, -1.0) * 2.0 ** -22 * scale * (1 + rng.random(u.size))
        d = np.clip(u + off, -1.0, 1.999)
        keep64 = u < d
        far = np.abs(u - d) > 2.0 ** -22
        keep32 = u.astype(np.float32) < d.astype(np.float32)
        assert np.array_equal(keep64[far], keep32[far])
