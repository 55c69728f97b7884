"""Pins of the oracle's symmetric-indefinite route (the paper's closing
remarks name plain symmetric matrices -- symmetric but not positive
definite -- for specialised handling; opt-in flag SYM_INDEF, n <= 1024).

* LAPACK, through scipy: the Bunch-Kaufman pivot sequence identical to
  xSYTRF's (unblocked: a workspace too small for blocking), 1 x 1 and
  2 x 2 pivots alike, and D and L equal to rounding; rcond equal to
  xSYCON's within 1e-11 (the same Higham estimator iteration).
* Invariants: P A P^T = L D L^T to rounding, D's 2 x 2 blocks indefinite
  (negative determinant), the growth of |L| bounded as Bunch-Kaufman
  guarantees (|l_ij| <= 1 / (1 - alpha) for 1 x 1 pivots).
* Cramer's rule in exact rationals on small integer matrices that force
  2 x 2 pivots (zero diagonal).
* Routing: symmetric within the Fig. 4 tolerance and not likely_sympd ->
  LDL^T; likely_sympd but not positive definite -> Cholesky fails -> LDL^T;
  non-symmetric, FORCE_LU, n > 1024, or without the flag -> the routes of
  Sec. 2; an exactly zero column -> the SVD fallback.
"""
from fractions import Fraction

import numpy as np
import pytest

lapack = pytest.importorskip("scipy.linalg.lapack")
ALPHA = (1 + np.sqrt(17.0)) / 8


def sym(n, rng):
    G = rng.standard_normal((n, n))
    return G + G.T


def lapack_pivots(ipiv):
    """LAPACK's 1-based signed pivots in the oracle's encoding."""
    return np.where(ipiv > 0, ipiv - 1, ipiv)


def unpack(F, ipiv):
    """L (unit lower), D (block diagonal) and the permutation P with
    P A P^T = L D L^T, from the factor storage (interchanges applied to
    the earlier columns of L, as the solve does implicitly)."""
    n = F.shape[0]
    L = np.eye(n)
    D = np.zeros((n, n))
    perm = np.arange(n)
    k = 0
    blocks = []
    while k < n:
        if ipiv[k] >= 0:
            kp, step = ipiv[k], 1
            kk = k
        else:
            kp, step = -ipiv[k] - 1, 2
            kk = k + 1
        if kp != kk:  # the interchange applies to the earlier columns of L too
            L[[kk, kp], :k] = L[[kp, kk], :k]
            perm[[kk, kp]] = perm[[kp, kk]]
        D[k, k] = F[k, k]
        if step == 2:
            D[k + 1, k] = D[k, k + 1] = F[k + 1, k]
            D[k + 1, k + 1] = F[k + 1, k + 1]
            L[k + 2:, k] = F[k + 2:, k]
            L[k + 2:, k + 1] = F[k + 2:, k + 1]
        else:
            L[k + 1:, k] = F[k + 1:, k]
        blocks.append((k, step))
        k += step
    return L, D, perm, blocks


@pytest.mark.parametrize("n", [1, 2, 3, 7, 20, 64])
@pytest.mark.parametrize("kind", ["random", "zero_diag", "ties"])
def test_ldlt_matches_sytrf_and_sycon(orc, n, kind):
    rng = np.random.default_rng(1000 + n + len(kind))
    A = sym(n, rng)
    if kind == "zero_diag":
        A[np.diag_indices(n)] = 0.0           # forces 2 x 2 pivots
    if kind == "ties":
        A = np.round(A)
        if n > 1:
            A[np.diag_indices(n)] = 0.0
    F, ipiv, info = orc.ldlt_factor(A)
    lu, piv, linfo = lapack.dsytrf(A, lower=1, lwork=max(n, 1))
    assert info == linfo
    np.testing.assert_array_equal(ipiv, lapack_pivots(piv))
    if kind == "zero_diag" and n >= 2:
        assert np.any(ipiv < 0)               # a 2 x 2 pivot was taken
    if info:
        return
    low = np.tril_indices(n)
    np.testing.assert_allclose(F[low], lu[low], rtol=1e-12, atol=1e-13 * np.abs(A).max())
    anorm = float(np.abs(A).sum(axis=0).max())
    rc_l, _ = lapack.dsycon(lu, piv, anorm, lower=1)
    assert orc.rcond_from(anorm, orc.est_inv_norm1_ldlt(F, ipiv)) == pytest.approx(rc_l, rel=1e-11)
    B = rng.standard_normal((n, 3))
    X = orc.ldlt_solve(F, ipiv, B)
    Xl, _ = lapack.dsytrs(lu, piv, B, lower=1)
    kinf = np.linalg.norm(A, np.inf) * np.linalg.norm(np.linalg.inv(A), np.inf)
    assert np.abs(X - Xl).max() <= 8 * n * 2.0 ** -52 * kinf * max(np.abs(Xl).max(), 1e-300)


@pytest.mark.parametrize("n", [5, 30, 200])
def test_ldlt_invariants(orc, n):
    rng = np.random.default_rng(1100 + n)
    A = sym(n, rng)
    A[np.diag_indices(n)] *= 0.05
    F, ipiv, info = orc.ldlt_factor(A)
    assert info == 0
    L, D, perm, blocks = unpack(F, ipiv)
    PA = A[np.ix_(perm, perm)]
    assert np.abs(L @ D @ L.T - PA).max() <= 64 * n * 2.0 ** -52 * np.abs(A).max() * max(1.0, np.abs(L).max()) ** 2
    for k, step in blocks:
        if step == 2:
            assert D[k, k] * D[k + 1, k + 1] - D[k + 1, k] ** 2 < 0  # indefinite block
        else:
            assert np.abs(L[k + 1:, k]).max(initial=0.0) <= 1.0 / (1.0 - ALPHA) + 1e-12


def _exact_solve(A, b):
    n = len(b)
    M = [[Fraction(int(A[i][j])) for j in range(n)] + [Fraction(int(b[i]))] for i in range(n)]
    for c in range(n):
        p = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                M[r] = [x - f * y for x, y in zip(M[r], M[c])]
    return [M[i][n] / M[i][i] for i in range(n)]


@pytest.mark.parametrize("A", [[[0, 1], [1, 0]], [[0, 2, 1], [2, 0, 3], [1, 3, 0]],
                               [[1, 4, 0, 2], [4, 0, 1, 1], [0, 1, -2, 5], [2, 1, 5, 0]]])
def test_ldlt_exact_small(orc, A):
    A = np.array(A, dtype=np.float64)
    n = A.shape[0]
    b = np.arange(1.0, n + 1)
    F, ipiv, info = orc.ldlt_factor(A)
    assert info == 0
    x = orc.ldlt_solve(F, ipiv, b)[:, 0]
    xe = np.array([float(v) for v in _exact_solve(A, b)])
    assert np.abs(x - xe).max() <= 64 * 2.0 ** -52 * np.abs(xe).max()


def test_ldlt_routing(orc):
    rng = np.random.default_rng(12)
    n = 40
    A = sym(n, rng)                                  # symmetric, indefinite: fails Fig. 4 (diagonal)
    b = rng.standard_normal((n, 1))
    X, i = orc.solve(A, b, flags=orc.SYM_INDEF)
    assert (i["cls"], i["route"], i["status"]) == (orc.CLS_GENERAL, orc.ROUTE_LDLT, orc.OK), i
    assert np.abs(A @ X - b).max() <= 1e-12 * np.abs(A).sum(1).max() * np.abs(X).max()
    _, i = orc.solve(A, b)
    assert i["route"] == orc.ROUTE_LU
    _, i = orc.solve(A, b, flags=orc.SYM_INDEF | orc.FORCE_LU)
    assert i["route"] == orc.ROUTE_LU
    Z = A.copy()
    Z[3, 7] += 1e-9                                  # asymmetric beyond 100 eps
    _, i = orc.solve(Z, b, flags=orc.SYM_INDEF)
    assert i["route"] == orc.ROUTE_LU
    eps = np.finfo(float).eps
    Y = 1e3 * A                                      # within the relative test only
    Y[3, 7] = Y[7, 3] * (1 + 50 * eps)
    assert abs(Y[3, 7] - Y[7, 3]) > 100 * eps
    _, i = orc.solve(Y, b, flags=orc.SYM_INDEF)
    assert i["route"] == orc.ROUTE_LDLT, i
    T = A.copy()                                     # within the absolute test only
    T[3, 7], T[7, 3] = 1e-20, 3e-20
    _, i = orc.solve(T, b, flags=orc.SYM_INDEF)
    assert i["route"] == orc.ROUTE_LDLT, i
    # passes Fig. 4 but is not positive definite: Cholesky fails -> LDL^T
    C = np.array([[1, .9, .9], [.9, 1, -.9], [.9, -.9, 1]])
    X, i = orc.solve(C, np.ones(3), flags=orc.SYM_INDEF)
    assert (i["cls"], i["route"]) == (orc.CLS_SYMPD, orc.ROUTE_CHOL_FAIL_LDLT), i
    assert np.abs(C @ X[:, 0] - 1).max() < 1e-13
    _, i = orc.solve(C, np.ones(3))
    assert i["route"] == orc.ROUTE_CHOL_FAIL_LU
    # a zero column: no LDL^T without a zero pivot -> the SVD fallback
    S = A.copy()
    S[:, 11] = 0.0
    S[11, :] = 0.0
    _, i = orc.solve(S, b, flags=orc.SYM_INDEF)
    assert (i["route"], i["status"], i["svd_rank"]) == (orc.ROUTE_LDLT, orc.W_APPROX, n - 1), i


def test_ldlt_size_limit(orc):
    rng = np.random.default_rng(13)
    n = orc.LDLT_NMAX + 1
    A = sym(n, rng)
    _, i = orc.solve(A, rng.standard_normal(n), flags=orc.SYM_INDEF)
    assert i["route"] == orc.ROUTE_LU
