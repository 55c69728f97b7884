"""Pins of the oracle's tridiagonal route (the closing remarks of the paper
name tridiagonal matrices, a common subtype of banded ones, for specialised
handling; opt-in flag TRIDIAG, banded systems with kl = ku = 1).

* LAPACK, through scipy: pivot sequence identical to xGTTRF and the four
  factor diagonals equal to rounding (both form the multiplier by division;
  ties keep the diagonal row), including small-integer matrices with ties;
  solutions equal to xGTTRS (A and A^T); rcond equal to xGTCON within
  1e-11 (the same Higham estimator iteration).
* The closed-form inverse of the tridiagonal Toeplitz matrix (Chebyshev
  polynomials, exact rationals): solution to the forward-error bound and an
  estimate never above the true ||inv(T)||_1.
* Routing: with the flag a banded tridiagonal system takes the tridiagonal
  route, in dense and in band storage (also with a declared band wider than
  the true one), and its X equals the band route's to the bit (the same
  pivots and the same operations in the same order); without the flag, or
  below the band rule's size, or with kl + ku > 2, the routes of Sec. 2.
* Failure: an exact zero pivot sends the system to the SVD (Sec. 2.5), as
  on the band route.
"""
from fractions import Fraction

import numpy as np
import pytest

from test_oracle_solvers import toeplitz_tridiag_inverse

lapack = pytest.importorskip("scipy.linalg.lapack")
RC_TOL = 1e-11


def tri(n, rng, ties=False, dominant=False):
    dl, d, du = rng.standard_normal(n - 1), rng.standard_normal(n), rng.standard_normal(n - 1)
    if ties:
        dl, d, du = np.round(2 * dl), np.round(2 * d), np.round(2 * du)
        d[d == 0] = 1.0
    if dominant:
        d = np.sign(d + 0.5) * (1.0 + np.abs(np.r_[dl, 0]) + np.abs(np.r_[0, du]))
    return dl, d, du


def dense(dl, d, du):
    return np.diag(d) + np.diag(dl, -1) + np.diag(du, 1)


@pytest.mark.parametrize("n", [3, 5, 17, 64, 301])
@pytest.mark.parametrize("ties", [False, True])
def test_gt_factor_matches_gttrf_gttrs_gtcon(orc, n, ties):
    rng = np.random.default_rng(700 + n + ties)
    dl, d, du = tri(n, rng, ties)
    fac = orc.gt_factor(dl, d, du)
    ldl, ld, ldu, ldu2, lpiv, linfo = lapack.dgttrf(dl, d, du)
    np.testing.assert_array_equal(fac[4], lpiv - 1)
    assert fac[5] == linfo
    if linfo:
        return
    assert np.any(fac[4] != np.arange(n)) or n < 17  # interchanges happen
    for got, ref in ((fac[0][:n - 1], ldl), (fac[1], ld), (fac[2][:n - 1], ldu), (fac[3][:max(n - 2, 0)], ldu2)):
        np.testing.assert_allclose(got, ref, rtol=1e-15, atol=1e-300)
    B = rng.standard_normal((n, 3))
    for trans in (0, 1):
        Xl, _ = lapack.dgttrs(ldl, ld, ldu, ldu2, lpiv, B, trans="T" if trans else "N")
        X = orc.gt_solve(fac, B, trans=bool(trans))
        A = dense(dl, d, du)
        At = A.T if trans else A
        kinf = np.linalg.norm(At, np.inf) * np.linalg.norm(np.linalg.inv(At), np.inf)
        assert np.abs(X - Xl).max() <= 8 * n * 2.0 ** -52 * kinf * np.abs(Xl).max()
    anorm = float(np.abs(dense(dl, d, du)).sum(axis=0).max())
    rc_l, _ = lapack.dgtcon(ldl, ld, ldu, ldu2, lpiv, anorm, norm="1")
    assert orc.rcond_from(anorm, orc.est_inv_norm1_gt(fac)) == pytest.approx(rc_l, rel=RC_TOL)


@pytest.mark.parametrize("n", [1, 2])
def test_gt_tiny_orders(orc, n):
    """Below xGTTRF's wrapper sizes: against the dense solve (n = 2: a row
    interchange when |dl| > |d|)."""
    d = np.array([0.5, 3.0][:n])
    dl, du = np.array([2.0][:n - 1]), np.array([1.0][:n - 1])
    fac = orc.gt_factor(dl, d, du)
    assert fac[5] == 0 and list(fac[4]) == ([1, 1] if n == 2 else [0])
    B = np.array([[1.0, -2.0], [0.25, 4.0]][:n])
    A = dense(dl, d, du)
    np.testing.assert_allclose(orc.gt_solve(fac, B), np.linalg.solve(A, B), rtol=1e-15)
    np.testing.assert_allclose(orc.gt_solve(fac, B, trans=True), np.linalg.solve(A.T, B), rtol=1e-15)


@pytest.mark.parametrize("n,a,b", [(12, 4, 1), (40, 3, -1), (64, 5, 2), (33, 2, -1)])
def test_gt_toeplitz_closed_form(orc, n, a, b):
    T = a * np.eye(n) + b * (np.eye(n, k=1) + np.eye(n, k=-1))
    inv = toeplitz_tridiag_inverse(n, a, b)
    rng = np.random.default_rng(n)
    bb = rng.integers(-5, 6, size=n)
    xe = np.array([float(sum(inv[i][k] * int(bb[k]) for k in range(n))) for i in range(n)])
    X, info = orc.solve(T, bb.astype(np.float64), flags=orc.TRIDIAG)
    assert info["route"] == orc.ROUTE_TRIDIAG and info["status"] == orc.OK, info
    kinf = np.abs(T).sum(1).max() * max(sum(abs(float(v)) for v in row) for row in inv)
    assert np.abs(X[:, 0] - xe).max() <= 4 * n * 2.0 ** -52 * kinf * np.abs(xe).max()
    true_inv1 = max(sum(abs(inv[i][j]) for i in range(n)) for j in range(n))
    assert info["rcond"] >= 1.0 / (np.abs(T).sum(0).max() * float(true_inv1)) * (1 - 1e-12)


def _band_storage(A, kld, kud):
    n = A.shape[0]
    AB = np.zeros((kld + kud + 1, n))
    for j in range(n):
        for i in range(max(0, j - kud), min(n, j + kld + 1)):
            AB[kud + i - j, j] = A[i, j]
    return AB


@pytest.mark.parametrize("n", [12, 50, 400])
def test_tridiag_route_equals_band_route(orc, n):
    rng = np.random.default_rng(800 + n)
    A = dense(*tri(n, rng))
    A[np.diag_indices(n)] += np.where(np.diag(A) < 0, -1.0, 1.0)
    B = rng.standard_normal((n, 2))
    Xt, it = orc.solve(A, B, flags=orc.TRIDIAG)
    Xb, ib = orc.solve(A, B)
    assert (it["cls"], it["route"], it["kl"], it["ku"]) == (orc.CLS_BANDED, orc.ROUTE_TRIDIAG, 1, 1), it
    assert (ib["cls"], ib["route"]) == (orc.CLS_BANDED, orc.ROUTE_BAND_LU), ib
    assert it["status"] == ib["status"] == orc.OK
    np.testing.assert_array_equal(Xt, Xb)
    assert it["rcond"] == ib["rcond"]
    # band storage, declared band wider than the true one
    Xs, isb = orc.solve_band(_band_storage(A, 3, 2), 3, 2, B, flags=orc.TRIDIAG)
    assert (isb["route"], isb["kl"], isb["ku"]) == (orc.ROUTE_TRIDIAG, 1, 1), isb
    np.testing.assert_array_equal(Xs, Xt)
    assert isb["rcond"] == it["rcond"]


def test_other_systems_keep_their_routes(orc):
    rng = np.random.default_rng(9)
    small = dense(*tri(8, rng, dominant=True))        # n < 12: not banded by the 25% rule
    _, i = orc.solve(small, np.ones(8), flags=orc.TRIDIAG)
    assert i["route"] != orc.ROUTE_TRIDIAG, i
    n = 60
    penta = dense(*tri(n, rng)) + np.diag(rng.standard_normal(n - 2), 2)   # ku = 2
    _, i = orc.solve(penta, np.ones(n), flags=orc.TRIDIAG)
    assert (i["cls"], i["route"]) == (orc.CLS_BANDED, orc.ROUTE_BAND_LU), i


def test_tridiag_zero_pivot_goes_to_svd(orc):
    n = 40
    rng = np.random.default_rng(10)
    A = dense(*tri(n, rng, dominant=True))
    A[:, 17] = 0.0
    B = rng.standard_normal((n, 1))
    Xt, it = orc.solve(A, B, flags=orc.TRIDIAG)
    Xb, ib = orc.solve(A, B)
    assert it["route"] == orc.ROUTE_TRIDIAG and it["status"] == orc.W_APPROX, it
    assert ib["status"] == orc.W_APPROX and it["svd_rank"] == ib["svd_rank"] == n - 1
    np.testing.assert_array_equal(Xt, Xb)  # the same SVD of the same A
    _, it = orc.solve(A, B, flags=orc.TRIDIAG | orc.NO_APPROX)
    assert it["status"] == orc.E_SINGULAR
