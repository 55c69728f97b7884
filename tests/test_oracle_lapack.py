"""Pins of the oracle's factorisations and condition estimates against the
LAPACK routines the paper names for each route (Sec. 2.1-2.4).

The paper defines each route by its LAPACK calls: xGBTRF + xGBCON for
banded systems (Sec. 2.1), xTRCON for triangular ones (Sec. 2.2), xPOTRF +
xPOCON for likely-SPD ones (Sec. 2.3) and xGETRF + xGECON for the general
case (Sec. 2.4).  The oracle is plain C written without LAPACK, so these
tests check it against scipy's LAPACK binding:

* partial-pivoting pivot sequences identical to xGETRF / xGBTRF, on random
  matrices and on small-integer matrices whose columns carry ties in
  modulus (the first maximum wins in both).  LAPACK forms the multipliers
  with the reciprocal of the pivot, the oracle divides by the pivot (the
  plain definition of a multiplier); the two round differently, so a
  candidate that ties the pivot to one rounding may be taken by one and not
  the other.  A difference is accepted only there: at the first step where
  the sequences part, LAPACK's multiplier for the oracle's row must have
  modulus 1 to rounding, and the sequences agree exactly before it;
* L and U (dense and band storage, fill rows included) equal to rounding;
* rcond identical to xGECON / xPOCON / xTRCON / xGBCON to rounding, on
  random and on row- and column-graded matrices (scales 1e-8 .. 1e8) where
  rcond falls to 1e-33;
* the minimum-norm solution of the SVD fallback (Sec. 2.5, xGELSD) on
  gapless geometric spectra down to 1e-12, full rank and rank deficient,
  with the same cut-off (singular values <= n eps sigma_max dropped): the
  same rank, and solutions within 2 n eps kappa_k of each other (kappa_k
  the condition number of the kept part; observed <= 1.5 eps kappa_k).

The estimator follows Higham's 1-norm method, as xLACN2 does; the two must
take the same branch at every step for the estimates to agree to rounding,
which makes these tests sensitive to a wrong sign, a dropped transpose or
a different stopping rule in the oracle.
"""
import numpy as np
import pytest

lapack = pytest.importorskip("scipy.linalg.lapack")

RC_TOL = 1e-11      # observed <= 4e-13 relative up to n = 120, graded
SIZES = (1, 2, 5, 17, 64, 150)


def _norm1(A):
    return float(np.abs(A).sum(axis=0).max())


def _graded(rng, n):
    d1 = 10.0 ** rng.uniform(-8, 8, n)
    d2 = 10.0 ** rng.uniform(-8, 8, n)
    return d1[:, None] * rng.standard_normal((n, n)) * d2[None, :]


def _ties(rng, n):
    T = rng.integers(-2, 3, (n, n)).astype(np.float64)
    T[np.diag_indices(n)] += (np.diag(T) == 0)
    return T


def assert_same_pivots(ipiv, piv, mult):
    """ipiv (oracle) equals piv (LAPACK), or first differs at a step k where
    the row the oracle took ties LAPACK's pivot to rounding; mult(r, k) is
    LAPACK's stored multiplier of row r (after its swap) in column k."""
    diff = np.nonzero(np.asarray(ipiv) != np.asarray(piv))[0]
    if diff.size == 0:
        return
    k = int(diff[0])
    r = int(ipiv[k]) if int(ipiv[k]) != k else int(piv[k])
    assert abs(abs(mult(r, k)) - 1.0) <= 1e-13, (k, ipiv[k], piv[k], mult(r, k))


def _random_band(rng, n, kl, ku):
    A = np.zeros((n, n))
    for d in range(-kl, ku + 1):
        if abs(d) < n:
            A += np.diag(rng.standard_normal(n - abs(d)), d)
    return A


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("kind", ["random", "graded", "ties"])
def test_lu_pivots_factors_and_gecon(orc, n, kind):
    rng = np.random.default_rng(100 + n + {"random": 0, "graded": 1, "ties": 2}[kind])
    A = {"random": lambda: rng.standard_normal((n, n)),
         "graded": lambda: _graded(rng, n),
         "ties": lambda: _ties(rng, n)}[kind]()
    F, ipiv, info = orc.lu_factor(A)
    lu, piv, linfo = lapack.dgetrf(A)
    assert info == linfo == 0
    if kind != "ties":
        np.testing.assert_array_equal(ipiv, piv)
    else:
        assert_same_pivots(ipiv, piv, lambda r, k: lu[r, k])
        if not np.array_equal(ipiv, piv):
            return
    if kind != "graded":
        assert np.abs(F - lu).max() <= 1e-14 * n * max(1.0, np.abs(A).max())
    else:
        # entries span 32 orders of magnitude: compare each with its own scale
        assert np.all(np.abs(F - lu) <= 1e-12 * n * np.abs(lu) + 1e-300)
    anorm = _norm1(A)
    rc_lapack, _ = lapack.dgecon(lu, anorm, norm="1")
    rc = orc.rcond_from(anorm, orc.est_inv_norm1_lu(F, ipiv))
    assert rc == pytest.approx(rc_lapack, rel=RC_TOL)


@pytest.mark.parametrize("n", SIZES)
def test_cholesky_factor_and_pocon(orc, n):
    rng = np.random.default_rng(200 + n)
    G = rng.standard_normal((n, n))
    S = G.T @ G / n + np.diag(10.0 ** rng.uniform(-3, 0, n))
    S = np.tril(S) + np.tril(S, -1).T
    F, info = orc.chol_factor(S)
    c, linfo = lapack.dpotrf(S, lower=1)
    assert info == linfo == 0
    assert np.abs(np.tril(F) - np.tril(c)).max() <= 1e-13 * max(1.0, np.abs(S).max())
    anorm = _norm1(S)
    rc_lapack, _ = lapack.dpocon(c, anorm, uplo="L")
    rc = orc.rcond_from(anorm, orc.est_inv_norm1_chol(F))
    assert rc == pytest.approx(rc_lapack, rel=RC_TOL)


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("lower", [True, False])
def test_triangular_trcon(orc, n, lower):
    rng = np.random.default_rng(300 + n + 7 * lower)
    T = rng.standard_normal((n, n)) * (10.0 ** rng.uniform(-6, 6, n))[None, :]
    T = np.tril(T) if lower else np.triu(T)
    rc_lapack, _ = lapack.dtrcon(T, norm="1", uplo="L" if lower else "U", diag="N")
    rc = orc.rcond_from(_norm1(T), orc.est_inv_norm1_tri(T, lower))
    assert rc == pytest.approx(rc_lapack, rel=RC_TOL)


@pytest.mark.parametrize("n,kl,ku", [(1, 0, 0), (2, 1, 1), (9, 0, 3), (9, 3, 0),
                                     (40, 2, 3), (64, 1, 1), (150, 5, 2),
                                     (150, 0, 0), (33, 12, 9)])
@pytest.mark.parametrize("ties", [False, True])
def test_band_pivots_factors_and_gbcon(orc, n, kl, ku, ties):
    rng = np.random.default_rng(400 + n + 31 * kl + 7 * ku + ties)
    A = _random_band(rng, n, kl, ku)
    if ties:
        A = np.round(A)
        A[np.diag_indices(n)] += (np.diag(A) == 0)
    AB = orc.band_pack(A, kl, ku)
    F, ipiv, info = orc.band_lu_factor(AB, kl, ku)
    lub, piv, linfo = lapack.dgbtrf(AB, kl, ku)
    kv = kl + ku
    if info > 0:
        # exact zero pivot: the oracle stops there (the route then falls back);
        # xGBTRF reports the same step and the pivots before it agree
        assert linfo == info
        assert_same_pivots(ipiv[:info], piv[:info], lambda r, k: lub[kv + r - k, k])
        return
    if not ties:
        np.testing.assert_array_equal(ipiv, piv)
    else:
        assert_same_pivots(ipiv, piv, lambda r, k: lub[kv + r - k, k])
        if not np.array_equal(ipiv, piv):
            # the factors then belong to different pivot orders; the oracle's
            # must still solve A x = b with its own pivots
            b = A @ np.linspace(-1.0, 1.0, n)
            x = orc.band_lu_solve(F, kl, ku, ipiv, b)[:, 0]
            assert np.abs(A @ x - b).max() <= 1e-12 * n * max(1.0, np.abs(b).max())
            return
    assert linfo == 0
    assert np.abs(F - lub).max() <= 1e-14 * n * max(1.0, np.abs(A).max())
    anorm = _norm1(A)
    rc_lapack, _ = lapack.dgbcon(kl, ku, lub, piv, anorm, norm="1")
    rc = orc.rcond_from(anorm, orc.est_inv_norm1_band(F, kl, ku, ipiv))
    assert rc == pytest.approx(rc_lapack, rel=RC_TOL)


def test_singular_pivot_step_matches_getrf(orc):
    """xGETRF reports the first exactly-zero pivot (1-based); so must the
    oracle, with the same pivots before it."""
    A = np.array([[1.0, 2.0, 3.0, 4.0],
                  [2.0, 4.0, 6.0, 8.0],
                  [1.0, 0.0, 1.0, 0.0],
                  [0.0, 1.0, 1.0, 5.0]])
    A[:, 2] = A[:, 0] + A[:, 1]
    F, ipiv, info = orc.lu_factor(A)
    lu, piv, linfo = lapack.dgetrf(A)
    assert linfo > 0 and info == linfo
    np.testing.assert_array_equal(ipiv[:linfo - 1], piv[:linfo - 1])


@pytest.mark.parametrize("n", [6, 30, 80])
@pytest.mark.parametrize("lo", [-4, -8, -12])
@pytest.mark.parametrize("deficient", [0, 3])
def test_svd_min_norm_matches_gelsd(orc, n, lo, deficient):
    linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(500 + n + 10 * lo + deficient)
    U, _ = np.linalg.qr(rng.standard_normal((n, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    kept = np.logspace(0, lo, n - deficient)
    sig = np.concatenate([kept, np.full(deficient, 1e-20)])
    A = (U * sig) @ V.T
    B = rng.standard_normal((n, 2))
    eps = np.finfo(np.float64).eps
    X, rank = orc.svd_solve(A, B)                 # default cut-off n eps
    Xg, _, rank_g, _ = linalg.lstsq(A, B, cond=n * eps, lapack_driver="gelsd")
    assert rank == rank_g == n - deficient
    kappa_k = kept[0] / kept[-1]
    assert np.abs(X - Xg).max() <= 2 * n * eps * kappa_k * np.abs(Xg).max()


@pytest.mark.parametrize("n,kl,ku", [(50, 2, 2), (300, 8, 3), (200, 1, 7), (64, 32, 32)])
def test_column_dominant_band_takes_no_interchanges(orc, n, kl, ku):
    """Gaussian elimination keeps diagonal dominance by columns in every
    Schur complement, so partial pivoting finds the diagonal entry first at
    every step: the oracle's band LU and xGBTRF both return the identity
    pivot sequence, and the factors are those of elimination without
    pivoting."""
    rng = np.random.default_rng(600 + n + kl)
    A = _random_band(rng, n, kl, ku)
    np.fill_diagonal(A, 0.0)
    d = 1.0 + np.abs(A).sum(axis=0)            # column sums: dominance by columns
    A[np.diag_indices(n)] = d * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    AB = orc.band_pack(A, kl, ku)
    F, ipiv, info = orc.band_lu_factor(AB, kl, ku)
    lub, piv, linfo = lapack.dgbtrf(AB, kl, ku)
    assert info == linfo == 0
    np.testing.assert_array_equal(ipiv, np.arange(n))
    np.testing.assert_array_equal(piv, np.arange(n))
    # factors of unpivoted elimination, from the dense oracle LU with the
    # same (identity) pivots
    Fd, ipd, _ = orc.lu_factor(A)
    np.testing.assert_array_equal(ipd, np.arange(n))
    kv = kl + ku
    for j in range(n):
        for i in range(max(0, j - ku), min(n, j + kl + 1)):
            assert F[kv + i - j, j] == pytest.approx(Fd[i, j], rel=1e-12, abs=1e-14)
