"""Pins of the oracle's band-storage driver (or_solve_band, Sec. 2.1).

A system given in compact band storage (A(i, j) at AB[ku + i - j, j],
ldab >= kl + ku + 1, LAPACK's layout for xGBTRF / xGBTRS / xGBCON) takes
the banded route with the true bandwidths found inside the declared band;
the driver takes ||A||_1 from the band, repacks into the factor layout
(kl extra fill rows) and densifies for the SVD fallback.  Nothing in it is
checked by the dense-input tests, so these tests pin it against:

* the dense-input oracle on the same matrix, where the scan routes it to the
  band solver: class, route and kl/ku equal, and X and rcond identical to
  the bit (the two drivers pack the same entries into the same factor
  layout, so any index slip in either packs a different matrix);
* scipy's xGBSV (the solution within the forward-error bound) and xGBTRF +
  xGBCON on the true band (rcond to rounding), with the declared band
  wider than the true one, one-sided bands, ldab above kl + ku + 1, and
  n <= 4 with declared bandwidths beyond n;
* entries of AB outside the matrix (the unused corners and rows below the
  declared band) set to NaN: they must never be read;
* a singular band (zero column): the SVD fallback on the densified matrix,
  equal to the dense oracle's and to xGELSD's minimum-norm solution.
"""
import numpy as np
import pytest

lapack = pytest.importorskip("scipy.linalg.lapack")
linalg = pytest.importorskip("scipy.linalg")

EPS = np.finfo(np.float64).eps
RC_TOL = 1e-11


def _random_band(rng, n, kl, ku):
    A = np.zeros((n, n))
    for d in range(-kl, ku + 1):
        if abs(d) < n:
            A += np.diag(rng.standard_normal(n - abs(d)), d)
    return A


def _storage(A, kld, kud, extra_rows=0, junk=np.nan):
    """Band storage of A with declared bandwidths kld/kud; every position that
    does not hold an entry of A (corners, rows below the band) is `junk`."""
    n = A.shape[0]
    ldab = kld + kud + 1 + extra_rows
    AB = np.full((ldab, n), junk)
    for j in range(n):
        for i in range(max(0, j - kud), min(n, j + kld + 1)):
            AB[kud + i - j, j] = A[i, j]
    return AB


def _true_bandwidths(A):
    nz = np.argwhere(A != 0.0)
    if nz.size == 0:
        return 0, 0
    d = nz[:, 0] - nz[:, 1]
    return int(max(0, d.max())), int(max(0, (-d).max()))


def _lapack_band(A, kl, ku):
    """xGBTRF input for the true band: kl fill rows on top."""
    n = A.shape[0]
    ab = np.zeros((2 * kl + ku + 1, n))
    for j in range(n):
        for i in range(max(0, j - ku), min(n, j + kl + 1)):
            ab[kl + ku + i - j, j] = A[i, j]
    return ab


CASES = [  # (n, true kl, true ku, declared extra kl, extra ku, extra ldab rows)
    (200, 2, 2, 0, 0, 0), (200, 3, 1, 2, 3, 0), (150, 0, 3, 0, 2, 1), (150, 4, 0, 3, 0, 2),
    (300, 7, 5, 1, 1, 3), (120, 1, 1, 5, 5, 0), (128, 12, 9, 0, 0, 4), (97, 0, 0, 2, 2, 0),
]


@pytest.mark.parametrize("n,kl,ku,xl,xu,xr", CASES)
def test_band_driver_against_dense_oracle_and_gbsv(orc, n, kl, ku, xl, xu, xr):
    rng = np.random.default_rng(900 + n + 13 * kl + 5 * ku + xl + 3 * xu)
    A = _random_band(rng, n, kl, ku)
    # a diagonal shifted away from zero keeps one-sided bands well conditioned;
    # two-sided ones still interchange rows under partial pivoting
    A[np.diag_indices(n)] += np.where(np.diag(A) < 0, -1.5, 1.5)
    tkl, tku = _true_bandwidths(A)
    assert (tkl, tku) == (kl, ku)
    B = rng.standard_normal((n, 3))
    AB = _storage(A, kl + xl, ku + xu, extra_rows=xr)
    X, info = orc.solve_band(AB, kl + xl, ku + xu, B)
    assert info["status"] == orc.OK, info
    assert (info["cls"], info["route"], info["kl"], info["ku"]) == \
        (orc.CLS_BANDED, orc.ROUTE_BAND_LU, kl, ku), info
    # the dense-input oracle routes the same matrix to the band solver
    Xd, infod = orc.solve(A, B)
    assert (infod["cls"], infod["route"], infod["kl"], infod["ku"]) == \
        (orc.CLS_BANDED, orc.ROUTE_BAND_LU, kl, ku), infod
    np.testing.assert_array_equal(X, Xd)
    assert info["rcond"] == infod["rcond"]
    # LAPACK: xGBSV's solution, xGBTRF + xGBCON's rcond on the true band
    Xs = linalg.solve_banded((kl, ku), _storage(A, kl, ku, junk=0.0), B)
    kinf = np.linalg.norm(A, np.inf) * np.linalg.norm(np.linalg.inv(A), np.inf)
    assert np.abs(X - Xs).max() <= 4 * n * EPS * kinf * np.abs(Xs).max()
    lub, piv, linfo = lapack.dgbtrf(_lapack_band(A, kl, ku), kl, ku)
    assert linfo == 0
    if kl > 0:
        assert np.any(piv != np.arange(n))   # the case exercises pivoting
    anorm = float(np.abs(A).sum(axis=0).max())
    rc_l, _ = lapack.dgbcon(kl, ku, lub, piv, anorm, norm="1")
    assert info["rcond"] == pytest.approx(rc_l, rel=RC_TOL)


@pytest.mark.parametrize("n", [1, 2, 3, 4])
@pytest.mark.parametrize("kld,kud", [(0, 0), (1, 0), (0, 1), (1, 1), (3, 2), (5, 5)])
def test_band_driver_tiny(orc, n, kld, kud):
    rng = np.random.default_rng(40 + n * 11 + kld * 3 + kud)
    A = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if -kud <= i - j <= kld:
                A[i, j] = float(rng.integers(-4, 5))
    A[np.diag_indices(n)] = 9.0 + np.arange(n)   # non-singular, exact small integers
    tkl, tku = _true_bandwidths(A)
    B = rng.standard_normal((n, 2))
    X, info = orc.solve_band(_storage(A, kld, kud), kld, kud, B)
    assert info["status"] == orc.OK, info
    assert (info["cls"], info["kl"], info["ku"]) == (orc.CLS_BANDED, tkl, tku), info
    np.testing.assert_allclose(X, np.linalg.solve(A, B), rtol=0, atol=64 * EPS * np.abs(B).max())
    if tkl + tku > 0:
        lub, piv, linfo = lapack.dgbtrf(_lapack_band(A, tkl, tku), tkl, tku)
        rc_l, _ = lapack.dgbcon(tkl, tku, lub, piv, float(np.abs(A).sum(axis=0).max()), norm="1")
    else:  # diagonal: rcond = min|d| / max|d| exactly
        d = np.abs(np.diag(A))
        rc_l = d.min() / d.max()
    assert info["rcond"] == pytest.approx(rc_l, rel=RC_TOL)


def test_band_driver_nonfinite_inside_band_only(orc):
    n, kl, ku = 50, 2, 3
    rng = np.random.default_rng(7)
    A = _random_band(rng, n, kl, ku)
    A[np.diag_indices(n)] += 4.0
    B = rng.standard_normal((n, 1))
    AB = _storage(A, kl, ku, extra_rows=2)    # NaN in every unused position
    _, info = orc.solve_band(AB, kl, ku, B)
    assert info["status"] == orc.OK
    AB[ku + 10 - 9, 9] = np.inf               # an entry of A inside the band
    _, info = orc.solve_band(AB, kl, ku, B)
    assert info["status"] == orc.E_NONFINITE
    AB = _storage(A, kl, ku)
    Bn = B.copy()
    Bn[17, 0] = np.nan
    _, info = orc.solve_band(AB, kl, ku, Bn)
    assert info["status"] == orc.E_NONFINITE


def test_band_driver_singular_goes_to_svd(orc):
    n, kl, ku = 60, 2, 1
    rng = np.random.default_rng(11)
    A = _random_band(rng, n, kl, ku)
    A[np.diag_indices(n)] += 5.0
    A[:, 23] = 0.0                            # a zero column: no LU exists
    B = rng.standard_normal((n, 2))
    X, info = orc.solve_band(_storage(A, kl, ku), kl, ku, B)
    assert info["status"] == orc.W_APPROX and info["route"] == orc.ROUTE_BAND_LU, info
    assert info["svd_rank"] == n - 1
    Xd, infod = orc.solve(A, B)
    assert infod["status"] == orc.W_APPROX and infod["route"] == orc.ROUTE_BAND_LU, infod
    np.testing.assert_array_equal(X, Xd)
    Xg, _, rank, sv = linalg.lstsq(A, B, cond=n * EPS, lapack_driver="gelsd")
    assert rank == n - 1
    kappa_k = sv[0] / sv[rank - 1]
    assert np.abs(X - Xg).max() <= 2 * n * EPS * kappa_k * np.abs(Xg).max()
