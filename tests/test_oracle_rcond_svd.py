"""Pins for the oracle's condition estimate, SVD fallback and compensated
residual (paper Sec. 2, 2.5).

The estimate of ||inv(A)||_1 is pinned by being a lower bound of the true
norm (computed from an explicit inverse), by exactness on diagonal matrices
and n = 1, and by staying within a small factor of the truth on random
matrices.  The Jacobi SVD is pinned against numpy's LAPACK SVD and its
invariants; the minimum-norm solve against the pseudo-inverse; the Dot2
residual against exact rational arithmetic.
"""
from fractions import Fraction

import numpy as np
import pytest

EPS = np.finfo(np.float64).eps


def inv_norm1(A):
    return np.abs(np.linalg.inv(A)).sum(axis=0).max()


def test_estimator_exact_on_diagonals(orc):
    for n in (1, 2, 7, 30):
        d = np.linspace(-3.0, 5.0, n) + 0.37
        A = np.diag(d)
        Fm, ipiv, _ = orc.lu_factor(A)
        est = orc.est_inv_norm1_lu(Fm, ipiv)
        assert est == pytest.approx(np.max(1.0 / np.abs(d)), rel=1e-15)
        assert orc.est_inv_norm1_tri(A, True) == pytest.approx(np.max(1 / np.abs(d)), rel=1e-15)


@pytest.mark.parametrize("kind", ["lu", "chol", "tri_lower", "tri_upper", "band"])
def test_estimator_lower_bound_and_quality(orc, kind):
    rng = np.random.default_rng({"lu": 1, "chol": 2, "tri_lower": 3, "tri_upper": 4, "band": 5}[kind])
    ratios = []
    for n in (2, 3, 10, 40, 100, 200):
        for _ in range(5):
            if kind == "lu":
                A = rng.standard_normal((n, n))
                Fm, ipiv, _ = orc.lu_factor(A)
                est = orc.est_inv_norm1_lu(Fm, ipiv)
            elif kind == "chol":
                G = rng.standard_normal((n, n))
                A = G.T @ G / n + 0.1 * np.eye(n)
                A = np.tril(A) + np.tril(A, -1).T
                Fm, _ = orc.chol_factor(A)
                est = orc.est_inv_norm1_chol(Fm)
            elif kind.startswith("tri"):
                lower = kind == "tri_lower"
                A = rng.standard_normal((n, n)) / np.sqrt(n)
                A = np.tril(A) if lower else np.triu(A)
                np.fill_diagonal(A, 1.0 + np.abs(rng.standard_normal(n)))
                est = orc.est_inv_norm1_tri(A, lower)
            else:
                kl, ku = min(2, n - 1), min(3, n - 1)
                A = np.zeros((n, n))
                for d in range(-kl, ku + 1):
                    A += np.diag(rng.standard_normal(n - abs(d)), d)
                Fm, ipiv, _ = orc.band_lu_factor(orc.band_pack(A, kl, ku), kl, ku)
                est = orc.est_inv_norm1_band(Fm, kl, ku, ipiv)
            true = inv_norm1(A)
            assert est <= true * (1 + 1e-10), (n, est, true)
            ratios.append(true / est)
    assert max(ratios) < 10.0 and np.median(ratios) < 1.5


def test_rcond_from_edge_cases(orc):
    assert orc.rcond_from(0.0, 5.0) == 0.0
    assert orc.rcond_from(2.0, np.inf) == 0.0
    assert orc.rcond_from(4.0, 0.5) == 0.5


def test_rcond_consistent_with_solve(orc):
    rng = np.random.default_rng(8)
    A = rng.standard_normal((60, 60))
    _, info = orc.solve(A, np.ones(60))
    true = 1.0 / (np.abs(A).sum(0).max() * inv_norm1(A))
    assert true * (1 - 1e-10) <= info["rcond"] <= 10 * true


# ------------------------------------------------------------------ SVD
def test_jacobi_svd_against_lapack(orc):
    rng = np.random.default_rng(31)
    for n in (1, 2, 5, 30, 64):
        A = rng.standard_normal((n, n))
        G, V, s, sweeps = orc.jacobi_svd(A)
        assert sweeps < 30
        ref = np.linalg.svd(A, compute_uv=False)
        assert np.allclose(np.sort(s)[::-1], ref, rtol=1e-13, atol=1e-14 * ref[0])
        assert np.abs(V.T @ V - np.eye(n)).max() < 1e-13 * max(n, 1)
        assert np.abs(G @ V.T - A).max() < 1e-13 * np.abs(A).max() * max(n, 1)
        U = G / np.where(s > 0, s, 1)[None, :]
        assert np.abs(U.T @ U - np.eye(n)).max() < 1e-12


def test_jacobi_svd_known_spectrum(orc):
    rng = np.random.default_rng(32)
    n = 40
    U, _ = np.linalg.qr(rng.standard_normal((n, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    sig = np.logspace(0, -6, n)
    A = (U * sig) @ V.T
    _, _, s, _ = orc.jacobi_svd(A)
    assert np.allclose(np.sort(s)[::-1], sig, rtol=0, atol=1e-14 * n)


def test_min_norm_solution_gapped(orc):
    """Rank-deficient A with a clean gap: the truncated SVD solve is the
    pseudo-inverse solution (within 1e-10 relative)."""
    rng = np.random.default_rng(33)
    n, k = 50, 6
    U, _ = np.linalg.qr(rng.standard_normal((n, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    sig = np.concatenate([np.logspace(0, -3, n - k), np.zeros(k)])
    A = (U * sig) @ V.T
    b = rng.standard_normal((n, 2))
    X, rank = orc.svd_solve(A, b)
    assert rank == n - k
    Xp = np.linalg.pinv(A, rcond=1e-10) @ b
    assert np.abs(X - Xp).max() <= 1e-10 * np.abs(Xp).max()
    # x lies in the row space; the residual is orthogonal to range(A)
    Vn = V[:, n - k:]
    assert np.abs(Vn.T @ X).max() < 1e-10 * np.abs(X).max()
    R = b - A @ X
    assert np.abs(A.T @ R).max() < 1e-10 * np.abs(A).max() * np.abs(R).max()


def test_svd_solve_full_rank_equals_lu(orc):
    rng = np.random.default_rng(34)
    A = rng.standard_normal((20, 20)) + 5 * np.eye(20)
    b = rng.standard_normal(20)
    Xs, rank = orc.svd_solve(A, b)
    Xl, info = orc.solve(A, b)
    assert rank == 20 and np.abs(Xs - Xl).max() < 1e-12 * np.abs(Xl).max()
    Xf, inf2 = orc.solve(A, b, flags=orc.FORCE_SVD)
    assert inf2["route"] == 7 and inf2["status"] == 1
    assert np.abs(Xf - Xs).max() == 0.0


def test_svd_truncation_threshold(orc):
    A = np.diag([1.0, 1e-3, 1e-9, 0.0])
    b = np.ones(4)
    X, rank = orc.svd_solve(A, b, trunc_rel=1e-6)
    assert rank == 2 and np.allclose(X[:, 0], [1.0, 1e3, 0.0, 0.0], rtol=1e-14)
    X, rank = orc.svd_solve(A, b)  # default n*eps keeps 1e-9
    assert rank == 3 and X[2, 0] == pytest.approx(1e9, rel=1e-14)


# -------------------------------------------------------------- residual
def test_dot2_residual_exact(orc):
    rng = np.random.default_rng(35)
    n = 24
    A = rng.standard_normal((n, n))
    x = np.linalg.solve(A, rng.standard_normal(n))
    b = A @ x  # residual is tiny: cancellation everywhere
    R, berr = orc.residual_dot2(A, x, b)
    for i in range(n):
        exact = Fraction(float(b[i])) - sum(Fraction(float(A[i, j])) * Fraction(float(x[j]))
                                            for j in range(n))
        mag = sum(abs(A[i, j] * x[j]) for j in range(n))
        assert abs(R[i, 0] - float(exact)) <= 2 * EPS * abs(float(exact)) + 2 * n * n * EPS * EPS * mag
    assert berr[0] == pytest.approx(np.abs(R).max() / (np.abs(A).sum(1).max() * np.abs(x).max()
                                                       + np.abs(b).max()), rel=1e-14)
