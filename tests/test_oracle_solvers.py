"""Pins for the oracle's solvers (paper Sec. 2.1-2.5, Eq. 3, Eq. 4).

Expected values come from exact rational arithmetic (Cramer's rule, exact
Gaussian elimination over the rationals), closed-form inverses (Hilbert,
tridiagonal Toeplitz), factorisation invariants, an independent library SVD
(numpy), and systems built from a known x -- never from the oracle.
"""
from fractions import Fraction
from math import comb

import numpy as np
import pytest

EPS = np.finfo(np.float64).eps


def F(x):
    return Fraction(float(x))


def det_frac(M):
    """Exact determinant by fraction-valued elimination."""
    M = [[Fraction(v) for v in row] for row in M]
    n, det = len(M), Fraction(1)
    for k in range(n):
        p = next((i for i in range(k, n) if M[i][k] != 0), None)
        if p is None:
            return Fraction(0)
        if p != k:
            M[k], M[p] = M[p], M[k]
            det = -det
        det *= M[k][k]
        for i in range(k + 1, n):
            f = M[i][k] / M[k][k]
            for j in range(k, n):
                M[i][j] -= f * M[k][j]
    return det


def cramer(A, b):
    n = len(A)
    d = det_frac(A)
    xs = []
    for i in range(n):
        Ai = [[(b[r] if c == i else A[r][c]) for c in range(n)] for r in range(n)]
        xs.append(det_frac(Ai) / d)
    return xs


def exact_solve(A, b):
    """Exact solution of A x = b over the rationals (A, b given as floats)."""
    n = A.shape[0]
    M = [[F(A[i, j]) for j in range(n)] + [F(b[i])] for i in range(n)]
    for k in range(n):
        p = next(i for i in range(k, n) if M[i][k] != 0)
        M[k], M[p] = M[p], M[k]
        for i in range(n):
            if i != k and M[i][k] != 0:
                f = M[i][k] / M[k][k]
                M[i] = [a - f * c for a, c in zip(M[i], M[k])]
    return np.array([float(M[i][n] / M[i][i]) for i in range(n)])


def kappa_inf(A):
    return np.linalg.norm(A, np.inf) * np.linalg.norm(np.linalg.inv(A), np.inf)


def fwd_ok(x, xe, A, c=8.0):
    n = A.shape[0]
    bound = c * n * kappa_inf(A) * EPS * max(np.abs(xe).max(), 1e-300)
    return np.abs(x - xe).max() <= bound


# ---------------------------------------------------------------- Cramer
@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_cramer_general(orc, n):
    rng = np.random.default_rng(7 * n)
    done = 0
    while done < 40:
        A = rng.integers(-5, 6, size=(n, n)).astype(np.float64)
        b = rng.integers(-9, 10, size=n).astype(np.float64)
        if det_frac(A.tolist()) == 0:
            continue
        xe = np.array([float(v) for v in cramer(A.tolist(), b.tolist())])
        X, info = orc.solve(A, b)
        assert info["status"] >= 0
        assert fwd_ok(X[:, 0], xe, A), (A, b, X[:, 0], xe, info)
        done += 1


@pytest.mark.parametrize("lower", [True, False])
def test_cramer_triangular(orc, lower):
    rng = np.random.default_rng(11 + lower)
    for n in (2, 3, 4):
        for _ in range(20):
            A = rng.integers(-5, 6, size=(n, n)).astype(np.float64)
            A = np.tril(A) if lower else np.triu(A)
            d = rng.integers(1, 6, size=n) * rng.choice([-1, 1], size=n)
            np.fill_diagonal(A, d)
            b = rng.integers(-9, 10, size=n).astype(np.float64)
            xe = np.array([float(v) for v in cramer(A.tolist(), b.tolist())])
            X, info = orc.solve(A, b)
            diag_only = not np.any(A - np.diag(np.diag(A)))
            assert info["route"] == (2 if (lower or diag_only) else 3)
            assert fwd_ok(X[:, 0], xe, A)
            Y, inf2 = orc.tri_solve(A, b, lower)
            assert inf2 == 0 and fwd_ok(Y[:, 0], xe, A)
            Z, _ = orc.tri_solve(A, b, lower, trans=True)  # A^T z = b
            ze = np.array([float(v) for v in cramer(A.T.tolist(), b.tolist())])
            assert fwd_ok(Z[:, 0], ze, A.T)


def test_exact_rational_all_routes(orc):
    """Integer systems of every class, against exact rational solutions."""
    rng = np.random.default_rng(5)
    seen = set()
    for trial in range(60):
        n = int(rng.integers(5, 17))
        kind = trial % 5
        if kind == 0:  # general
            A = rng.integers(-6, 7, size=(n, n)).astype(np.float64)
        elif kind == 1:  # sympd integer: G^T G + n I
            G = rng.integers(-2, 3, size=(n, n)).astype(np.float64)
            A = G.T @ G + 2 * n * np.eye(n)
        elif kind == 2:  # banded with pivoting needed (kl=2, ku=1), n >= 12
            n = max(n, 14)
            A = np.zeros((n, n))
            for d in (-2, -1, 0, 1):
                A += np.diag(rng.integers(-9, 10, size=n - abs(d)).astype(np.float64), d)
        elif kind == 3:
            A = np.tril(rng.integers(-4, 5, size=(n, n))).astype(np.float64)
            np.fill_diagonal(A, rng.integers(1, 4, size=n))
        else:
            A = np.triu(rng.integers(-4, 5, size=(n, n))).astype(np.float64)
            np.fill_diagonal(A, -rng.integers(1, 4, size=n))
        if abs(np.linalg.det(A)) < 0.5:
            continue
        b = rng.integers(-20, 21, size=n).astype(np.float64)
        xe = exact_solve(A, b)
        X, info = orc.solve(A, b)
        assert info["status"] == 0, info
        seen.add(info["route"])
        assert fwd_ok(X[:, 0], xe, A), (trial, info)
    assert {1, 2, 3, 4, 6} <= seen, seen


# ---------------------------------------------------------------- Hilbert
def hilbert_scaled(n):
    """L*H with L = lcm(1..2n-1): integer entries, exact in FP64."""
    from math import lcm
    L = 1
    for k in range(1, 2 * n):
        L = lcm(L, k)
    H = np.array([[L // (i + j + 1) for j in range(n)] for i in range(n)], dtype=np.float64)
    return H, L


def hilbert_inverse(n):
    """Closed-form integer inverse of the n x n Hilbert matrix (1-based i,j):
    (-1)^(i+j) (i+j-1) C(n+i-1, n-j) C(n+j-1, n-i) C(i+j-2, i-1)^2."""
    return [[(-1) ** (i + j) * (i + j - 1) * comb(n + i - 1, n - j) * comb(n + j - 1, n - i)
             * comb(i + j - 2, i - 1) ** 2 for j in range(1, n + 1)] for i in range(1, n + 1)]


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7, 8])
def test_hilbert_closed_form(orc, n):
    H, L = hilbert_scaled(n)
    Hinv = hilbert_inverse(n)
    # the closed form really is the inverse of the (unscaled) Hilbert matrix
    for i in range(n):
        for j in range(n):
            s = sum(Fraction(1, i + k + 1) * Hinv[k][j] for k in range(n))
            assert s == (1 if i == j else 0)
    b = np.arange(1, n + 1, dtype=np.float64)
    # x = (L H)^-1 b = H^-1 b / L, exactly
    xe = np.array([float(sum(Fraction(Hinv[i][k]) * int(b[k]) for k in range(n)) / L)
                   for i in range(n)])
    X, info = orc.solve(H, b)
    assert info["cls"] == 4 and info["route"] == 4 and info["status"] == 0
    assert fwd_ok(X[:, 0], xe, H)


def test_hilbert_ill_conditioned_routes_to_svd(orc):
    n = 12
    H = np.array([[1.0 / (i + j + 1) for j in range(n)] for i in range(n)])
    # true rcond_1 is far below 0.5*eps (Hilbert n=12: kappa_1 ~ 4e16)
    Hinv = np.array(hilbert_inverse(n), dtype=np.float64)
    assert 1.0 / (np.abs(H).sum(0).max() * np.abs(Hinv).sum(0).max()) < 0.25 * EPS
    X, info = orc.solve(H, np.ones(n))
    assert info["status"] == 1 and info["svd_used"] == 1


# ------------------------------------------------------ tridiagonal Toeplitz
def cheb_u(k, x):
    u0, u1 = Fraction(1), 2 * x
    if k == 0:
        return u0
    for _ in range(k - 1):
        u0, u1 = u1, 2 * x * u1 - u0
    return u1


def toeplitz_tridiag_inverse(n, a, b):
    """(T^-1)_ij = (-1)^(i+j) U_{i-1}(x) U_{n-j}(x) / (b U_n(x)), i <= j
    (1-based), x = a/(2b); symmetric."""
    x = Fraction(a, 2 * b)
    Un = cheb_u(n, x)
    inv = [[Fraction(0)] * n for _ in range(n)]
    for i in range(1, n + 1):
        for j in range(i, n + 1):
            v = (-1) ** (i + j) * cheb_u(i - 1, x) * cheb_u(n - j, x) / (b * Un)
            inv[i - 1][j - 1] = inv[j - 1][i - 1] = v
    return inv


@pytest.mark.parametrize("n,a,b", [(2, 4, 1), (3, 4, 1), (12, 4, 1), (16, 4, 1), (40, 3, -1),
                                   (64, 5, 2)])
def test_tridiagonal_toeplitz_closed_form(orc, n, a, b):
    T = a * np.eye(n) + b * (np.eye(n, k=1) + np.eye(n, k=-1))
    inv = toeplitz_tridiag_inverse(n, a, b)
    if n <= 16:  # closed form agrees with exact elimination
        rhs = [Fraction(k + 1) for k in range(n)]
        xe_closed = [sum(inv[i][k] * rhs[k] for k in range(n)) for i in range(n)]
        assert np.allclose(exact_solve(T, np.arange(1.0, n + 1)),
                           [float(v) for v in xe_closed], rtol=1e-15, atol=0)
    rng = np.random.default_rng(n)
    bb = rng.integers(-5, 6, size=n).astype(np.float64)
    xe = np.array([float(sum(inv[i][k] * int(bb[k]) for k in range(n))) for i in range(n)])
    X, info = orc.solve(T, bb)
    assert info["route"] == (1 if n >= 12 else 4 if a > 0 and abs(2 * b) < a else info["route"])
    assert info["kl"] == 1 and info["ku"] == 1
    assert fwd_ok(X[:, 0], xe, T)
    # the estimate never exceeds the true ||T^-1||_1
    true_inv1 = max(sum(abs(inv[i][j]) for i in range(n)) for j in range(n))
    assert info["rcond"] >= 1.0 / (np.abs(T).sum(0).max() * float(true_inv1)) * (1 - 1e-12)


# ---------------------------------------------------------- invariants
def test_lu_invariant(orc):
    rng = np.random.default_rng(3)
    for n in (1, 2, 5, 33, 120):
        A = rng.standard_normal((n, n))
        Fm, ipiv, info = orc.lu_factor(A)
        assert info == 0
        L = np.tril(Fm, -1) + np.eye(n)
        U = np.triu(Fm)
        PA = A.copy()
        for k in range(n):
            PA[[k, ipiv[k]]] = PA[[ipiv[k], k]]
        bound = 2 * n * EPS * (np.abs(L) @ np.abs(U)).max()
        assert np.abs(PA - L @ U).max() <= bound
        # partial pivoting: |l_ij| <= 1, first index of the max
        assert np.abs(L).max() <= 1.0
    # pivot = first index among ties (IDAMAX convention)
    A = np.array([[1.0, 2.0], [-1.0, 3.0]])
    _, ipiv, _ = orc.lu_factor(A)
    assert ipiv[0] == 0


def test_cholesky_invariant(orc):
    rng = np.random.default_rng(4)
    for n in (1, 3, 40, 150):
        G = rng.standard_normal((n, n))
        A = G.T @ G / n + np.eye(n)
        A = np.tril(A) + np.tril(A, -1).T
        Lf, info = orc.chol_factor(A)
        assert info == 0
        L = np.tril(Lf)
        assert np.abs(L @ L.T - A).max() <= 4 * n * EPS * (np.abs(L) @ np.abs(L.T)).max()
        assert np.all(np.diag(L) > 0)


def test_cholesky_failure_reports_step(orc):
    A = np.array([[4.0, 2, 0], [2, 1, 0], [0, 0, 1]])  # second pivot exactly 0
    _, info = orc.chol_factor(A)
    assert info == 2


def test_band_lu_matches_dense_and_reconstructs(orc):
    rng = np.random.default_rng(9)
    for (n, kl, ku) in ((1, 0, 0), (5, 1, 2), (30, 2, 1), (60, 3, 3), (80, 0, 4), (80, 4, 0)):
        A = np.zeros((n, n))
        for d in range(-kl, ku + 1):
            A += np.diag(rng.standard_normal(n - abs(d)), d)
        AB = orc.band_pack(A, kl, ku)
        # packing places A(i,j) at row kl+ku+i-j
        for j in range(n):
            for i in range(max(0, j - ku), min(n, j + kl + 1)):
                assert AB[kl + ku + i - j, j] == A[i, j]
        Fb, ipb, infob = orc.band_lu_factor(AB, kl, ku)
        assert infob == 0
        b = rng.standard_normal((n, 3))
        Xb = orc.band_lu_solve(Fb, kl, ku, ipb, b)
        Xt = orc.band_lu_solve(Fb, kl, ku, ipb, b, trans=True)
        xe = np.linalg.solve(A, b)
        xte = np.linalg.solve(A.T, b)
        k = kappa_inf(A)
        assert np.abs(Xb - xe).max() <= 8 * n * k * EPS * np.abs(xe).max()
        assert np.abs(Xt - xte).max() <= 8 * n * k * EPS * np.abs(xte).max()
        # same pivot sequence as dense partial pivoting
        _, ipd, _ = orc.lu_factor(A)
        assert np.array_equal(ipb, ipd)


def test_lu_transposed_solve(orc):
    rng = np.random.default_rng(12)
    A = rng.standard_normal((25, 25))
    Fm, ipiv, _ = orc.lu_factor(A)
    b = rng.standard_normal(25)
    x = orc.lu_solve(Fm, ipiv, b, trans=True)[:, 0]
    assert np.abs(A.T @ x - b).max() <= 1e-12 * np.abs(b).max() * kappa_inf(A)


def test_known_x_systems(orc):
    """b = A x_true in exact integer arithmetic; every route recovers x_true."""
    rng = np.random.default_rng(21)
    for kind in ("general", "spd", "lower", "upper", "band"):
        n = 48
        if kind == "general":
            A = rng.integers(-8, 9, size=(n, n)).astype(np.float64)
        elif kind == "spd":
            G = rng.integers(-3, 4, size=(n, n)).astype(np.float64)
            A = G.T @ G + 4 * n * np.eye(n)
        elif kind == "lower":
            A = np.tril(rng.integers(-3, 4, size=(n, n))).astype(np.float64)
            np.fill_diagonal(A, 40.0)
        elif kind == "upper":
            A = np.triu(rng.integers(-3, 4, size=(n, n))).astype(np.float64)
            np.fill_diagonal(A, -40.0)
        else:
            A = np.zeros((n, n))
            for d in (-3, -1, 0, 2):
                A += np.diag(rng.integers(-9, 10, size=n - abs(d)).astype(np.float64), d)
            np.fill_diagonal(A, 30.0)
        xt = rng.integers(-50, 51, size=(n, 2)).astype(np.float64)
        b = A @ xt  # exact: small integers
        X, info = orc.solve(A, b)
        assert info["status"] == 0
        assert np.abs(X - xt).max() <= 8 * n * kappa_inf(A) * EPS * np.abs(xt).max(), kind


# ---------------------------------------------------------- special routes
def test_special_routes(orc):
    # indefinite matrix passing Fig. 4: eigenvalues {-0.8, 1.9, 1.9}
    A = np.array([[1, .9, .9], [.9, 1, -.9], [.9, -.9, 1]])
    assert np.linalg.eigvalsh(A).min() < 0
    X, info = orc.solve(A, np.ones(3))
    assert info["cls"] == 4 and info["route"] == 5 and info["status"] == 0
    assert np.abs(A @ X[:, 0] - 1).max() < 1e-14
    # zero matrix, n >= 4: banded (kl=ku=0) -> singular -> SVD, x = 0, rank 0
    X, info = orc.solve(np.zeros((5, 5)), np.ones(5))
    assert info["cls"] == 1 and info["route"] == 1 and info["status"] == 1
    assert info["svd_rank"] == 0 and np.all(X == 0)
    # general matrix with a zero column: exact zero pivot -> SVD
    rng = np.random.default_rng(2)
    A = rng.standard_normal((30, 30))
    A[:, 7] = 0.0
    X, info = orc.solve(A, rng.standard_normal(30))
    assert info["route"] == 6 and info["svd_used"] == 1 and info["svd_rank"] == 29
    # NO_APPROX: singular -> E_SINGULAR with X zeroed
    X, info = orc.solve(A, np.ones(30), flags=orc.NO_APPROX)
    assert info["status"] == orc.E_SINGULAR and np.all(X == 0)
    # singular triangular (zero on the diagonal)
    T = np.tril(np.ones((6, 6)))
    T[3, 3] = 0.0
    X, info = orc.solve(T, np.ones(6))
    assert info["route"] == 2 and info["svd_used"] == 1
    # non-finite input
    B = np.eye(4)
    B[1, 2] = np.inf
    _, info = orc.solve(B, np.ones(4))
    assert info["status"] == orc.E_NONFINITE
    _, info = orc.solve(np.eye(4), np.array([1, np.nan, 0, 0]))
    assert info["status"] == orc.E_NONFINITE
    # n = 0
    X, info = orc.solve(np.zeros((0, 0)), np.zeros(0))
    assert info["status"] == 0 and info["route"] == 0
    # FORCE_LU on a triangular matrix: class still reported, route LU
    X, info = orc.solve(np.tril(np.ones((6, 6))) + 5 * np.eye(6), np.ones(6), flags=orc.FORCE_LU)
    assert info["cls"] == 2 and info["route"] == 6
    # a raised threshold sends a well-posed but graded system to the SVD
    A = np.diag(np.logspace(0, -10, 8)) + np.eye(8, k=1) * 1e-3
    _, info = orc.solve(A, np.ones(8), cfg=orc.config(rcond_threshold=1e-6))
    assert info["svd_used"] == 1
    _, info = orc.solve(A, np.ones(8), cfg=orc.config(rcond_threshold=1e-6), flags=orc.NO_APPROX)
    assert info["status"] == orc.W_ILLCOND


def test_threshold_is_strict(orc):
    """rcond exactly at the threshold is not 'below' it (Sec. 2.5)."""
    A = np.diag([1.0, 2.0, 4.0, 8.0])  # banded; estimator exact on diagonals
    X, info = orc.solve(A, np.ones(4))
    r = info["rcond"]
    assert r == pytest.approx(1.0 / 8.0, rel=0, abs=0)  # (1/1)/8 exactly
    _, info = orc.solve(A, np.ones(4), cfg=orc.config(rcond_threshold=r))
    assert info["status"] == 0
    _, info = orc.solve(A, np.ones(4), cfg=orc.config(rcond_threshold=np.nextafter(r, 1)))
    assert info["svd_used"] == 1
