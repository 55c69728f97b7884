"""GPU SVD fallback for one large system (Sec. 2.5; n > 1024, the whole-GPU
one-sided Jacobi of svd_large.cu).

* n = 1100 (a ragged 32-row tail), gapped spectrum (kept singular values in
  [1e-3, 1], three at 1e-20): the routed LU's rcond falls below the
  threshold and the SVD answers.  Against the oracle: class, route, status
  W_APPROX and kept rank equal, X within 1e-10 relative.  Also FORCE_SVD.
* A lower-triangular n = 1100 system with an exact zero on the diagonal:
  the substitution fails (Sec. 2.2) and the SVD answers, as in the oracle.
* n = 2048, gapped spectrum: rank and X against LAPACK's xGELSD with the
  same cut-off (the oracle's Jacobi needs about a minute there).
* n = 4096 with a zero column: W_APPROX, rank n - 1, the minimum-norm
  property (no component along the null vector e_j) and the least-squares
  property (A^T (b - A x) = 0 to rounding); with NO_APPROX, E_SINGULAR and
  X zeroed.
* FORCE_SVD above the fallback's limit (n = 8200): E_UNSUPPORTED.
"""
import numpy as np
import pytest
import torch

from gpu_util import dev_colmajor, dev_rhs, host_from_dev

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps
SVD_RTOL = 1e-10


@pytest.fixture(scope="module")
def ctx():
    from paper_2007_11208_gb300 import asolve, build
    build.build()
    c = asolve.Context(precision=asolve.PREC_FP64)
    yield c
    c.close()


def gapped(n, k, lo, seed):
    """U diag(s) V^T, s = logspace(0, lo, n - k) then k values 1e-20."""
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((n, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    s = np.concatenate([np.logspace(0, lo, n - k), np.full(k, 1e-20)])
    return (U * s) @ V.T, rng


def solve(ctx, A, B, flags=0):
    n = A.shape[0]
    dA = dev_colmajor(A)
    dB, nrhs = dev_rhs(B, n)
    dX = torch.zeros_like(dB)
    rc, info = ctx.solve(dA, dB, n, nrhs, dX, flags)
    return rc, info, host_from_dev(dX, n, nrhs)


def rel(X, Xr):
    return np.abs(X - Xr).max() / np.abs(Xr).max()


def test_gapped_1100_against_oracle(ctx, orc):
    from paper_2007_11208_gb300 import asolve
    A, rng = gapped(1100, 3, -3, 11)
    B = rng.standard_normal((1100, 2))
    Xo, io = orc.solve(A, B)
    assert io["status"] == orc.W_APPROX and io["route"] == orc.ROUTE_LU, io
    rc, info, X = solve(ctx, A, B, asolve.BERR)
    assert (rc, info["cls"], info["route"], info["svd_rank"]) == \
        (io["status"], io["cls"], io["route"], io["svd_rank"]), (info, io)
    assert rel(X, Xo) <= SVD_RTOL, rel(X, Xo)
    assert info["berr"] == info["berr"]  # reported
    # FORCE_SVD: the same SVD, reported on the SVD route (as the oracle does)
    rc, info, X = solve(ctx, A, B, asolve.FORCE_SVD)
    assert (rc, info["route"], info["svd_rank"]) == (asolve.W_APPROX, asolve.ROUTE_SVD, io["svd_rank"]), info
    assert rel(X, Xo) <= SVD_RTOL


def test_triangular_zero_diagonal_1100(ctx, orc):
    from paper_2007_11208_gb300 import asolve
    n = 1100
    rng = np.random.default_rng(12)
    A = np.tril(rng.standard_normal((n, n)), -1) / np.sqrt(n)
    A[np.diag_indices(n)] = 1.0 + rng.random(n)
    A[700, 700] = 0.0
    B = rng.standard_normal((n, 1))
    Xo, io = orc.solve(A, B)
    assert io["status"] == orc.W_APPROX and io["route"] == orc.ROUTE_TRI_LOWER, io
    rc, info, X = solve(ctx, A, B)
    assert (rc, info["cls"], info["route"], info["svd_rank"]) == \
        (io["status"], io["cls"], io["route"], io["svd_rank"]), (info, io)
    assert rel(X, Xo) <= SVD_RTOL, rel(X, Xo)
    rc, info, X = solve(ctx, A, B, asolve.NO_APPROX)
    assert rc == asolve.E_SINGULAR and np.all(X == 0.0)


def test_gapped_2048_against_gelsd(ctx):
    linalg = pytest.importorskip("scipy.linalg")
    from paper_2007_11208_gb300 import asolve
    n = 2048
    A, rng = gapped(n, 5, -3, 13)
    B = rng.standard_normal((n, 3))
    rc, info, X = solve(ctx, A, B)
    assert rc == asolve.W_APPROX and info["route"] == asolve.ROUTE_LU, info
    Xg, _, rank, _ = linalg.lstsq(A, B, cond=n * EPS, lapack_driver="gelsd")
    assert info["svd_rank"] == rank == n - 5
    assert rel(X, Xg) <= SVD_RTOL, rel(X, Xg)


def test_zero_column_4096(ctx):
    from paper_2007_11208_gb300 import asolve
    n, j = 4096, 1234
    rng = np.random.default_rng(14)
    A = rng.standard_normal((n, n)) + 2.0 * np.sqrt(n) * np.eye(n)
    A[:, j] = 0.0
    B = rng.standard_normal((n, 1))
    rc, info, X = solve(ctx, A, B, asolve.BERR)
    assert rc == asolve.W_APPROX and info["route"] == asolve.ROUTE_LU, info
    assert info["svd_rank"] == n - 1
    x = X[:, 0]
    assert abs(x[j]) <= 1e-12 * np.abs(x).max()           # minimum norm: no null-space part
    r = B[:, 0] - A @ x
    normal = np.abs(A.T @ r).max()                         # least squares: A^T r = 0
    assert normal <= 1e-10 * np.abs(A).sum(axis=0).max() ** 2 * np.abs(x).max()
    rc, info, X = solve(ctx, A, B, asolve.NO_APPROX)
    assert rc == asolve.E_SINGULAR and np.all(X == 0.0)


def test_force_svd_above_the_limit(ctx):
    from paper_2007_11208_gb300 import asolve
    n = 8200
    dA = torch.eye(n, dtype=torch.float64, device="cuda")
    dB = torch.ones(n, dtype=torch.float64, device="cuda")
    dX = torch.zeros_like(dB)
    rc, info = ctx.solve(dA, dB, n, 1, dX, asolve.FORCE_SVD)
    assert rc == asolve.E_UNSUPPORTED, info
