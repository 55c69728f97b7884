"""GPU parity of the symmetric-indefinite route (ASOLVE_SYM_INDEF; the
paper names plain symmetric matrices for specialised handling) against
the oracle run with its SYM_INDEF flag, on the batched path (n <= 1024).

* Symmetric indefinite systems of several sizes (tiles and ragged tails),
  zero diagonals that force 2 x 2 pivots, and Fig. 4-passing matrices
  whose Cholesky fails: class, route (9 or 10) and status equal to the
  oracle's; X within the forward-error bound of the oracle's X; the
  estimate of ||inv(A)||_1 within 1e-10 of the oracle's (the same
  factors: the GPU rounds every operation as the oracle does), rcond
  within the scan's norm accuracy; backward error <= 1e-13.
* Without the flag, non-symmetric matrices and FORCE_LU: the routes of
  Sec. 2.  A zero column: the SVD fallback.  More than 8 right-hand sides
  at n <= 1024: E_UNSUPPORTED.
"""
import numpy as np
import pytest
import torch

from gpu_util import EPS, dev_colmajor, kappa_inf, pack_batch, run_batch, solve_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2007_11208_gb300 import asolve, build
    build.build()
    c = asolve.Context(precision=asolve.PREC_MIXED)
    yield c
    c.close()


def sym(n, rng, zero_diag=False):
    G = rng.standard_normal((n, n))
    A = G + G.T
    if zero_diag:
        A[np.diag_indices(n)] = 0.0
    return A


def check(orc, ctx, A, B, X, info):
    Xo, io = orc.solve(A, B, flags=orc.SYM_INDEF)
    assert (info["cls"], info["route"], info["status"]) == (io["cls"], io["route"], io["status"]), (info, io)
    assert io["status"] == 0
    n = A.shape[0]
    assert np.abs(X - Xo).max() / np.abs(Xo).max() <= 2.0 ** -52 * n * kappa_inf(A)
    norm1_gpu = ctx.scan(dev_colmajor(A), n)["norm1"]
    est_g = 1.0 / (info["rcond"] * norm1_gpu)
    est_o = 1.0 / (io["rcond"] * np.abs(A).sum(axis=0).max())
    assert abs(est_g - est_o) <= 1e-10 * est_o, (est_g, est_o)
    _, berr = orc.residual_dot2(A, X, B)
    assert berr.max() <= 1e-13, berr


def test_batched_ldlt_routes(ctx, orc):
    from paper_2007_11208_gb300 import asolve
    rng = np.random.default_rng(31)
    mats = [sym(n, rng, zero_diag=(k % 3 == 1)) for k, n in enumerate((2, 5, 31, 33, 100, 257, 600, 1024))]
    mats.append(np.array([[1, .9, .9], [.9, 1, -.9], [.9, -.9, 1]]))  # Fig. 4 passes, Cholesky fails
    rhs = [rng.standard_normal((A.shape[0], 1 + k % 4)) for k, A in enumerate(mats)]
    pk = pack_batch(mats, rhs)
    Xs, infos = run_batch(ctx, pk, asolve.SYM_INDEF | asolve.BERR)
    for A, B, X, i in zip(mats, rhs, Xs, infos):
        check(orc, ctx, A, B, X, i)
        assert i["route"] in (asolve.ROUTE_LDLT, asolve.ROUTE_CHOL_FAIL_LDLT), i
        assert i["berr"] <= 1e-13, i
    _, infos = run_batch(ctx, pk)
    assert all(i["route"] in (asolve.ROUTE_LU, asolve.ROUTE_CHOL_FAIL_LU) for i in infos), infos


def test_single_ldlt_and_other_routes(ctx, orc):
    from paper_2007_11208_gb300 import asolve
    rng = np.random.default_rng(32)
    A = sym(300, rng)
    B = rng.standard_normal((300, 2))
    rc, info, X = solve_gpu(ctx, A, B, asolve.SYM_INDEF)
    check(orc, ctx, A, B, X, info)
    rc, info, X = solve_gpu(ctx, A, B, asolve.SYM_INDEF | asolve.FORCE_LU)
    assert info["route"] == asolve.ROUTE_LU
    Z = A.copy()
    Z[3, 7] += 1e-9
    rc, info, X = solve_gpu(ctx, Z, B, asolve.SYM_INDEF)
    assert info["route"] == asolve.ROUTE_LU
    S = A.copy()
    S[:, 11] = 0.0
    S[11, :] = 0.0
    rc, info, X = solve_gpu(ctx, S, B, asolve.SYM_INDEF)
    Xo, io = orc.solve(S, B, flags=orc.SYM_INDEF)
    assert (rc, info["route"], info["svd_rank"]) == (io["status"], io["route"], io["svd_rank"]) == \
        (asolve.W_APPROX, asolve.ROUTE_LDLT, 299), (info, io)
    assert np.abs(X - Xo).max() <= 1e-10 * np.abs(Xo).max()


def test_many_rhs_unsupported(ctx):
    from paper_2007_11208_gb300 import asolve
    n = 200
    dA = torch.eye(n, dtype=torch.float64, device="cuda")
    dB = torch.ones(9 * n, dtype=torch.float64, device="cuda")
    dX = torch.zeros_like(dB)
    rc, info = ctx.solve(dA, dB, n, 9, dX, asolve.SYM_INDEF)
    assert rc == asolve.E_UNSUPPORTED
