"""GPU parity of the tridiagonal route (ASOLVE_TRIDIAG; the paper names
tridiagonal matrices, a common subtype of banded ones, for specialised
handling) against the oracle run with its TRIDIAG flag.

* Batched (n <= 1024, the band kernel with kl = ku = 1, whose pivots and
  operations are xGTTRF's) and the large dense path (n = 2048, the
  elimination): route 8, class and bandwidths as the oracle's; without the
  flag the band route.
* Band storage, long systems: strictly dominant ones (n = 4096 to 10^6) by
  the partitioned route (detail bit 4), weakly dominant and non-dominant
  ones by the elimination; X within the forward-error bound of the
  oracle's X (kappa from the oracle's rcond), rcond within 1e-5 relative,
  backward error <= 1e-13.
* An exact zero pivot: the SVD fallback (W_APPROX, rank n - 1).
"""
import numpy as np
import pytest

from gpu_util import EPS, pack_batch, run_batch, solve_gpu
from test_gpu_band import band_storage, solve_band_gpu, to_dense

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2007_11208_gb300 import asolve, build
    build.build()
    c = asolve.Context(precision=asolve.PREC_FP64)
    yield c
    c.close()


def tri_dense(n, rng, dominant=False):
    dl, d, du = rng.standard_normal(n - 1), rng.standard_normal(n), rng.standard_normal(n - 1)
    if dominant:
        d = np.sign(d + 0.25) * (1.0 + np.abs(np.r_[dl, 0]) + np.abs(np.r_[0, du]))
    else:
        d = d + np.where(d < 0, -0.5, 0.5)
    return np.diag(d) + np.diag(dl, -1) + np.diag(du, 1)


def check(orc, A, B, rc, info, X, Xo, io):
    n = A.shape[0]
    assert (info["cls"], info["route"], info["kl"], info["ku"]) == (io["cls"], io["route"], io["kl"], io["ku"]), \
        (info, io)
    assert rc == io["status"] == 0, (rc, info, io)
    kappa = n / io["rcond"]
    assert np.abs(X - Xo).max() / np.abs(Xo).max() <= EPS * n * kappa
    assert abs(info["rcond"] - io["rcond"]) <= 1e-5 * io["rcond"], (info["rcond"], io["rcond"])


def test_batched_tridiag_route(ctx, orc):
    from paper_2007_11208_gb300 import asolve
    rng = np.random.default_rng(21)
    mats = [tri_dense(n, rng, dominant=(k % 2 == 0)) for k, n in enumerate((12, 13, 50, 300, 777, 1024))]
    rhs = [rng.standard_normal((A.shape[0], 1 + k % 3)) for k, A in enumerate(mats)]
    pk = pack_batch(mats, rhs)
    Xs, infos = run_batch(ctx, pk, asolve.TRIDIAG)
    for A, B, X, i in zip(mats, rhs, Xs, infos):
        Xo, io = orc.solve(A, B, flags=orc.TRIDIAG)
        assert io["route"] == orc.ROUTE_TRIDIAG
        check(orc, A, B, i["status"], i, X, Xo, io)
    _, infos = run_batch(ctx, pk)
    assert all(i["route"] == asolve.ROUTE_BAND_LU for i in infos), infos


def test_large_dense_tridiag(ctx, orc):
    from paper_2007_11208_gb300 import asolve
    rng = np.random.default_rng(22)
    A = tri_dense(2048, rng)
    B = rng.standard_normal((2048, 2))
    rc, info, X = solve_gpu(ctx, A, B, asolve.TRIDIAG)
    Xo, io = orc.solve(A, B, flags=orc.TRIDIAG)
    check(orc, A, B, rc, info, X, Xo, io)
    assert not info["detail"] & 64  # below the cyclic reduction's minimum order


@pytest.mark.parametrize("n,kind,nrhs", [(100000, "dominant", 1), (100000, "laplace", 5), (1000000, "dominant", 2),
                                         (300000, "laplace", 1), (20000, "none", 1), (4096, "dominant", 1)])
def test_band_storage_tridiag(ctx, orc, n, kind, nrhs):
    """Strictly dominant: the partitioned route (detail bit 4); weakly
    dominant symmetric M-matrices (off-diagonals -U(0.5, 1.5), |d_i| =
    |dl_i| + |du_i| in every row but the first and the last, like a 1-D
    Laplacian), whose spikes do not decay, and non-dominant ones: the
    elimination with xGTTRF's pivots (bit 4 clear)."""
    from paper_2007_11208_gb300 import asolve
    rng = np.random.default_rng(n + nrhs)
    AB, kld, kud = band_storage(n, 1, 1, rng, dominant=(kind != "none"), extra=(1, 0))
    if kind == "none":  # diagonal N(0,1) + 1/2 away from zero: interchanges, no dominance
        AB[kud, :] += np.where(AB[kud, :] < 0, -0.5, 0.5)
    if kind == "laplace":  # symmetric, equality in every row but the first and the last
        u = rng.uniform(0.5, 1.5, size=n - 1)
        AB[:, :] = 0.0
        AB[kud + 1, :n - 1] = -u           # A(i+1, i)
        AB[kud - 1, 1:] = -u               # A(i, i+1)
        d = np.zeros(n)
        d[:-1] += u
        d[1:] += u
        d[0] += 1.0
        d[-1] += 1.0
        AB[kud, :] = d
    B = rng.standard_normal((n, nrhs))
    rc, info, X = solve_band_gpu(ctx, AB, kld, kud, B, asolve.TRIDIAG | asolve.BERR)
    Xo, io = orc.solve_band(AB, kld, kud, B, flags=orc.TRIDIAG)
    assert io["route"] == orc.ROUTE_TRIDIAG, io
    assert (info["cls"], info["route"], info["kl"], info["ku"]) == (io["cls"], io["route"], 1, 1), (info, io)
    assert rc == io["status"] == 0, (rc, info)
    kappa = n / io["rcond"]
    assert np.abs(X - Xo).max() / np.abs(Xo).max() <= EPS * n * kappa
    assert abs(info["rcond"] - io["rcond"]) <= 1e-5 * io["rcond"], (info["rcond"], io["rcond"])
    assert info["berr"] <= 1e-13, info
    assert (info["detail"] & 16) == {"dominant": 16, "laplace": 0, "none": 0}[kind], info


def test_tridiag_zero_pivot_svd(ctx):
    from paper_2007_11208_gb300 import asolve
    n = 2000
    rng = np.random.default_rng(23)
    AB, kld, kud = band_storage(n, 1, 1, rng)
    AB[:, 900] = 0.0
    B = rng.standard_normal((n, 1))
    rc, info, X = solve_band_gpu(ctx, AB, kld, kud, B, asolve.TRIDIAG)
    assert rc == asolve.W_APPROX and info["route"] == asolve.ROUTE_TRIDIAG and info["svd_rank"] == n - 1, info
    rc, info, X = solve_band_gpu(ctx, AB, kld, kud, B, asolve.TRIDIAG | asolve.NO_APPROX)
    assert rc == asolve.E_SINGULAR and np.all(X == 0.0)
