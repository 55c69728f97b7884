"""GPU parity of the banded route (Sec. 2.1) for band-storage input
(asolve_solve_band) and for dense banded matrices with n > 1024, against the
oracle's band LU (xGBTRF/xGBTRS/xGBCON semantics).

Bar: kl, ku, class and route identical; X within the forward-error bound
2^-52 * n * kappa_inf of the oracle's X (checked as a relative error against
a kappa estimate from the oracle's rcond); rcond within 1e-5 relative (the
same FP64 estimator iteration on factors with the same pivots); backward
error <= 1e-13 when asked for.
"""
import numpy as np
import pytest
import torch

from gpu_util import dev_colmajor, dev_rhs, host_from_dev

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -52


@pytest.fixture(scope="module")
def ctx():
    from paper_2007_11208_gb300 import asolve, build
    build.build()
    c = asolve.Context()
    yield c
    c.close()


def band_storage(n, kl, ku, rng, dominant=True, extra=(0, 0)):
    """(ldab, n) Fortran-ordered band storage with declared bandwidths
    kl+extra[0], ku+extra[1] (the extra diagonals are zero)."""
    kld, kud = kl + extra[0], ku + extra[1]
    ldab = kld + kud + 1
    AB = np.zeros((ldab, n), order="F")
    for d in range(-kl, ku + 1):  # d = j - i
        if d == 0:
            continue
        m = n - abs(d)
        if m <= 0:
            continue
        v = rng.standard_normal(m)
        j = np.arange(m) + max(d, 0)
        i = j - d
        AB[kud + i - j, j] = v
    rows = np.zeros(n)
    for r in range(ldab):
        j = np.arange(n)
        i = r - kud + j
        ok = (i >= 0) & (i < n) & (r != kud)
        np.add.at(rows, i[ok], np.abs(AB[r, j[ok]]))
    diag = 1.0 + rows if dominant else rng.standard_normal(n)
    AB[kud, :] = diag
    return AB, kld, kud


def to_dense(AB, kld, kud, n):
    A = np.zeros((n, n))
    for r in range(AB.shape[0]):
        j = np.arange(n)
        i = r - kud + j
        ok = (i >= 0) & (i < n)
        A[i[ok], j[ok]] = AB[r, j[ok]]
    return A


def solve_band_gpu(ctx, AB, kld, kud, B, flags=0):
    n = AB.shape[1]
    dAB = torch.from_numpy(np.asfortranarray(AB).ravel(order="F").copy()).cuda()
    dB, nrhs = dev_rhs(B, n)
    dX = torch.zeros_like(dB)
    rc, info = ctx.solve_band(dAB, AB.shape[0], kld, kud, dB, n, nrhs, dX, flags)
    return rc, info, host_from_dev(dX, n, nrhs)


def check_against_oracle(orc, AB, kld, kud, B, rc, info, X, berr=False):
    Xo, io = orc.solve_band(AB, kld, kud, B)
    assert rc == io["status"] == 0, (rc, io["status"])
    assert (info["cls"], info["route"], info["kl"], info["ku"]) == (io["cls"], io["route"], io["kl"], io["ku"])
    n = AB.shape[1]
    kappa = 1.0 / io["rcond"]
    err = np.abs(X - Xo).max() / max(np.abs(Xo).max(), 1e-300)
    assert err <= max(n, 16) * EPS * kappa * 4, (err, kappa)
    assert abs(info["rcond"] - io["rcond"]) <= 1e-5 * io["rcond"], (info["rcond"], io["rcond"])
    if berr:
        assert info["berr"] <= 1e-13


CASES = [(1, 0, 0, 1), (2, 1, 0, 1), (5, 1, 1, 2), (33, 2, 3, 3), (100, 8, 8, 1), (257, 0, 7, 2),
         (300, 5, 0, 1), (1000, 32, 32, 4), (1025, 31, 1, 1), (2000, 40, 20, 3), (5000, 2, 2, 16),
         (4097, 60, 50, 2),
         # n >= 2048 with windows of at most 72: the partitioned sweeps (one-sided
         # bands, the widest window, a block count that leaves a ragged last block)
         (2048, 0, 9, 3), (3001, 7, 0, 2), (2100, 35, 35, 1), (20011, 3, 4, 5)]


@pytest.mark.parametrize("n,kl,ku,nrhs", CASES)
def test_band_storage_vs_oracle(ctx, orc, n, kl, ku, nrhs):
    from paper_2007_11208_gb300 import asolve
    rng = np.random.default_rng(n * 7 + kl * 3 + ku)
    AB, kld, kud = band_storage(n, kl, ku, rng, extra=(1, 2))
    B = rng.standard_normal((n, nrhs))
    rc, info, X = solve_band_gpu(ctx, AB, kld, kud, B, asolve.BERR)
    check_against_oracle(orc, AB, kld, kud, B, rc, info, X, berr=True)


@pytest.mark.parametrize("n,kl,ku", [(64, 3, 2), (700, 8, 5), (3000, 16, 16), (2500, 33, 40)])
def test_band_pivoting_vs_oracle(ctx, orc, n, kl, ku):
    """Diagonal not dominant: rows are interchanged inside the band."""
    rng = np.random.default_rng(n + kl)
    AB, kld, kud = band_storage(n, kl, ku, rng, dominant=False)
    B = rng.standard_normal((n, 2))
    rc, info, X = solve_band_gpu(ctx, AB, kld, kud, B)
    Xo, io = orc.solve_band(AB, kld, kud, B)
    if io["status"] != 0:
        pytest.skip("oracle did not solve this draw")
    check_against_oracle(orc, AB, kld, kud, B, rc, info, X)


def test_band_singular_and_svd(ctx, orc):
    from paper_2007_11208_gb300 import asolve
    rng = np.random.default_rng(3)
    n = 80
    AB, kld, kud = band_storage(n, 2, 2, rng)
    AB[:, 40] = 0.0  # a zero column: the band LU meets an exact zero pivot
    B = rng.standard_normal((n, 1))
    rc, info, X = solve_band_gpu(ctx, AB, kld, kud, B, asolve.NO_APPROX)
    assert rc == asolve.E_SINGULAR and np.all(X == 0.0)
    rc, info, X = solve_band_gpu(ctx, AB, kld, kud, B)
    Xo, io = orc.solve_band(AB, kld, kud, B)
    assert rc == io["status"] == asolve.W_APPROX
    assert info["route"] == io["route"] == asolve.ROUTE_BAND_LU
    assert info["svd_rank"] == io["svd_rank"]
    assert np.abs(X - Xo).max() <= 1e-10 * max(np.abs(Xo).max(), 1.0)


def test_band_nonfinite_and_invalid(ctx):
    from paper_2007_11208_gb300 import asolve
    rng = np.random.default_rng(4)
    AB, kld, kud = band_storage(50, 1, 1, rng)
    AB[kud, 7] = np.inf
    rc, info, _ = solve_band_gpu(ctx, AB, kld, kud, rng.standard_normal((50, 1)))
    assert rc == asolve.E_NONFINITE
    dAB = torch.zeros(30, dtype=torch.float64, device="cuda")
    X = torch.zeros(10, dtype=torch.float64, device="cuda")
    assert ctx.solve_band(dAB, 2, 1, 1, X, 10, 1, X)[0] == asolve.E_INVALID  # ldab < kl+ku+1


def test_band_host_buffers(ctx, orc):
    from paper_2007_11208_gb300 import asolve
    rng = np.random.default_rng(8)
    n, nrhs = 3000, 2
    AB, kld, kud = band_storage(n, 4, 6, rng)
    B = rng.standard_normal((n, nrhs))
    hAB = np.asfortranarray(AB).ravel(order="F").copy()
    hB = np.ascontiguousarray(B.T)
    hX = np.zeros_like(hB)
    rc, info = ctx.solve_band(hAB.ctypes.data, AB.shape[0], kld, kud, hB.ctypes.data, n, nrhs,
                              hX.ctypes.data, asolve.HOST_BUFFERS)
    check_against_oracle(orc, AB, kld, kud, B, rc, info, hX.T)


@pytest.mark.parametrize("n,kl,ku", [(1100, 3, 5), (2048, 16, 16), (1500, 130, 140)])
def test_dense_banded_large(ctx, orc, n, kl, ku):
    """Dense input with n > 1024 that the scan finds banded: the banded route
    (the last case is wider than the band kernels' windows and runs the
    dense LU, which pivots the same way)."""
    from paper_2007_11208_gb300 import asolve
    rng = np.random.default_rng(n + ku)
    AB, kld, kud = band_storage(n, kl, ku, rng)
    A = to_dense(AB, kld, kud, n)
    B = rng.standard_normal((n, 2))
    dA = dev_colmajor(A)
    dB, nrhs = dev_rhs(B, n)
    for prec in (asolve.PREC_FP64, asolve.PREC_MIXED):
        c = asolve.Context(precision=prec)
        dX = torch.zeros_like(dB)
        rc, info = c.solve(dA, dB, n, nrhs, dX, asolve.BERR)
        c.close()
        X = host_from_dev(dX, n, nrhs)
        Xo, io = orc.solve(A, B)
        assert rc == io["status"] == 0
        assert (info["cls"], info["route"], info["kl"], info["ku"]) == (io["cls"], io["route"], io["kl"], io["ku"])
        assert info["berr"] <= 1e-13
        kappa = 1.0 / io["rcond"]
        assert np.abs(X - Xo).max() / np.abs(Xo).max() <= n * EPS * kappa * 4


def test_band_million(ctx, orc):
    """Band storage at the memory-bound size: n = 10^6, kl = ku = 8."""
    from paper_2007_11208_gb300 import asolve, synth
    n, kl, ku = 1_000_000, 8, 8
    g = synth.gen(11, "cuda")
    AB_t = synth.band_storage_dd(n, kl, ku, g, device="cuda")  # (n, ldab): row j = column j
    B = synth.rhs(n, 1, g, "cuda")
    X = torch.zeros_like(B)
    rc, info = ctx.solve_band(AB_t, kl + ku + 1, kl, ku, B, n, 1, X, asolve.BERR)
    assert rc == 0 and info["berr"] <= 1e-13
    ABh = AB_t.cpu().numpy().T  # (ldab, n), Fortran-contiguous view
    Xo, io = orc.solve_band(ABh, kl, ku, B.cpu().numpy().reshape(n, 1))
    assert (info["kl"], info["ku"]) == (io["kl"], io["ku"])
    x = X.cpu().numpy().reshape(n)
    assert np.abs(x - Xo[:, 0]).max() <= 1e-12 * np.abs(Xo).max()
    assert abs(info["rcond"] - io["rcond"]) <= 1e-5 * io["rcond"]
