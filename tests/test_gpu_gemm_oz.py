"""The Ozaki-split FP64 product (asolve_gemm_oz: C -= A op(B) from exact
BF16 slices on the tcgen05 tensor cores) against the oracle's compensated
residual of the same product (Dot2, accurate to about 2^-104 |A||B|).

The bound is the method's, per K chunk c of 128 columns:
|error(i, j)| <= 2^-44 sum_c max_{k in c} |A(i, k)| max_{k in c} |op(B)(k, j)|
(slicing 2^-57 of the row / column scale, the dropped slice products
about 2^-48.4, the conversion and the FMA 2^-52 of the chunk's result; the
scales are at most 4x the maxima), plus 2^-52 |C| for the final rounding.
Cases: tiles and ragged edges in M, N and K, transposed B, rows and
columns whose magnitudes span 2^+-300 (per-row / per-column scales), a
row with a wide range of magnitudes inside it, zero rows and columns,
and a non-finite entry (its row of C becomes NaN, the rest exact)."""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def run(A, B, Cm, transb=False):
    from paper_2007_11208_gb300 import asolve, build
    build.build()
    L = asolve.lib()
    M, K = A.shape
    N = B.shape[0] if transb else B.shape[1]
    dA = torch.from_numpy(np.asfortranarray(A).ravel(order="F").copy()).cuda()
    dB = torch.from_numpy(np.asfortranarray(B).ravel(order="F").copy()).cuda()
    dC = torch.from_numpy(np.asfortranarray(Cm).ravel(order="F").copy()).cuda()
    wsb = L.asolve_gemm_oz_ws_bytes(M, N, K)
    ws = torch.empty(wsb + 256, dtype=torch.uint8, device="cuda")
    wp = (ws.data_ptr() + 255) & ~255
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    ldb = N if transb else K
    rc = L.asolve_gemm_oz(C.c_void_p(dC.data_ptr()), M, C.c_void_p(dA.data_ptr()), M, C.c_void_p(dB.data_ptr()),
                          ldb, M, N, K, int(transb), C.c_void_p(wp), wsb, C.c_void_p(err.data_ptr()), None)
    assert rc == 0
    torch.cuda.synchronize()
    assert err.item() == 0
    return dC.cpu().numpy().reshape((N, M)).T


def bound(A, Bop, Cm):
    M, K = A.shape
    N = Bop.shape[1]
    b = np.zeros((M, N))
    for k0 in range(0, K, 128):
        am = np.abs(A[:, k0:k0 + 128]).max(axis=1)
        bm = np.abs(Bop[k0:k0 + 128, :]).max(axis=0)
        b += np.outer(am, bm)
    return 2.0 ** -44 * b + 2.0 ** -52 * np.abs(Cm - A @ Bop)


def reference(orc, A, Bop, Cm):
    """Cm - A Bop by the oracle's compensated residual (A embedded in a
    square matrix, the extra rows and columns zero)."""
    M, K = A.shape
    N = Bop.shape[1]
    n = max(M, K)
    As = np.zeros((n, n))
    As[:M, :K] = A
    X = np.zeros((n, N))
    X[:K] = Bop
    Bm = np.zeros((n, N))
    Bm[:M] = Cm
    R, _ = orc.residual_dot2(As, X, Bm)
    return R[:M]


@pytest.mark.parametrize("M,N,K", [(128, 64, 128), (300, 130, 257), (1, 1, 1), (517, 65, 1000), (129, 63, 64),
                                   (1024, 512, 128)])
@pytest.mark.parametrize("transb", [False, True])
def test_random_products(orc, M, N, K, transb):
    rng = np.random.default_rng(M * 7 + N * 3 + K + transb)
    A = rng.standard_normal((M, K))
    Bop = rng.standard_normal((K, N))
    Cm = rng.standard_normal((M, N))
    got = run(A, Bop.T.copy() if transb else Bop, Cm, transb)
    ref = reference(orc, A, Bop, Cm)
    err = np.abs(got - ref)
    assert np.all(err <= bound(A, Bop, Cm)), (err.max(), (err / bound(A, Bop, Cm)).max())
    # and no worse than a few times an FP64 GEMM's own error on these data
    fp64 = np.abs((Cm - A @ Bop) - ref)
    assert err.max() <= 8 * fp64.max() + 1e-300, (err.max(), fp64.max())


def test_scaled_rows_and_columns(orc):
    """Per-row and per-column scales: magnitudes 2^-300 .. 2^300."""
    rng = np.random.default_rng(11)
    M, N, K = 256, 96, 300
    A = rng.standard_normal((M, K)) * np.exp2(rng.integers(-300, 300, size=(M, 1)))
    Bop = rng.standard_normal((K, N)) * np.exp2(rng.integers(-300, 300, size=(1, N)))
    Cm = A @ Bop * 0.5
    got = run(A, Bop, Cm)
    ref = reference(orc, A, Bop, Cm)
    assert np.all(np.abs(got - ref) <= bound(A, Bop, Cm))


def test_wide_range_inside_a_row_and_zeros(orc):
    rng = np.random.default_rng(12)
    M, N, K = 200, 70, 260
    A = rng.standard_normal((M, K))
    A[3] *= np.exp2(rng.integers(-60, 0, size=K))  # one row spanning 2^-60 .. 1
    A[5] = 0.0                                       # a zero row
    A[:, 7] = 0.0                                    # a zero column of A
    Bop = rng.standard_normal((K, N))
    Bop[:, 9] = 0.0                                  # a zero column of op(B)
    Cm = rng.standard_normal((M, N))
    got = run(A, Bop, Cm)
    ref = reference(orc, A, Bop, Cm)
    assert np.all(np.abs(got - ref) <= bound(A, Bop, Cm))
    assert np.array_equal(got[5], Cm[5]) and np.array_equal(got[:, 9], Cm[:, 9])


def test_non_finite_entry_poisons_its_row_only(orc):
    rng = np.random.default_rng(13)
    M, N, K = 130, 40, 150
    A = rng.standard_normal((M, K))
    A[17, 100] = np.inf
    Bop = rng.standard_normal((K, N))
    Cm = rng.standard_normal((M, N))
    got = run(A, Bop, Cm)
    assert np.all(np.isnan(got[17]))
    keep = np.ones(M, bool)
    keep[17] = False
    A2 = A.copy()
    A2[17] = 0.0
    ref = reference(orc, A2, Bop, Cm)
    assert np.all(np.abs(got[keep] - ref[keep]) <= bound(A2, Bop, Cm)[keep])


def test_workspace_checks():
    from paper_2007_11208_gb300 import asolve, build
    build.build()
    L = asolve.lib()
    dC = torch.zeros(64 * 64, dtype=torch.float64, device="cuda")
    need = L.asolve_gemm_oz_ws_bytes(64, 64, 64)
    assert need > 0 and L.asolve_gemm_oz_ws_bytes(0, 64, 64) == 0
    ws = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
    wp = (ws.data_ptr() + 255) & ~255
    p = C.c_void_p(dC.data_ptr())
    assert L.asolve_gemm_oz(p, 64, p, 64, p, 64, 64, 64, 64, 0, C.c_void_p(wp), need - 1, None, None) == asolve.E_INVALID
    assert L.asolve_gemm_oz(p, 64, p, 64, p, 64, 64, 64, 64, 0, C.c_void_p(wp + 8), need, None, None) == asolve.E_INVALID
    assert L.asolve_gemm_oz(p, 63, p, 64, p, 64, 64, 64, 64, 0, C.c_void_p(wp), need, None, None) == asolve.E_INVALID
