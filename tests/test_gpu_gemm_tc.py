"""The tcgen05 trailing-update GEMM (C -= A B, FP32 storage, tensor cores)
against an FP64 product: plain TF32 within 2^-10 sqrt(K) of |A||B|, the
3-pass split within 2^-20 sqrt(K); single-pass BF16 and FP16 operands
within 2^-7 and 2^-9 of |A||B| (twice the unit roundoff of the 16-bit type
per product, with margin), FP16 also for operands outside its range; FP8
E4M3 operands (per-tile scaled) within 2^-2.5 of |A||B|, and well inside
that on average."""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 128, 32), (300, 200, 100), (64, 17, 5), (1024, 768, 128),
                                   (129, 131, 33)])
@pytest.mark.parametrize("passes", [1, 3, 16, 17, 18])
def test_gemm_tc(M, N, K, passes):
    from paper_2007_11208_gb300 import asolve, build
    build.build()
    L = asolve.lib()
    rng = np.random.default_rng(M * 1000 + N + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.standard_normal((K, N)).astype(np.float32)
    Cm = rng.standard_normal((M, N)).astype(np.float32)
    dA = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
    dB = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    dC = torch.from_numpy(np.ascontiguousarray(Cm.T)).cuda()
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = L.asolve_gemm_sub(C.c_void_p(dC.data_ptr()), M, C.c_void_p(dA.data_ptr()), M,
                           C.c_void_p(dB.data_ptr()), K, M, N, K, passes,
                           C.c_void_p(err.data_ptr()), None)
    assert rc == 0
    torch.cuda.synchronize()
    assert err.item() == 0
    got = dC.cpu().numpy().T
    ref = Cm.astype(np.float64) - A.astype(np.float64) @ B.astype(np.float64)
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64) + np.abs(Cm)
    # FP8 E4M3: 3 stored mantissa bits (unit roundoff 2^-4) per operand, plus
    # entries below the tile's 2^-16 (subnormal range after the tile scale)
    tol = {1: 2.0 ** -10 * np.sqrt(K), 3: 2.0 ** -20 * np.sqrt(K), 16: 2.0 ** -7, 17: 2.0 ** -9,
           18: 2.0 ** -2.5}[passes]
    assert np.all(np.abs(got - ref) <= tol * scale + 1e-6 * np.abs(Cm)), np.max(np.abs(got - ref) / scale)


@pytest.mark.parametrize("a_mag,b_mag", [(1e5, 1e-7), (1e-6, 1e6), (3e4, 3e4)])
def test_gemm_fp16_tile_scaling(a_mag, b_mag):
    """FP16 operands beyond its range (max 65504, smallest normal 2^-14)
    keep the 2^-9 bound: each tile is scaled by a power of two first."""
    from paper_2007_11208_gb300 import asolve, build
    build.build()
    L = asolve.lib()
    M, N, K = 256, 130, 64
    rng = np.random.default_rng(5)
    A = (rng.standard_normal((M, K)) * a_mag).astype(np.float32)
    B = (rng.standard_normal((K, N)) * b_mag).astype(np.float32)
    Cm = np.zeros((M, N), dtype=np.float32)
    dA = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
    dB = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    dC = torch.from_numpy(np.ascontiguousarray(Cm.T)).cuda()
    rc = L.asolve_gemm_sub(C.c_void_p(dC.data_ptr()), M, C.c_void_p(dA.data_ptr()), M,
                           C.c_void_p(dB.data_ptr()), K, M, N, K, asolve.GEMM_FP16, None, None)
    assert rc == 0
    torch.cuda.synchronize()
    got = dC.cpu().numpy().T.astype(np.float64)
    ref = -(A.astype(np.float64) @ B.astype(np.float64))
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64)
    assert np.all(np.isfinite(got))
    assert np.all(np.abs(got - ref) <= 2.0 ** -9 * scale), np.max(np.abs(got - ref) / scale)


def test_gemm_mode_invalid():
    from paper_2007_11208_gb300 import asolve, build
    build.build()
    L = asolve.lib()
    x = torch.zeros(16, dtype=torch.float32, device="cuda")
    p = C.c_void_p(x.data_ptr())
    assert L.asolve_gemm_sub(p, 4, p, 4, p, 4, 4, 4, 4, 2, None, None) == asolve.E_INVALID


def test_gemm_fp8_typical_error():
    """The FP8 E4M3 product is FP8 arithmetic, not noise: its typical error
    is near two E4M3 roundings (2^-4 each) of |A||B|, far below its bound."""
    from paper_2007_11208_gb300 import asolve, build
    build.build()
    L = asolve.lib()
    M, N, K = 512, 256, 256
    rng = np.random.default_rng(8)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.standard_normal((K, N)).astype(np.float32)
    dA = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
    dB = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    dC = torch.zeros(M * N, dtype=torch.float32, device="cuda")
    rc = L.asolve_gemm_sub(C.c_void_p(dC.data_ptr()), M, C.c_void_p(dA.data_ptr()), M,
                           C.c_void_p(dB.data_ptr()), K, M, N, K, asolve.GEMM_FP8, None, None)
    assert rc == 0
    torch.cuda.synchronize()
    got = dC.cpu().numpy().reshape(N, M).T
    ref = -(A.astype(np.float64) @ B.astype(np.float64))
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64)
    rel = np.abs(got - ref) / scale
    assert np.median(rel) <= 2.0 ** -5, np.median(rel)
    assert np.median(rel) >= 2.0 ** -12, np.median(rel)  # and not a higher precision in disguise
