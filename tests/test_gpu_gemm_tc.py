"""The tcgen05 trailing-update GEMM (C -= A B, FP32 storage, TF32 tensor
cores) against an FP64 product: plain TF32 within 2^-10 sqrt(K) of
|A||B|, the 3-pass split within 2^-20 sqrt(K)."""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 128, 32), (300, 200, 100), (64, 17, 5), (1024, 768, 128),
                                   (129, 131, 33)])
@pytest.mark.parametrize("passes", [1, 3])
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
    tol = (2.0 ** -10 if passes == 1 else 2.0 ** -20) * np.sqrt(K)
    assert np.all(np.abs(got - ref) <= tol * scale + 1e-6 * np.abs(Cm)), np.max(np.abs(got - ref) / scale)
