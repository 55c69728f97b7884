"""Failure detection without a GPU fault.

* A bounded device wait that runs out: with ASOLVE_WAIT_LIMIT=1 the tensor-
  core GEMM's stage waits (mbarrier polls) give up at once; the kernel must
  raise its error flag and return -- after draining its MMAs with the full
  limit, before it frees tensor memory -- and leave the context usable: the
  same call without the limit then gives the right product.  Then the same
  through a whole large solve, which must report ASOLVE_E_TIMEOUT.
* An allocation failure at call k (host side, ASOLVE_FAIL_ALLOC=1 while the
  call needs a larger workspace): the call returns E_NOMEM with nothing
  launched on a missing buffer, and the next call on the same context
  solves correctly.
"""
import ctypes as C
import os

import numpy as np
import pytest
import torch

from gpu_util import solve_gpu

pytestmark = pytest.mark.gpu


class env:
    def __init__(self, **kw):
        self.kw = kw

    def __enter__(self):
        self.old = {k: os.environ.get(k) for k in self.kw}
        os.environ.update({k: str(v) for k, v in self.kw.items()})

    def __exit__(self, *exc):
        for k, v in self.old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def gemm(L, dA, dB, dC, err, M, N, K):
    return L.asolve_gemm_sub(C.c_void_p(dC.data_ptr()), M, C.c_void_p(dA.data_ptr()), M,
                             C.c_void_p(dB.data_ptr()), K, M, N, K, 3, C.c_void_p(err.data_ptr()), None)


def test_gemm_wait_runs_out_and_the_context_survives():
    from paper_2007_11208_gb300 import asolve, build
    build.build()
    L = asolve.lib()
    M, N, K = 256, 256, 2048  # 64 K chunks: 64 waits, each with one poll
    rng = np.random.default_rng(5)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.standard_normal((K, N)).astype(np.float32)
    dA = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
    dB = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    dC = torch.zeros(M * N, dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    with env(ASOLVE_WAIT_LIMIT=1):
        assert gemm(L, dA, dB, dC, err, M, N, K) == asolve.OK
        torch.cuda.synchronize()  # the kernel returned: no hang, no fault
    assert err.item() == 1
    err.zero_()
    dC.zero_()
    assert gemm(L, dA, dB, dC, err, M, N, K) == asolve.OK
    torch.cuda.synchronize()
    assert err.item() == 0
    got = dC.cpu().numpy().reshape(N, M).T
    ref = -(A.astype(np.float64) @ B.astype(np.float64))
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64)
    assert np.all(np.abs(got - ref) <= 2.0 ** -20 * np.sqrt(K) * scale)


def test_large_solve_reports_timeout_then_solves(orc):
    from paper_2007_11208_gb300 import asolve, build
    build.build()
    rng = np.random.default_rng(6)
    n = 2048
    A = rng.standard_normal((n, n)) + 2 * np.sqrt(n) * np.eye(n)
    B = rng.standard_normal((n, 1))
    ctx = asolve.Context(precision=asolve.PREC_MIXED)  # 3xTF32 trailing updates on the GEMM
    with env(ASOLVE_WAIT_LIMIT=1):
        rc, info, X = solve_gpu(ctx, A, B)
    assert rc == asolve.E_TIMEOUT, info
    rc, info, X = solve_gpu(ctx, A, B)
    assert rc == asolve.OK, info
    _, berr = orc.residual_dot2(A, X, B)
    assert berr.max() <= 1e-13
    ctx.close()


def test_allocation_failure_at_call_k_then_recovery(orc):
    from paper_2007_11208_gb300 import asolve, build
    build.build()
    rng = np.random.default_rng(7)
    ctx = asolve.Context(precision=asolve.PREC_FP64)
    small = rng.standard_normal((1100, 1100)) + 70 * np.eye(1100)
    big = rng.standard_normal((2100, 2100)) + 100 * np.eye(2100)
    b1, b2 = rng.standard_normal((1100, 1)), rng.standard_normal((2100, 1))
    rc, _, _ = solve_gpu(ctx, small, b1)                  # call 1: workspace for n = 1100
    assert rc == asolve.OK
    with env(ASOLVE_FAIL_ALLOC=1):
        rc, _, _ = solve_gpu(ctx, small, b1)              # fits the workspace: no allocation
        assert rc == asolve.OK
        rc, _, _ = solve_gpu(ctx, big, b2)                # call 3 needs more: the allocation fails
        assert rc == asolve.E_NOMEM
    rc, info, X = solve_gpu(ctx, big, b2)                 # the context is still usable
    assert rc == asolve.OK, info
    Xo, io = orc.solve(big, b2)
    assert np.abs(X - Xo).max() <= 1e-10 * np.abs(Xo).max()
    ctx.close()
