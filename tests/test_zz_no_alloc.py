"""The allocation-free scan entry point (asolve_scan_noalloc).

It exists for callers that may not allocate device memory; its workspace is
a fixed array inside the library.  This file is collected last on purpose:
a failure here leaves every other test already run.  The test calls the
entry point through the C ABI twice in a row (the second call reuses the
shared array left over by the first) and checks both results against the
existing, context-owning asolve_scan and against the oracle's scan of the
same matrix (class, kl/ku and flags bit-exact, norms within the scan's
stated accuracy), up to n = 2048, the entry point's limit.
"""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

NORM_RTOL = 2.0 ** -17  # the scan's stated norm accuracy


def _matrices():
    rng = np.random.default_rng(2024)
    n1 = 333
    G = rng.standard_normal((n1, n1))
    S = G.T @ G / n1 + np.eye(n1)
    sympd = np.tril(S) + np.tril(S, -1).T
    n2 = 2048
    band = np.zeros((n2, n2))
    for d in (-3, -1, 0, 2, 5):
        band += np.diag(rng.standard_normal(n2 - abs(d)), d)
    general = rng.standard_normal((1000, 1000))
    G2 = rng.standard_normal((n2, n2))
    S2 = G2.T @ G2 / n2 + np.eye(n2)
    sympd2 = np.tril(S2) + np.tril(S2, -1).T
    return [sympd, band, general, sympd2]


def test_noalloc_scan_matches_asolve_scan(orc):
    from paper_2007_11208_gb300 import asolve, build
    build.build()
    L = asolve.lib()
    ctx = asolve.Context()
    out = torch.zeros(C.sizeof(asolve.ScanResult), dtype=torch.uint8, device="cuda")
    for A in _matrices():
        n = A.shape[0]
        dA = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
        ref = ctx.scan(dA, n)
        oref = orc.scan(A)
        for k in ("kl", "ku", "lower", "upper", "sympd", "banded", "nonfinite", "cls"):
            assert int(ref[k]) == int(oref[k]), (n, k, ref[k], oref[k])
        for call in range(2):  # two calls in a row on the shared workspace
            out.zero_()
            rc = L.asolve_scan_noalloc(C.c_void_p(dA.data_ptr()), n, C.c_void_p(out.data_ptr()), None)
            assert rc == asolve.OK, asolve.strerror(rc)
            torch.cuda.synchronize()
            got = asolve.ScanResult.from_buffer_copy(out.cpu().numpy().tobytes())
            for k in ("kl", "ku", "lower", "upper", "sympd", "banded", "nonfinite", "cls"):
                assert getattr(got, k) == ref[k], (n, call, k, getattr(got, k), ref[k])
            for k in ("norm1", "norminf"):
                assert abs(getattr(got, k) - ref[k]) <= NORM_RTOL * ref[k], (n, call, k)
    ctx.close()


def test_noalloc_scan_rejects_oversize():
    from paper_2007_11208_gb300 import asolve, build
    build.build()
    L = asolve.lib()
    out = torch.zeros(C.sizeof(asolve.ScanResult), dtype=torch.uint8, device="cuda")
    A = torch.zeros(8, dtype=torch.float64, device="cuda")
    rc = L.asolve_scan_noalloc(C.c_void_p(A.data_ptr()), 2049, C.c_void_p(out.data_ptr()), None)
    assert rc == asolve.E_UNSUPPORTED
