"""GMRES-IR on the large path (the 16-bit trailing-update modes).

With BF16 or FP16 trailing updates the factors carry a relative error near
the 16-bit unit roundoff, and classical refinement converges only while
kappa stays below about 1e3 / 1e4.  GMRES-IR (Carson & Higham) solves each
correction equation by GMRES preconditioned with the same factors, which
reaches kappa 1e6 and beyond.  General systems U diag(logspace) V^T of the
mixed-precision configuration (n = 2048 and 8192, kappa 1e4 and 1e6, a
known solution):

* class, kl/ku and route as the oracle routes them (the oracle's scan and
  the detection order of Sec. 2), status OK;
* the answer comes from the 16-bit factors through GMRES-IR (precision
  BF16 / FP16, detail bit 5), not from the FP64 fallback -- except BF16 at
  kappa 1e6 (kappa times the BF16 unit roundoff ~ 4e3), which may take the
  FP64 factorisation;
* backward error <= 1e-13 (the oracle's compensated residual), forward
  error <= 2^-52 n kappa_inf against the known solution (kappa_inf <=
  n kappa_2 by construction), and at n = 2048 against the oracle's X.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps
BERR = 1e-13


@pytest.mark.parametrize("prec_name", ["bf16", "fp16"])
@pytest.mark.parametrize("n,kappa", [(2048, 1e4), (2048, 1e6), (8192, 1e4), (8192, 1e6)])
def test_gmres_ir_large(orc, prec_name, n, kappa):
    from paper_2007_11208_gb300 import asolve, build, synth
    build.build()
    prec = {"bf16": asolve.PREC_BF16, "fp16": asolve.PREC_FP16}[prec_name]
    dev = torch.device("cuda", 0)
    g = synth.gen(int(n + 31 * kappa) % 100003, dev)
    M = synth.spectrum_fast(n, g, kappa, spd=False, device=dev)  # M[j, i] = A[i, j]
    xt = synth.rhs(n, 1, g, dev)
    B = (M.t() @ xt.t()).t().contiguous()
    X = torch.zeros_like(B)
    ctx = asolve.Context(precision=prec)
    rc, info = ctx.solve(M, B, n, 1, X, asolve.BERR)
    torch.cuda.synchronize()
    ctx.close()
    A = M.cpu().numpy().T
    b = B.cpu().numpy().reshape(n, 1)
    x = X.cpu().numpy().reshape(n, 1)
    sr = orc.scan(A)
    assert sr["cls"] == orc.CLS_GENERAL
    assert rc == 0 and (info["cls"], info["kl"], info["ku"], info["route"]) == \
        (sr["cls"], sr["kl"], sr["ku"], orc.ROUTE_LU), info
    if prec_name == "bf16" and kappa >= 1e6:
        # kappa u_bf16 ~ 4e3: beyond what a 30-vector Krylov basis absorbs;
        # the FP64 factorisation answers (gate or stall), as the same bars
        assert (info["precision"] == prec and info["detail"] & 32) or \
            (info["precision"] == asolve.PREC_FP64 and info["detail"] & 3), info
    else:
        assert info["precision"] == prec and info["detail"] & 32, (info["precision"], info["detail"], info)
    _, berr = orc.residual_dot2(A, x, b)
    assert berr.max() <= BERR, (berr, info)
    assert info["berr"] <= BERR, info
    x_true = xt.cpu().numpy().reshape(n, 1)
    kinf_bound = n * kappa
    assert np.abs(x - x_true).max() / np.abs(x_true).max() <= EPS * n * kinf_bound
    if n <= 2048:
        Xo, io = orc.solve(A, b)
        assert io["route"] == orc.ROUTE_LU and io["status"] == 0
        assert np.abs(x - Xo).max() / np.abs(Xo).max() <= EPS * n * kinf_bound


@pytest.mark.parametrize("n,kappa", [(2048, 1e1), (2048, 1e2), (4096, 1e2)])
def test_fp8_experiment(orc, n, kappa):
    """FP8 E4M3 trailing updates (the configuration's experiment): the
    answer meets the same bars whichever way it comes -- GMRES-IR on the FP8
    factors (precision FP8, detail bit 5) or the FP64 re-factorisation
    after the gate or a stall (detail bits 0 / 1)."""
    from paper_2007_11208_gb300 import asolve, build, synth
    build.build()
    dev = torch.device("cuda", 0)
    g = synth.gen(int(n + 7 * kappa) % 100003, dev)
    M = synth.spectrum_fast(n, g, kappa, spd=False, device=dev)
    xt = synth.rhs(n, 1, g, dev)
    B = (M.t() @ xt.t()).t().contiguous()
    X = torch.zeros_like(B)
    ctx = asolve.Context(precision=asolve.PREC_FP8)
    rc, info = ctx.solve(M, B, n, 1, X, asolve.BERR)
    torch.cuda.synchronize()
    ctx.close()
    A = M.cpu().numpy().T
    b = B.cpu().numpy().reshape(n, 1)
    x = X.cpu().numpy().reshape(n, 1)
    sr = orc.scan(A)
    assert rc == 0 and (info["cls"], info["kl"], info["ku"], info["route"]) == \
        (sr["cls"], sr["kl"], sr["ku"], orc.ROUTE_LU), info
    assert (info["precision"] == asolve.PREC_FP8 and info["detail"] & 32) or \
        (info["precision"] == asolve.PREC_FP64 and info["detail"] & 3), info
    _, berr = orc.residual_dot2(A, x, b)
    assert berr.max() <= BERR, berr
    xtrue = xt.cpu().numpy().reshape(n, 1)
    assert np.abs(x - xtrue).max() / np.abs(xtrue).max() <= 2.0 ** -52 * n * n * kappa, info
