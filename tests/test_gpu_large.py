"""Large single systems (n > 1024): blocked Cholesky / LU on the whole GPU
(tcgen05 3xTF32 trailing updates in the mixed mode, mma.sync f64 in the
FP64 mode, Ozaki-split BF16 tensor products in the FP64_OZ mode), blocked
triangular solves, FP64 refinement.

Element-wise parity with the oracle at sizes it solves in seconds; at
larger n the backward error (oracle Dot2 residual) and the forward error
against a known solution."""
import numpy as np
import pytest

from gpu_util import fwd_err, kappa_inf, solve_gpu

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module", params=["fp64", "mixed", "fp64_oz"])
def ctx(request):
    from paper_2007_11208_gb300 import asolve, build
    build.build()
    prec = {"fp64": asolve.PREC_FP64, "mixed": asolve.PREC_MIXED, "fp64_oz": asolve.PREC_FP64_OZ}[request.param]
    c = asolve.Context(precision=prec)
    c.prec = request.param
    yield c
    c.close()


def make(kind, n, rng):
    if kind == "general":
        return rng.standard_normal((n, n)) + 2 * np.sqrt(n) * np.eye(n)
    if kind == "general_raw":
        return rng.standard_normal((n, n))
    if kind == "spd":
        G = rng.standard_normal((n, n))
        S = G.T @ G / n + np.eye(n)
        return np.tril(S) + np.tril(S, -1).T
    if kind == "lower":
        A = np.tril(rng.standard_normal((n, n)), -1)
        return A + np.diag(1 + np.abs(A).sum(1))
    if kind == "upper":
        A = np.triu(rng.standard_normal((n, n)), 1)
        return A + np.diag(1 + np.abs(A).sum(1))
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["general", "general_raw", "spd", "lower", "upper"])
@pytest.mark.parametrize("n", [1100, 1411])
def test_large_vs_oracle(ctx, orc, kind, n):
    rng = np.random.default_rng(n + len(kind))
    A = make(kind, n, rng)
    nrhs = 3
    B = rng.standard_normal((n, nrhs))
    rc, info, X = solve_gpu(ctx, A, B)
    Xo, io = orc.solve(A, B)
    assert (info["cls"], info["kl"], info["ku"], info["route"]) == (io["cls"], io["kl"], io["ku"], io["route"]), \
        (info, io)
    assert rc == io["status"] == 0, (rc, info)
    assert fwd_err(X, Xo) <= 2.0 ** -52 * n * kappa_inf(A), (fwd_err(X, Xo), info)
    _, berr = orc.residual_dot2(A, X, B)
    assert berr.max() <= 1e-13, (berr, info)
    assert io["rcond"] / 3 <= info["rcond"] <= io["rcond"] * 3, (info["rcond"], io["rcond"])


def spectrum(n, kappa, rng, spd=False):
    U, _ = np.linalg.qr(rng.standard_normal((n, n)))
    s = np.logspace(0, -np.log10(kappa), n)
    if spd:
        A = (U * s) @ U.T
        return np.tril(A) + np.tril(A, -1).T
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return (U * s) @ V.T


@pytest.mark.parametrize("kind,n,nrhs", [("lower", 2048, 9), ("upper", 1100, 64), ("lower", 2048, 256),
                                          ("general", 1100, 40), ("spd", 1411, 17)])
def test_large_many_rhs(ctx, orc, kind, n, nrhs):
    """Right-hand sides spanning several 8-column chunks of the wavefront
    triangular solve and of the residual kernel, with a ragged last chunk."""
    rng = np.random.default_rng(n + nrhs)
    A = make(kind, n, rng)
    B = rng.standard_normal((n, nrhs))
    rc, info, X = solve_gpu(ctx, A, B)
    Xo, io = orc.solve(A, B)
    assert rc == io["status"] == 0 and info["route"] == io["route"], (rc, info, io)
    ka = kappa_inf(A)
    for j in range(nrhs):  # column by column: a wrong chunk shows which one
        assert fwd_err(X[:, j], Xo[:, j]) <= 2.0 ** -52 * n * ka, (j, fwd_err(X[:, j], Xo[:, j]))
    _, berr = orc.residual_dot2(A, X, B)
    assert berr.max() <= 1e-13, (berr.max(), info)


@pytest.mark.parametrize("kappa", [1e2, 1e4, 1e6])
@pytest.mark.parametrize("spd", [False, True])
def test_large_known_x_spectra(ctx, orc, kappa, spd):
    n = 2304
    rng = np.random.default_rng(int(np.log10(kappa)) + 10 * spd)
    A = spectrum(n, kappa, rng, spd)
    xt = rng.standard_normal((n, 2))
    B = A @ xt
    rc, info, X = solve_gpu(ctx, A, B)
    assert rc == 0, info
    _, berr = orc.residual_dot2(A, X, B)
    assert berr.max() <= 1e-13, (berr, info)
    k_inf = kappa * n  # construction bound on kappa_inf
    assert np.abs(X - xt).max() / np.abs(xt).max() <= 2.0 ** -52 * n * k_inf
    if ctx.prec == "mixed":  # refinement converges up to kappa 1e6 with FP32-level factors
        assert info["precision"] == 1 and info["ir_iters"] >= 1, info


def test_large_chol_fail_to_lu(ctx, orc):
    n = 1200
    rng = np.random.default_rng(3)
    A = spectrum(n, 1e3, rng, spd=True)
    A -= 0.5 * np.eye(n) * np.abs(np.linalg.eigvalsh(A)).min() * 0  # keep exactly symmetric
    # make it indefinite but still passing the Fig. 4 predicates: flip one small eigenvalue
    w, U = np.linalg.eigh(A)
    w[0] = -w[0]
    A = (U * w) @ U.T
    A = np.tril(A) + np.tril(A, -1).T
    s = orc.scan(A)
    if s["cls"] != 4:
        pytest.skip("matrix does not pass the likely_sympd predicates")
    B = rng.standard_normal(n)
    rc, info, X = solve_gpu(ctx, A, B)
    assert info["route"] == 5 and rc == 0, info
    _, berr = orc.residual_dot2(A, X, B)
    assert berr.max() <= 1e-13


@pytest.mark.parametrize("prec_name", ["bf16", "fp16"])
@pytest.mark.parametrize("kind,n,kappa", [("general", 2048, None), ("spd", 1411, None), ("general", 1100, 1e2),
                                          ("spd", 2304, 1e2), ("general", 1500, 1e6)])
def test_large_16bit_updates(orc, prec_name, kind, n, kappa):
    """Trailing updates as single 16-bit tensor products (BF16, or FP16 with
    per-tile scaling), FP64 refinement: the answer meets the same bars as
    the FP64 path; well-conditioned systems finish in the 16-bit mode, and
    kappa above the classical refinement's limit goes to GMRES-IR (or, if
    that does not converge, to the FP64 factorisation)."""
    from paper_2007_11208_gb300 import asolve, build
    build.build()
    prec = {"bf16": asolve.PREC_BF16, "fp16": asolve.PREC_FP16}[prec_name]
    rng = np.random.default_rng(n + (0 if kappa is None else int(np.log10(kappa))))
    A = make(kind, n, rng) if kappa is None else spectrum(n, kappa, rng, kind == "spd")
    B = rng.standard_normal((n, 2))
    c = asolve.Context(precision=prec)
    rc, info, X = solve_gpu(c, A, B)
    c.close()
    Xo, io = orc.solve(A, B)
    assert rc == io["status"] == 0, (rc, info)
    assert (info["cls"], info["route"]) == (io["cls"], io["route"]), (info, io)
    _, berr = orc.residual_dot2(A, X, B)
    assert berr.max() <= 1e-13, (berr, info)
    assert fwd_err(X, Xo) <= 2.0 ** -52 * n * kappa_inf(A), (fwd_err(X, Xo), info)
    if kappa is not None and kappa >= 1e6:
        # beyond the classical refinement's limit: GMRES-IR with the 16-bit
        # factors, else the FP64 factorisation
        assert (info["precision"] == prec and info["detail"] & 32) or \
            (info["precision"] == asolve.PREC_FP64 and info["detail"] & 3), info
    elif kappa is None:
        assert info["precision"] == prec and info["ir_iters"] >= 1, info


def test_mixed_fallback_refactors_with_ozaki_updates(orc):
    """A system beyond the FP32 factors' kappa gate: the mixed mode
    re-factors it in FP64 with Ozaki-split trailing updates (detail bit 6),
    and the answer meets the FP64 bar against the oracle."""
    from paper_2007_11208_gb300 import asolve, build
    build.build()
    rng = np.random.default_rng(77)
    n = 2048
    A = spectrum(n, 1e12, rng)
    B = rng.standard_normal((n, 2))
    ctx = asolve.Context(precision=asolve.PREC_MIXED)
    rc, info, X = solve_gpu(ctx, A, B, asolve.BERR)
    ctx.close()
    Xo, io = orc.solve(A, B)
    assert (info["route"], rc) == (io["route"], io["status"]), (info, io)
    assert info["precision"] == asolve.PREC_FP64 and info["detail"] & 64 and info["detail"] & 1, info
    _, berr = orc.residual_dot2(A, X, B)
    assert berr.max() <= 1e-13, berr
    assert fwd_err(X, Xo) <= 2.0 ** -52 * n * n * 1e12
    assert abs(info["rcond"] - io["rcond"]) <= 1e-2 * io["rcond"], (info["rcond"], io["rcond"])
