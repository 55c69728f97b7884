"""Parity of the whole-GPU property scan (one large system, Sec. 2.1, 2.2,
Fig. 4) with the oracle's scan on the very bytes the GPU read.

The matrices are drawn on the device by the same generators the large
configuration uses (U diag(logspace) V^T, exactly symmetric for SPD), and
queued on torch's stream right before the call: the binding must order the
library's stream after them.  Each matrix is scanned twice; the two results
must be equal, and class, kl/ku and every flag equal to the oracle's
(norms within the FP32-partial bound of the scan kernel).

A second group plants pairs that reach each shortcut of the Fig. 4 pair
test in the scan kernel: exponent gaps of 1, 2 and 3 between A_ij and
A_ji, tiny asymmetric pairs that only the absolute tolerance accepts, a
lower element tied with the largest diagonal entry, and a dominance sum
exactly equal to A_ii + A_jj -- in diagonal and off-diagonal tiles.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
NORM_RTOL = 2.0 ** -17
FLAGS = ("kl", "ku", "lower", "upper", "sympd", "banded", "nonfinite", "cls")


@pytest.fixture(scope="module")
def ctx():
    from paper_2007_11208_gb300 import asolve, build
    build.build()
    c = asolve.Context(precision=asolve.PREC_FP64)
    yield c
    c.close()


def scan_twice_against_oracle(ctx, orc, M, n):
    """M: device tensor whose memory holds A column by column."""
    r1 = ctx.scan(M, n)
    r2 = ctx.scan(M, n)
    assert r1 == r2, (r1, r2)
    A = M.reshape(n, n).cpu().numpy().T  # A[i, j], Fortran-ordered view of the same bytes
    ref = orc.scan(A)
    for k in FLAGS:
        assert int(r1[k]) == int(ref[k]), (k, r1, ref)
    for k in ("norm1", "norminf"):
        assert abs(r1[k] - ref[k]) <= NORM_RTOL * ref[k], (k, r1[k], ref[k])
    return r1, ref


CASES = [(n, kind, kappa) for n in (4096, 8192) for kind in ("spd", "general")
         for kappa in (1e2, 1e4, 1e6)] + [(16384, "spd", 1e4), (16384, "general", 1e6)]


@pytest.mark.parametrize("n,kind,kappa", CASES)
def test_large_scan_spectra(ctx, orc, n, kind, kappa):
    from paper_2007_11208_gb300 import asolve, synth
    dev = torch.device("cuda", 0)
    g = synth.gen(int(n + 17 * kappa) % 100003, dev)
    M = synth.spectrum_fast(n, g, kappa, spd=(kind == "spd"), device=dev)
    got, ref = scan_twice_against_oracle(ctx, orc, M, n)
    assert got["cls"] == (asolve.CLS_SYMPD if kind == "spd" else asolve.CLS_GENERAL), got


def _spd_host(n, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, n))
    S = G.T @ G / n + np.eye(n)
    return np.tril(S) + np.tril(S, -1).T


def _put_pair(A, i, j, a, b):
    """A[i, j] = a (below the diagonal), A[j, i] = b."""
    assert i > j
    A[i, j], A[j, i] = a, b


def _planted_cases(n):
    """(name, A, expected sympd) built from one SPD matrix of order n."""
    S = _spd_host(n, n)
    out = []
    md = float(np.max(np.diag(S)))
    # (i, j): in a diagonal tile (same 32-block) and in an off-diagonal tile
    spots = [(n // 2 + 5, n // 2 + 1), (n - 3, 7)]
    for (i, j) in spots:
        for gap in (1, 2, 3):  # exponents of A_ij and A_ji differ by `gap`
            A = S.copy()
            _put_pair(A, i, j, 0.75, 0.75 * 2.0 ** -gap)
            out.append((f"gap{gap}@{i},{j}", A, False))
        A = S.copy()  # tiny asymmetric pair: |a - b| below the absolute tolerance
        _put_pair(A, i, j, 1e-20, 1e-22)
        out.append((f"tiny@{i},{j}", A, True))
        eps = np.finfo(float).eps
        for (a, b, ok, tag) in ((2.0 ** -44, 2.0 ** -46, False, "gapedge"),  # decided by exponents
                                (2.0 ** -45, 2.0 ** -47, True, "gapabs"),    # only |a-b| <= tol passes
                                (8.0, 8.0 * (1 + 101 * eps), False, "rel"),  # both tests fail
                                (8.0, 8.0 * (1 + 50 * eps), True, "relok")):  # relative test passes
            A = S.copy()
            A[i, i] = A[j, j] = 64.0
            _put_pair(A, i, j, a, b)
            out.append((f"{tag}@{i},{j}", A, ok))
        A = S.copy()  # lower element tied with the largest diagonal entry
        _put_pair(A, i, j, -md, -md)
        out.append((f"maxdiag@{i},{j}", A, False))
        A = S.copy()  # |A_ij| + |A_ji| == A_ii + A_jj exactly (dyadic values)
        A[i, i], A[j, j] = 1.5, 0.5
        _put_pair(A, i, j, 1.0, 1.0)
        out.append((f"dom_eq@{i},{j}", A, False))
        A = S.copy()  # ... and just below it
        A[i, i], A[j, j] = 1.5, 0.5
        _put_pair(A, i, j, 1.0 - 2.0 ** -40, 1.0 - 2.0 ** -40)
        out.append((f"dom_lt@{i},{j}", A, True))
    return out


@pytest.mark.parametrize("n", [4096, 4100])
def test_large_scan_planted_pairs(ctx, orc, n):
    from paper_2007_11208_gb300 import asolve
    dev = torch.device("cuda", 0)
    for name, A, sympd in _planted_cases(n):
        # the oracle's verdict first: the plant must do what its name says
        assert orc.scan(A)["sympd"] == int(sympd), name
        M = torch.from_numpy(np.ascontiguousarray(A.T)).to(dev)
        got, ref = scan_twice_against_oracle(ctx, orc, M, n)
        assert got["cls"] == (asolve.CLS_SYMPD if sympd else asolve.CLS_GENERAL), (name, got)
