"""GPU scan parity: class, kl/ku, triangular and likely_sympd flags must match
the oracle bit-exactly; norms within 2^-17 relative (FP32 partial sums of
truncated magnitudes, see the scan kernel)."""
import itertools
import json
import os

import numpy as np
import pytest
import torch

from gpu_util import dev_colmajor, pack_batch, run_batch

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EPS = np.finfo(np.float64).eps
NORM_RTOL = 2.0 ** -17


@pytest.fixture(scope="module")
def ctx():
    from paper_2007_11208_gb300 import asolve, build
    build.build()
    c = asolve.Context(precision=asolve.PREC_FP64)
    yield c
    c.close()


def check_scan(got, ref, A):
    for k in ("kl", "ku", "lower", "upper", "sympd", "banded", "nonfinite", "cls"):
        assert int(got[k]) == int(ref[k]), (k, got, ref, A if A.size < 50 else A.shape)
    for k in ("norm1", "norminf"):
        assert abs(got[k] - ref[k]) <= NORM_RTOL * ref[k], (k, got[k], ref[k])


def single_scan(ctx, A):
    return ctx.scan(dev_colmajor(A), A.shape[0])


def test_fixtures(ctx, orc):
    for f in ("fig1_structures.json", "fig4_predicates.json"):
        for c in json.load(open(os.path.join(GOLDEN, f)))["cases"]:
            A = np.array([[float(eval(str(x), {"__builtins__": {}}, {"eps": EPS})) for x in r]
                          for r in c["rows"]])
            check_scan(single_scan(ctx, A), orc.scan(A), A)


@pytest.mark.parametrize("n", [1, 2, 3, 7, 31, 32, 33, 64, 65, 100, 257, 513, 1024, 1100, 2049])
def test_classes_many_sizes(ctx, orc, n):
    rng = np.random.default_rng(n)
    mats = []
    G = rng.standard_normal((n, n))
    mats.append(G)                                      # general
    S = G.T @ G / n + np.eye(n)
    mats.append(np.tril(S) + np.tril(S, -1).T)          # sympd
    mats.append(np.tril(G))                             # lower
    mats.append(np.triu(G, 1) + np.diag(np.abs(np.diag(G)) + 1))  # upper
    for kl, ku in ((0, 0), (1, 1), (2, 5), (n // 8, n // 9)):
        B = np.zeros((n, n))
        for d in range(-min(kl, n - 1), min(ku, n - 1) + 1):
            B += np.diag(rng.standard_normal(n - abs(d)), d)
        mats.append(B)
    Z = S.copy()
    Z[n // 2, n // 3] *= 1 + 1e-10                      # breaks symmetry beyond tol
    mats.append(Z)
    for A in mats:
        check_scan(single_scan(ctx, A), orc.scan(A), A)


def test_exhaustive_3x3_batched(ctx, orc):
    vals = np.array([-1.0, 0.0, 1.0, 2.0])
    idx = np.array(list(itertools.product(range(4), repeat=9)))
    As = vals[idx].reshape(-1, 3, 3)
    pk = pack_batch(list(As), [np.ones(3)] * len(As))
    _, infos = run_batch(ctx, pk)
    ref = orc.scan_many(As)
    for c in range(len(As)):
        i, r = infos[c], ref[c]
        if i["status"] == -2:
            continue
        assert (i["cls"], i["kl"], i["ku"]) == (r.cls, r.kl, r.ku), (As[c], i, r.cls)


def test_random_patterns_batched(ctx, orc):
    rng = np.random.default_rng(77)
    mats = []
    for trial in range(6000):
        n = int(rng.integers(4, 9))
        density = rng.uniform(0.05, 0.9)
        A = np.where(rng.uniform(size=(n, n)) < density,
                     rng.choice([-2.0, -1.0, 1.0, 3.0, 1e-300, 1e300], size=(n, n)), 0.0)
        if trial % 3 == 0:
            A = np.tril(A) + np.tril(A, -1).T
            np.fill_diagonal(A, rng.uniform(0.5, 9.0, n))
        mats.append(A)
    pk = pack_batch(mats, [np.ones(m.shape[0]) for m in mats])
    _, infos = run_batch(ctx, pk)
    for A, i in zip(mats, infos):
        r = orc.scan(A)
        assert (i["cls"], i["kl"], i["ku"]) == (r["cls"], r["kl"], r["ku"]), (A, i, r)


def test_nonfinite_detected(ctx, orc):
    A = np.eye(40)
    A[3, 30] = np.nan
    assert single_scan(ctx, A)["nonfinite"] == 1
    A[3, 30] = -np.inf
    assert single_scan(ctx, A)["nonfinite"] == 1
