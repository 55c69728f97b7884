"""Pins for the oracle's property scan and routing (paper Sec. 2.1, 2.2, Fig. 4).

Every expected value here comes from the paper (Fig. 1, Fig. 4 fixtures under
tests/golden/) or from an independent brute-force definition written with
numpy set operations -- never from the oracle itself.
"""
import itertools
import json
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EPS = np.finfo(np.float64).eps
CLS = {"NONE": 0, "BANDED": 1, "LOWER": 2, "UPPER": 3, "SYMPD": 4, "GENERAL": 5}


def _entry(s):
    return float(eval(str(s), {"__builtins__": {}}, {"eps": EPS}))


def brute_scan(A, band_frac=0.25, tol=100 * EPS):
    """Definition-level restatement: bandwidth = largest |i-j| over non-zeros
    on each side, triangularity by masks, likely_sympd as set predicates."""
    n = A.shape[0]
    i, j = np.indices((n, n))
    nz = A != 0.0
    kl = int(np.max(np.where(nz & (i > j), i - j, 0), initial=0))
    ku = int(np.max(np.where(nz & (i < j), j - i, 0), initial=0))
    lower = not np.any(nz & (i < j))
    upper = not np.any(nz & (i > j))
    d = np.diag(A)
    if n == 0 or np.any(d <= 0):
        sympd = False
    else:
        md = d.max()
        low = i > j
        a, at = A[low], A.T[low]
        delta = np.abs(a - at)
        sym_bad = (delta > tol) & (delta > tol * np.maximum(np.abs(a), np.abs(at)))
        mod_bad = np.abs(a) >= md
        dom_bad = (np.abs(a) + np.abs(at)) >= (d[i[low]] + d[j[low]])
        sympd = not (sym_bad.any() or mod_bad.any() or dom_bad.any())
    # band positions counted one by one
    cnt = int(np.sum((i - j <= kl) & (j - i <= ku)))
    banded = cnt <= band_frac * n * n
    if n == 0:
        cls = 0
    elif banded:
        cls = 1
    elif lower:
        cls = 2
    elif upper:
        cls = 3
    elif sympd:
        cls = 4
    else:
        cls = 5
    return dict(kl=kl, ku=ku, lower=int(lower), upper=int(upper), sympd=int(sympd),
                banded=int(banded), cls=cls)


def test_fig1_structures(orc):
    cases = json.load(open(os.path.join(GOLDEN, "fig1_structures.json")))["cases"]
    for c in cases:
        A = np.array(c["rows"], dtype=np.float64)
        s = orc.scan(A)
        assert (s["kl"], s["ku"]) == (c["kl"], c["ku"]), c["name"]
        assert bool(s["lower"]) == c["lower"] and bool(s["upper"]) == c["upper"], c["name"]
        assert bool(s["sympd"]) == c["sympd"], c["name"]
        assert bool(s["banded"]) == c["banded"], c["name"]
        assert s["cls"] == CLS[c["cls"]], c["name"]


def test_fig4_predicates(orc):
    cases = json.load(open(os.path.join(GOLDEN, "fig4_predicates.json")))["cases"]
    for c in cases:
        A = np.array([[_entry(x) for x in r] for r in c["rows"]], dtype=np.float64)
        assert orc.likely_sympd(A) == c["likely_sympd"], c["name"]
        assert bool(brute_scan(A)["sympd"]) == c["likely_sympd"], c["name"]


def test_band_count_closed_form(orc):
    for n in range(0, 13):
        i, j = np.indices((n, n))
        for kl in range(0, max(n, 1)):
            for ku in range(0, max(n, 1)):
                cnt = int(np.sum((i - j <= kl) & (j - i <= ku)))
                assert orc.band_count(n, kl, ku) == cnt, (n, kl, ku)


def test_band_rule_boundaries(orc):
    # diagonal: banded only from n = 4 (n positions <= n^2/4)
    for n in range(1, 9):
        s = orc.scan(np.diag(np.arange(1.0, n + 1)))
        assert s["banded"] == (n >= 4)
        assert s["cls"] == (CLS["BANDED"] if n >= 4 else CLS["LOWER"])
    # tridiagonal: 3n-2 positions <= n^2/4  <=>  n >= 12
    for n in range(2, 16):
        A = np.diag(np.full(n, 4.0)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)
        assert orc.scan(A)["banded"] == (n >= 12), n
    # bands of half-width k at n = 16, 32, 64, 100: largest banded k is 1, 3, 8, 12
    for n, kmax in ((16, 1), (32, 3), (64, 8), (100, 12)):
        for k in range(0, kmax + 3):
            A = np.zeros((n, n))
            for d in range(-k, k + 1):
                A += np.diag(np.ones(n - abs(d)), d)
            assert bool(orc.scan(A)["banded"]) == (k <= kmax), (n, k)


def test_zero_and_signed_zero(orc):
    A = np.eye(5)
    A[0, 4] = -0.0          # negative zero is zero
    A[4, 0] = np.nextafter(0, 1)  # smallest subnormal is not zero
    s = orc.scan(A)
    assert s["ku"] == 0 and s["kl"] == 4


def test_nonfinite_flag(orc):
    A = np.eye(4)
    A[2, 1] = np.nan
    assert orc.scan(A)["nonfinite"] == 1
    A[2, 1] = np.inf
    assert orc.scan(A)["nonfinite"] == 1
    assert orc.scan(np.eye(4))["nonfinite"] == 0


def test_norms(orc):
    rng = np.random.default_rng(1)
    A = rng.standard_normal((7, 7))
    assert orc.norm1(A) == pytest.approx(np.abs(A).sum(axis=0).max(), rel=1e-15)
    assert orc.norminf(A) == pytest.approx(np.abs(A).sum(axis=1).max(), rel=1e-15)


def test_exhaustive_3x3(orc):
    vals = np.array([-1.0, 0.0, 1.0, 2.0])
    idx = np.array(list(itertools.product(range(4), repeat=9)))
    As = vals[idx].reshape(-1, 3, 3)
    out = orc.scan_many(As)
    mism = 0
    for c in range(As.shape[0]):
        b = brute_scan(As[c])
        s = out[c]
        got = dict(kl=s.kl, ku=s.ku, lower=s.lower, upper=s.upper, sympd=s.sympd,
                   banded=s.banded, cls=s.cls)
        if got != b:
            mism += 1
            assert got == b, (As[c], got, b)
    assert mism == 0


@pytest.mark.parametrize("n", [4, 5, 6])
def test_random_sparsity_patterns(orc, n):
    rng = np.random.default_rng(100 + n)
    for trial in range(3000):
        density = rng.uniform(0.05, 0.9)
        A = np.where(rng.uniform(size=(n, n)) < density,
                     rng.choice([-2.0, -1.0, 1.0, 3.0], size=(n, n)), 0.0)
        if trial % 3 == 0:
            A = np.tril(A) + np.tril(A, -1).T  # symmetric patterns
            np.fill_diagonal(A, rng.uniform(0.5, 9.0, n))
        s = orc.scan(A)
        b = brute_scan(A)
        for k in b:
            assert s[k] == b[k], (k, A)
