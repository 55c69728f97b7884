"""The synthetic inputs follow the recipes the benchmark states (no GPU):
the batched mix, the size and right-hand-side ranges, the structure of each
class, and determinism under a seed."""
import numpy as np

from paper_2007_11208_gb300 import synth


def test_batch_mix_and_ranges():
    specs = synth.batch_specs(10000, 1)
    kinds = [s[0] for s in specs]
    for kind, p in synth.BATCH_MIX:
        frac = kinds.count(kind) / len(specs)
        assert abs(frac - p) < 0.02, (kind, frac, p)
    ns = np.array([s[1] for s in specs])
    rs = np.array([s[2] for s in specs])
    assert ns.min() >= 16 and ns.max() <= 512 and abs(ns.mean() - 264) < 5
    assert rs.min() >= 1 and rs.max() <= 8 and set(rs.tolist()) == set(range(1, 9))
    for s in specs:
        if s[0] == "banded":
            assert 1 <= s[3] <= 16 and 1 <= s[4] <= 16


def test_batch_is_deterministic_under_its_seed():
    a = synth.packed_batch(synth.batch_specs(20, 5), 9)
    b = synth.packed_batch(synth.batch_specs(20, 5), 9)
    assert all(np.array_equal(a[k].numpy(), b[k].numpy()) for k in ("A", "B", "n", "a_off"))


def test_class_structures():
    g = synth.gen(3)
    n = 40
    lower = synth.colmajor_to_dense(synth.tri_dd(n, g, lower=True)).numpy()
    assert np.array_equal(lower, np.tril(lower))
    assert np.all(np.diag(lower) >= 1 + np.abs(np.tril(lower, -1)).sum(1) - 1e-12)
    spd = synth.colmajor_to_dense(synth.spd(n, g)).numpy()
    assert np.array_equal(spd, spd.T) and np.linalg.eigvalsh(spd).min() > 0
    band = synth.colmajor_to_dense(synth.banded_dd(n, 3, 5, g)).numpy()
    i, j = np.nonzero(band)
    assert (i - j).max() == 3 and (j - i).max() == 5
    off = np.abs(band).sum(1) - np.abs(np.diag(band))
    assert np.all(np.abs(np.diag(band)) > off)


def test_spectrum_fast_has_the_stated_condition_number():
    for spd in (False, True):
        M = synth.spectrum_fast(300, synth.gen(4), 1e6, spd=spd)
        A = synth.colmajor_to_dense(M).numpy()
        s = np.linalg.svd(A, compute_uv=False)
        assert abs(s[0] / s[-1] / 1e6 - 1) < 1e-9
        if spd:
            assert np.array_equal(A, A.T)
