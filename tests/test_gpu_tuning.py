"""GPU tests of the panel-width autotuner: the knob is validated, any
admissible table leaves every answer within the parity bar, and the tuner
produces a table of admissible widths."""
import numpy as np
import pytest
import torch

from gpu_util import pack_batch, run_batch

pytestmark = pytest.mark.gpu


def _mats(rng, n, count):
    out = []
    for i in range(count):
        if i % 2:
            G = rng.standard_normal((n, n))
            S = G.T @ G / n + np.eye(n)
            out.append(np.tril(S) + np.tril(S, -1).T)
        else:
            out.append(rng.standard_normal((n, n)) + 2 * np.sqrt(n) * np.eye(n))
    return out


def test_set_panel_widths_validation():
    from paper_2007_11208_gb300 import asolve, build
    build.build()
    ctx = asolve.Context()
    assert ctx.set_panel_widths(0, [8] * 32) == asolve.OK
    assert ctx.set_panel_widths(0, [12]) == asolve.E_INVALID
    assert ctx.set_panel_widths(4, [8]) == asolve.E_INVALID
    assert ctx.set_panel_widths(1, [8] * 33) == asolve.E_INVALID
    assert ctx.set_panel_widths(3, []) == asolve.OK
    ctx.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_widths_keep_parity(orc, prec):
    from paper_2007_11208_gb300 import asolve
    rng = np.random.default_rng(17)
    mats = _mats(rng, 200, 6) + _mats(rng, 37, 4) + _mats(rng, 511, 2)
    rhs = [rng.standard_normal((A.shape[0], 2)) for A in mats]
    pk = pack_batch(mats, rhs)
    p = asolve.PREC_MIXED if prec == "mixed" else asolve.PREC_FP64
    for widths in (4, 8, 16):
        ctx = asolve.Context(precision=p)
        for kind in range(4):
            assert ctx.set_panel_widths(kind, [widths] * 32) == asolve.OK
        X, infos = run_batch(ctx, pk, asolve.BERR)
        ctx.close()
        for A, B, x, inf in zip(mats, rhs, X, infos):
            _, io = orc.solve(A, B)
            assert inf["status"] == io["status"] == 0
            assert inf["route"] == io["route"]
            assert inf["berr"] <= 1e-13


def test_autotune_small(tmp_path):
    from paper_2007_11208_gb300 import autotune
    res = autotune.tune(buckets=[1, 6], kinds=["lu32", "chol64"], reps=1)
    for key in ("lu32", "chol64"):
        assert res["nb"][key][1] in autotune.CANDIDATES and res["nb"][key][6] in autotune.CANDIDATES
    import json
    p = tmp_path / "t.json"
    p.write_text(json.dumps(res))
    from paper_2007_11208_gb300 import asolve
    ctx = asolve.Context(tuning=str(p))
    ctx.close()
