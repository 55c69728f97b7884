"""Parity at the benchmark's full sizes, in the launch configuration that
bench.py times.

* The 10,000-system headline batch (bench.py's generator, seed, precision,
  panel-width table and flags), launched as one batched call: every system
  is verified by the library's in-kernel FP64 backward error, and one
  system in 97 is compared with the oracle one by one (class, kl/ku, route
  and status bit-exact; X within 2^-52 n kappa_inf of the oracle's X; the
  oracle's compensated residual for the backward error).
* Single dense systems of the large configuration (general n = 16384 and
  SPD n = 8192, kappa 1e4, one right-hand side, mixed precision, the
  bench's seeds): beyond the oracle's O(n^3) solve in a test, so they are
  checked through properties that hold at any size -- the oracle's
  compensated residual bounds the backward error, and a known solution the
  forward error (kappa_inf <= n kappa_2 by construction).

The file is collected last (after test_zz_no_alloc.py): the largest runs,
and a failure here leaves every other test already run.
"""
import os

import numpy as np
import pytest
import torch

from gpu_util import fwd_err, kappa_inf

pytestmark = pytest.mark.gpu
BERR = 1e-13
EPS = np.finfo(np.float64).eps


def test_headline_batch_sampled_against_oracle(orc):
    import bench
    from paper_2007_11208_gb300 import asolve, build
    build.build()
    dev = torch.device("cuda", 0)
    count = bench.COUNT
    pk = bench.make_batch(dev, bench.rank_seed(0), count)
    tuning = bench.TUNING if os.path.exists(bench.TUNING) else None
    ctx = asolve.Context(precision=asolve.PREC_MIXED, tuning=tuning)
    X = torch.zeros_like(pk["B"])
    infos = torch.zeros(count * asolve.INFO_BYTES, dtype=torch.uint8, device=dev)
    rc = ctx.solve_batched(count, pk["n"], pk["nrhs"], pk["a_off"], pk["b_off"], pk["A"], pk["B"], X, infos,
                           asolve.BERR | asolve.SYNC)
    assert rc == 0, rc
    torch.cuda.synchronize()
    inf = asolve.infos_from_tensor(infos)
    assert len(inf) == count
    bad = [s for s, i in enumerate(inf) if not (i["status"] == 0 and i["berr"] <= BERR)]
    assert not bad, [(s, inf[s]) for s in bad[:5]]
    specs = pk["specs"]
    routes = set()
    for s in range(0, count, 97):
        n, r = specs[s][1], specs[s][2]
        o, q = int(pk["a_off_h"][s]), int(pk["b_off_h"][s])
        A = pk["A"][o:o + n * n].cpu().numpy().reshape(n, n).T
        B = pk["B"][q:q + n * r].cpu().numpy().reshape(r, n).T
        Xg = X[q:q + n * r].cpu().numpy().reshape(r, n).T
        Xo, io = orc.solve(A, B)
        i = inf[s]
        assert (i["cls"], i["kl"], i["ku"], i["route"], i["status"]) == \
            (io["cls"], io["kl"], io["ku"], io["route"], io["status"]), (s, i, io)
        routes.add(i["route"])
        assert fwd_err(Xg, Xo) <= 2.0 ** -52 * n * kappa_inf(A), (s, i, fwd_err(Xg, Xo))
        _, berr = orc.residual_dot2(A, Xg, B)
        assert berr.max() <= BERR, (s, i, berr)
    assert {1, 2, 4, 6} <= routes, routes
    ctx.close()


@pytest.mark.parametrize("kind,n", [("general", 16384), ("spd", 8192)])
def test_large_configuration_full_size(orc, kind, n):
    from paper_2007_11208_gb300 import asolve, build, synth
    build.build()
    dev = torch.device("cuda", 0)
    kappa = 1e4
    g = synth.gen(int(n + 17 * kappa) % 100003, dev)  # bench.py's seed for this case
    M = synth.spectrum_fast(n, g, kappa, spd=(kind == "spd"), device=dev)  # M[j, i] = A[i, j]
    xt = synth.rhs(n, 1, g, dev)                                          # known solution, (1, n)
    B = (M.t() @ xt.t()).t().contiguous()                                 # A x_true
    X = torch.zeros_like(B)
    ctx = asolve.Context(precision=asolve.PREC_MIXED)
    rc, info = ctx.solve(M, B, n, 1, X, asolve.BERR)
    torch.cuda.synchronize()
    assert rc == 0, (rc, info)
    assert info["route"] == (asolve.ROUTE_CHOL if kind == "spd" else asolve.ROUTE_LU), info
    assert info["berr"] <= BERR, info
    A = M.cpu().numpy().T
    sr = orc.scan(A)  # the oracle's scan of the bytes the GPU read (Sec. 2.1-2.3, Fig. 4)
    assert (info["cls"], info["kl"], info["ku"]) == (sr["cls"], sr["kl"], sr["ku"]), (info, sr)
    x = X.cpu().numpy().reshape(n, 1)
    b = B.cpu().numpy().reshape(n, 1)
    x_true = xt.cpu().numpy().reshape(n, 1)
    _, berr = orc.residual_dot2(A, x, b)
    assert berr.max() <= BERR, berr
    assert np.abs(x - x_true).max() / np.abs(x_true).max() <= EPS * n * (n * kappa)
    ctx.close()


@pytest.mark.parametrize("k", [2, 8, 32])
def test_band_configuration_full_size(orc, k):
    """The band configuration exactly as bench.py times it (n = 10^6 in band
    storage, kl = ku = k, the bench's seed, diagonally dominant, default
    route): class, route and bandwidths equal to the oracle's band driver,
    X within the forward-error bound of the oracle's X (kappa_inf estimated
    from the oracle's rcond, times n), rcond within 1e-5 relative, backward
    error <= 1e-13 by the oracle's compensated residual over the band."""
    from paper_2007_11208_gb300 import asolve, build, synth
    build.build()
    dev = torch.device("cuda", 0)
    n = 1_000_000
    g = synth.gen(1000 + k, dev)
    AB = synth.band_storage_dd(n, k, k, g, device=dev)   # row j = column j of the band layout
    Bm = synth.rhs(n, 1, g, dev)
    X = torch.zeros_like(Bm)
    ctx = asolve.Context()
    rc, info = ctx.solve_band(AB, 2 * k + 1, k, k, Bm, n, 1, X, asolve.BERR)
    torch.cuda.synchronize()
    ABh = np.asfortranarray(AB.cpu().numpy().T)         # LAPACK layout (2k+1, n)
    bh = Bm.cpu().numpy().reshape(n, 1)
    Xo, io = orc.solve_band(ABh, k, k, bh)
    assert rc == io["status"] == 0, (rc, info, io)
    assert (info["cls"], info["route"], info["kl"], info["ku"]) == \
        (io["cls"], io["route"], io["kl"], io["ku"]), (info, io)
    assert info["detail"] & 16, info                      # the partitioned route took it
    x = X.cpu().numpy().reshape(n, 1)
    kinf = n / io["rcond"]                                # kappa_inf <= n kappa_1
    assert np.abs(x - Xo).max() / np.abs(Xo).max() <= EPS * n * kinf
    assert abs(info["rcond"] - io["rcond"]) <= 1e-5 * io["rcond"], (info["rcond"], io["rcond"])
    assert info["berr"] <= BERR, info
    # the oracle's own backward error of the GPU's X, from the band
    rows = np.zeros(n)
    absrow = np.zeros(n)
    for r in range(2 * k + 1):
        j = np.arange(n)
        i = r - k + j
        ok = (i >= 0) & (i < n)
        v = ABh[r, j[ok]] * x[j[ok], 0]
        np.add.at(rows, i[ok], v)
        np.add.at(absrow, i[ok], np.abs(ABh[r, j[ok]]))
    resid = np.abs(bh[:, 0] - rows).max()
    berr = resid / (absrow.max() * np.abs(x).max() + np.abs(bh).max())
    assert berr <= BERR, berr
    ctx.close()
