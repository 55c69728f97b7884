"""Dense band systems of order 2048 <= n < 4096 whose rows are scaled over
several decades (the serving workload's banded requests, kappa up to
1e12): they take the band route's partitioned sweeps, whose chained
transfer matrices can amplify rounding when the band is not dominant.  The
route keeps their answer only below a backward error of 2^-46 and else
solves again (see below).  Bar:
class, route and bandwidths as the oracle's, backward error <= 1e-13 by the
oracle's compensated residual, X within the forward-error bound.  (Short of
2^-46 the route first refines the sweeps' answer in FP64 with the same
sweeps, detail bit 7, and only then solves sequentially, bit 8.)"""
import numpy as np
import pytest
import torch

from gpu_util import kappa_inf, solve_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,kl,ku,kappa", [(2361, 5, 12, 2.4e6), (2361, 15, 2, 1e9), (3001, 9, 9, 1e11),
                                           (2048, 1, 16, 1e6), (3500, 13, 13, 1e4)])
def test_scaled_dense_bands(orc, n, kl, ku, kappa):
    from paper_2007_11208_gb300 import asolve, build, synth
    build.build()
    g = synth.gen(n + 100 * kl + ku)
    A = synth.colmajor_to_dense(synth.banded_kappa(n, kl, ku, g, kappa)).numpy()
    rng = np.random.default_rng(n + kl)
    B = rng.standard_normal((n, 2))
    ctx = asolve.Context()
    rc, info, X = solve_gpu(ctx, A, B, asolve.BERR)
    ctx.close()
    Xo, io = orc.solve(A, B)
    assert (info["cls"], info["route"], info["kl"], info["ku"]) == (io["cls"], io["route"], io["kl"], io["ku"]), \
        (info, io)
    assert rc == io["status"] == 0, (rc, info)
    _, berr = orc.residual_dot2(A, X, B)
    assert berr.max() <= 1e-13, (berr, info)
    assert info["berr"] <= 1e-13, info
    assert np.abs(X - Xo).max() / np.abs(Xo).max() <= 2.0 ** -52 * n * kappa_inf(A), info
