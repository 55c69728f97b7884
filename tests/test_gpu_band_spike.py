"""GPU parity of the partitioned route for diagonally dominant bands
(band_spike.cuh; the default for long dominant bands, turned off by
ASOLVE_BAND_SPIKE=0 in the environment, which skips these tests).

Same bar as the GBTRF-order route (test_gpu_band.py): class, route and
bandwidths identical to the oracle's, X within the forward-error bound,
rcond within 1e-5 relative, backward error <= 1e-13; plus which route ran
(asolve_info.detail bit 4)."""
import os

import numpy as np
import pytest

from test_gpu_band import band_storage, check_against_oracle, solve_band_gpu

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(os.environ.get("ASOLVE_BAND_SPIKE") == "0",
                                 reason="the partitioned band route is turned off by ASOLVE_BAND_SPIKE=0")]


@pytest.fixture(scope="module")
def ctx():
    from paper_2007_11208_gb300 import asolve, build
    build.build()
    c = asolve.Context()
    yield c
    c.close()


@pytest.mark.parametrize("n,kl,ku,nrhs", [(20011, 3, 4, 5), (100000, 2, 2, 1), (100000, 8, 8, 3),
                                          (100000, 32, 32, 1), (65537, 0, 6, 2), (65537, 5, 0, 2),
                                          (77777, 31, 17, 2), (40000, 1, 1, 1), (50001, 33, 3, 1),
                                          (1000000, 8, 8, 2)])
def test_dominant_bands_take_the_partitioned_route(ctx, orc, n, kl, ku, nrhs):
    from paper_2007_11208_gb300 import asolve
    rng = np.random.default_rng(n + 31 * kl + ku)
    AB, kld, kud = band_storage(n, kl, ku, rng, extra=(1, 0))
    B = rng.standard_normal((n, nrhs))
    rc, info, X = solve_band_gpu(ctx, AB, kld, kud, B, asolve.BERR)
    assert info["detail"] & 16, info
    check_against_oracle(orc, AB, kld, kud, B, rc, info, X, berr=True)


@pytest.mark.parametrize("n,kl,ku,dominant", [(5000, 4, 4, False), (3000, 2, 2, True)])
def test_other_bands_keep_the_gbtrf_order_route(ctx, orc, n, kl, ku, dominant):
    """Not dominant, or shorter than the partitioned route's minimum."""
    from paper_2007_11208_gb300 import asolve
    rng = np.random.default_rng(n + kl)
    AB, kld, kud = band_storage(n, kl, ku, rng, dominant=dominant)
    B = rng.standard_normal((n, 2))
    rc, info, X = solve_band_gpu(ctx, AB, kld, kud, B, asolve.BERR)
    assert not info["detail"] & 16, info
    check_against_oracle(orc, AB, kld, kud, B, rc, info, X, berr=True)
