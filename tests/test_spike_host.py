"""The partitioned band solve's per-thread routines (csrc/band_spike.cuh),
compiled as host C++ and run thread index by thread index (no GPU), against
the oracle: solves with A and with A^T on diagonally dominant band systems,
one-sided and diagonal bands, and the far-tip bound that decides whether
the truncated boundary systems are exact."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2007_11208_gb300", "csrc")


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("spike") / "libspike_host.so")
    subprocess.check_call([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-ffp-contract=off",
                           "-I" + CSRC, os.path.join(ROOT, "tests", "spike_host.cpp"), "-o", out])
    lib = C.CDLL(out)
    pd, i64 = C.POINTER(C.c_double), C.c_int64
    lib.spike_host_solve.argtypes = [pd, i64, C.c_int, C.c_int, i64, i64, pd, pd, pd, pd,
                                     C.POINTER(C.c_int), C.c_int]
    lib.spike_host_solve.restype = C.c_int
    return lib


def _p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def run(shim, AB, kl, ku, m, b, warp=0):
    """AB: (kl+ku+1, n) band storage, A(i,j) at AB[ku+i-j, j].  warp: the
    one-warp-per-block routines, lanes run phase by phase."""
    AB = np.asfortranarray(AB, dtype=np.float64)
    n = AB.shape[1]
    x, xt, far = np.zeros(n), np.zeros(n), np.zeros(2)
    dom = (C.c_int * 2)()
    rc = shim.spike_host_solve(_p(AB), AB.shape[0], kl, ku, n, m, _p(np.ascontiguousarray(b)), _p(x),
                               _p(xt), _p(far), dom, int(warp))
    return rc, x, xt, far, (dom[0], dom[1])


def dense(AB, kl, ku):
    n = AB.shape[1]
    A = np.zeros((n, n))
    for r in range(kl + ku + 1):
        d = r - ku  # i - j
        j = np.arange(max(0, -d), min(n, n - d))
        A[j + d, j] = AB[r, j]
    return A


def row_dominant(n, kl, ku, seed):
    from paper_2007_11208_gb300 import synth
    return np.ascontiguousarray(synth.band_storage_dd(n, kl, ku, synth.gen(seed)).numpy().T)


def check(orc, AB, kl, ku, x, xt, b):
    A = dense(AB, kl, ku)
    Xo, io = orc.solve_band(AB, kl, ku, b)
    assert io["status"] == 0
    Xt, it = orc.solve(A.T, b)
    assert it["status"] == 0
    _, be = orc.residual_dot2(A, x, b)
    _, bt = orc.residual_dot2(A.T, xt, b)
    assert be.max() <= 1e-14 and bt.max() <= 1e-14, (be, bt)
    assert np.abs(x - Xo[:, 0]).max() <= 1e-12 * np.abs(Xo).max()
    assert np.abs(xt - Xt[:, 0]).max() <= 1e-12 * np.abs(Xt).max()


@pytest.mark.parametrize("n,kl,ku,m", [(3000, 2, 2, 300), (3000, 8, 8, 375), (3000, 32, 32, 750),
                                       (2500, 3, 0, 250), (2500, 0, 5, 250), (2000, 7, 2, 333),
                                       (1999, 1, 9, 401)])
@pytest.mark.parametrize("warp", [0, 1, 3])
def test_row_dominant_bands_against_oracle(orc, shim, n, kl, ku, m, warp):
    AB = row_dominant(n, kl, ku, n + kl)
    b = np.random.default_rng(kl + 10 * ku).standard_normal(n)
    rc, x, xt, far, dom = run(shim, AB, kl, ku, m, b, warp)
    assert rc == 0 and dom[0] == 1
    assert far.max() < 1e-20, far  # truncation exact to rounding
    check(orc, AB, kl, ku, x, xt, b)


def test_diagonal_band(orc, shim):
    n = 1000
    AB = np.random.default_rng(1).uniform(1.0, 2.0, (1, n))
    b = np.arange(1.0, n + 1)
    rc, x, xt, far, dom = run(shim, AB, 0, 0, 100, b)
    assert rc == 0 and dom == (1, 1) and far.max() == 0.0
    assert np.allclose(x, b / AB[0], rtol=1e-15) and np.allclose(xt, b / AB[0], rtol=1e-15)


def test_column_dominant_band(orc, shim):
    n, kl, ku = 2400, 4, 6
    rng = np.random.default_rng(7)
    A = dense(rng.standard_normal((kl + ku + 1, n)), kl, ku)
    np.fill_diagonal(A, 0.0)
    np.fill_diagonal(A, 1.0 + np.abs(A).sum(axis=0))
    AB = np.zeros((kl + ku + 1, n))
    for r in range(kl + ku + 1):
        d = r - ku
        j = np.arange(max(0, -d), min(n, n - d))
        AB[r, j] = A[j + d, j]
    b = rng.standard_normal(n)
    for warp in (1, 3):
        rc, x, xt, far, dom = run(shim, AB, kl, ku, 300, b, warp=warp)
        assert rc == 0 and dom[1] == 1
        assert far.max() < 1e-20, far
        check(orc, AB, kl, ku, x, xt, b)


def test_far_tips_flag_short_blocks(shim):
    """With blocks too short for the spikes to decay, the far tips are far
    from negligible: the bound is what tells the two cases apart."""
    n, k = 2000, 8
    AB = row_dominant(n, k, k, 3)
    b = np.ones(n)
    for warp in (0, 3):
        rc, x, xt, far, dom = run(shim, AB, k, k, 40, b, warp)
        assert rc == 0 and far.max() > 1e-12, far
        rc, x, xt, far, dom = run(shim, AB, k, k, 500, b, warp)
        assert rc == 0 and far.max() < 1e-20, far


def test_zero_pivot_reports_the_block(shim):
    n, k = 600, 2
    AB = row_dominant(n, k, k, 4)
    AB[k, 450] = 0.0  # column 450: block 3 (0-based) of 4, m = 150
    AB[:, 450] = 0.0
    for warp in (0, 3):
        rc, *_ = run(shim, AB, k, k, 150, np.ones(n), warp)
        assert rc == -1 - 3


def test_warp_and_thread_routines_agree(shim):
    """The two versions take the same arithmetic steps per element (only the
    order of the dot-product sums of the transposed solve differs)."""
    n, k = 3000, 20
    AB = row_dominant(n, k, k, 9)
    b = np.random.default_rng(9).standard_normal(n)
    r1 = run(shim, AB, k, k, 700, b, warp=False)
    r2 = run(shim, AB, k, k, 700, b, warp=True)
    assert r1[0] == r2[0] == 0
    assert np.array_equal(r1[1], r2[1])
    assert np.abs(r1[2] - r2[2]).max() <= 1e-14 * np.abs(r1[2]).max()


@pytest.mark.parametrize("kl,ku,mode", [(20, 20, 1), (40, 5, 1), (3, 37, 1), (70, 70, 1),
                                        (20, 20, 3), (32, 32, 3), (31, 2, 3), (1, 30, 3)])
def test_warp_phases_do_not_depend_on_lane_order(shim, kl, ku, mode):
    """Within a phase no lane reads what another lane writes: running the
    lanes of every phase in the opposite order gives the same bits."""
    n = 4000
    AB = row_dominant(n, kl, ku, kl + ku)
    b = np.random.default_rng(kl).standard_normal(n)
    m = max(16 * (kl + ku), 256)
    fwd = run(shim, AB, kl, ku, m, b, warp=mode)
    rev = run(shim, AB, kl, ku, m, b, warp=mode + 1)
    assert fwd[0] == rev[0] == 0
    assert np.array_equal(fwd[1], rev[1]) and np.array_equal(fwd[2], rev[2])


def test_dominance_flags_refuse_a_plain_random_band(shim):
    """A band with N(0,1) entries and no boosted diagonal is dominant
    neither by rows nor by columns: the route is not taken for it."""
    n, k = 3000, 4
    AB = np.random.default_rng(12).standard_normal((2 * k + 1, n))
    rc, x, xt, far, dom = run(shim, AB, k, k, 300, np.ones(n))
    assert dom == (0, 0)
    # the one-sided case: dominance by rows is exactly diag >= sum of the row
    AB = row_dominant(n, k, k, 5)
    AB[k, 1234] *= 0.5  # one row loses its dominance
    rc, x, xt, far, dom = run(shim, AB, k, k, 300, np.ones(n))
    assert dom[0] == 0


@pytest.mark.parametrize("n,kl,ku,m", [(4000, 32, 32, 1024), (3001, 17, 9, 433), (2600, 1, 1, 130)])
def test_window_routines_against_oracle_and_the_per_thread_ones(orc, shim, n, kl, ku, m):
    """The bands-up-to-32 routines (window spikes, per-column block
    factorisation, one warp per boundary system) against the oracle, and
    their boundary systems' far tips against the per-thread routines'."""
    AB = row_dominant(n, kl, ku, n + kl + 3)
    b = np.random.default_rng(n).standard_normal(n)
    r0 = run(shim, AB, kl, ku, m, b, 0)
    r3 = run(shim, AB, kl, ku, m, b, 3)
    assert r0[0] == r3[0] == 0
    check(orc, AB, kl, ku, r3[1], r3[2], b)
    assert np.abs(r0[1] - r3[1]).max() <= 1e-13 * np.abs(r0[1]).max()
    assert np.abs(r0[3] - r3[3]).max() <= 1e-6 * np.abs(r0[3]).max() + 1e-300, (r0[3], r3[3])
