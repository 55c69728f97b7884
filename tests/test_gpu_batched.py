"""Batched class-routed pipeline: every system of a mixed batch matches the
oracle (class, kl/ku, route bit-exact; X within the forward-error bound), the
pipeline is deterministic, each system's result is the same alone and in the
mix, and the host-buffer entry gives the same bytes."""
import numpy as np
import pytest
import torch

from gpu_util import fwd_err, kappa_inf, pack_batch, run_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["fp64", "mixed"])
def ctx(request):
    from paper_2007_11208_gb300 import asolve, build
    build.build()
    prec = asolve.PREC_FP64 if request.param == "fp64" else asolve.PREC_MIXED
    c = asolve.Context(precision=prec)
    yield c
    c.close()


def batch(seed, count, nmax=200):
    from paper_2007_11208_gb300 import synth
    specs = synth.batch_specs(count, seed, nmin=1, nmax=nmax)
    g = synth.gen(seed + 1)
    mats, rhss = [], []
    for sp in specs:
        mats.append(synth.batch_matrix(sp, g).numpy().T.copy())
        rhss.append(synth.rhs(sp[1], sp[2], g).numpy().T.copy())
    return mats, rhss


def test_batch_matches_oracle(ctx, orc):
    mats, rhss = batch(3, 160)
    pk = pack_batch(mats, rhss)
    Xs, infos = run_batch(ctx, pk)
    routes = set()
    for A, B, X, inf in zip(mats, rhss, Xs, infos):
        Xo, io = orc.solve(A, B)
        assert (inf["cls"], inf["kl"], inf["ku"], inf["route"]) == \
            (io["cls"], io["kl"], io["ku"], io["route"]), (inf, io)
        assert inf["status"] == io["status"], (inf, io)
        routes.add(inf["route"])
        if io["status"] == 0:
            n = A.shape[0]
            assert fwd_err(X, Xo) <= 2.0 ** -52 * n * kappa_inf(A), (inf, fwd_err(X, Xo))
    assert {1, 2, 3, 4, 6} <= routes or len(routes) >= 4, routes


def test_deterministic_and_alone_vs_mix(ctx, orc):
    mats, rhss = batch(4, 64, nmax=300)
    pk = pack_batch(mats, rhss)
    X1, i1 = run_batch(ctx, pk)
    X2, i2 = run_batch(ctx, pk)
    for a, b in zip(X1, X2):
        assert np.array_equal(a, b)
    for s in (0, 7, 33):
        pk1 = pack_batch([mats[s]], [rhss[s]])
        Xa, ia = run_batch(ctx, pk1)
        assert np.array_equal(Xa[0], X1[s]), s
        assert ia[0]["route"] == i1[s]["route"]


def test_host_buffers_same_bytes(ctx):
    from paper_2007_11208_gb300 import asolve
    mats, rhss = batch(5, 40)
    pk = pack_batch(mats, rhss)
    Xd, idev = run_batch(ctx, pk)
    n = pk["n"].cpu().numpy()
    r = pk["nrhs"].cpu().numpy()
    ao = pk["a_off"].cpu().numpy()
    bo = pk["b_off"].cpu().numpy()
    A = pk["A"].cpu().numpy()
    B = pk["B"].cpu().numpy()
    X = np.zeros_like(B)
    infos = np.zeros(len(mats) * asolve.INFO_BYTES, dtype=np.uint8)
    rc = ctx.solve_batched(len(mats), n.ctypes.data, r.ctypes.data, ao.ctypes.data, bo.ctypes.data,
                           A.ctypes.data, B.ctypes.data, X.ctypes.data, infos.ctypes.data,
                           asolve.HOST_BUFFERS)
    assert rc == 0
    for s in range(len(mats)):
        q = pk["b_off_h"][s]
        got = X[q:q + n[s] * r[s]].reshape(r[s], n[s]).T
        assert np.array_equal(got, Xd[s])
    ih = asolve.infos_from_tensor(torch.from_numpy(infos))
    assert [i["route"] for i in ih] == [i["route"] for i in idev]


def test_host_buffers_shuffled_layout(ctx):
    """A host-buffer batch of 2,600 systems stored in shuffled order (offsets
    not increasing with the system index) gives the same bytes as the
    device-buffer call."""
    from paper_2007_11208_gb300 import asolve
    rng = np.random.default_rng(12)
    count = 2600
    mats, rhss = [], []
    for s in range(count):
        n = int(rng.integers(4, 24))
        mats.append(rng.standard_normal((n, n)) + 2 * np.sqrt(n) * np.eye(n))
        rhss.append(rng.standard_normal((n, 1 + s % 3)))
    order = rng.permutation(count)  # storage order of the blocks
    pk = pack_batch([mats[i] for i in order], [rhss[i] for i in order])
    pos = np.empty(count, dtype=np.int64)
    pos[order] = np.arange(count)  # system s is stored as block pos[s]
    n = np.array([mats[s].shape[0] for s in range(count)], dtype=np.int64)
    r = np.array([rhss[s].shape[1] for s in range(count)], dtype=np.int64)
    ao = np.array([pk["a_off_h"][pos[s]] for s in range(count)], dtype=np.int64)
    bo = np.array([pk["b_off_h"][pos[s]] for s in range(count)], dtype=np.int64)
    A = pk["A"].cpu().numpy()
    B = pk["B"].cpu().numpy()
    Xh = np.zeros_like(B)
    ih = np.zeros(count * asolve.INFO_BYTES, dtype=np.uint8)
    rc = ctx.solve_batched(count, n.ctypes.data, r.ctypes.data, ao.ctypes.data, bo.ctypes.data, A.ctypes.data,
                           B.ctypes.data, Xh.ctypes.data, ih.ctypes.data, asolve.HOST_BUFFERS)
    assert rc == 0
    dn, dr, dao, dbo = (torch.from_numpy(a).cuda() for a in (n, r, ao, bo))
    Xd = torch.zeros_like(pk["B"])
    idv = torch.zeros(count * asolve.INFO_BYTES, dtype=torch.uint8, device="cuda")
    rc = ctx.solve_batched(count, dn, dr, dao, dbo, pk["A"], pk["B"], Xd, idv, asolve.SYNC)
    assert rc == 0
    assert np.array_equal(Xh, Xd.cpu().numpy())
    assert np.array_equal(ih, idv.cpu().numpy())


def test_invalid_entries(ctx):
    mats = [np.eye(4), np.eye(3)]
    pk = pack_batch(mats, [np.ones(4), np.ones(3)])
    pk["n"][1] = 2000  # beyond the batched limit
    Xs, infos = run_batch(ctx, pk)
    assert infos[0]["status"] == 0 and infos[1]["status"] == -8
