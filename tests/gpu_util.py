"""Helpers shared by the GPU parity tests (marshalling between numpy, torch
and the C ABI; tolerance formulas)."""
import numpy as np
import torch

EPS = np.finfo(np.float64).eps


def dev_colmajor(A):
    """numpy (n, n) dense -> CUDA tensor holding A column-major."""
    return torch.from_numpy(np.ascontiguousarray(np.asarray(A, dtype=np.float64).T)).cuda()


def dev_rhs(B, n):
    B = np.asarray(B, dtype=np.float64).reshape(n, -1)
    return torch.from_numpy(np.ascontiguousarray(B.T)).cuda(), B.shape[1]


def host_from_dev(X, n, nrhs):
    return X.cpu().numpy().reshape(nrhs, n).T


def solve_gpu(ctx, A, B, flags=0):
    n = A.shape[0]
    dA = dev_colmajor(A)
    dB, nrhs = dev_rhs(B, n)
    dX = torch.zeros_like(dB)
    rc, info = ctx.solve(dA, dB, n, nrhs, dX, flags)
    return rc, info, host_from_dev(dX, n, nrhs)


def kappa_inf(A):
    return np.linalg.norm(A, np.inf) * np.linalg.norm(np.linalg.inv(A), np.inf)


def fwd_err(X, Xo):
    return np.abs(X - Xo).max() / max(np.abs(Xo).max(), 1e-300)


def pack_batch(mats, rhss):
    """Pack lists of numpy matrices / rhs into flat column-major buffers with
    even (16-byte aligned) offsets.  Returns device tensors."""
    a_off, b_off, ao, bo = [], [], 0, 0
    for A, B in zip(mats, rhss):
        n = A.shape[0]
        r = B.reshape(n, -1).shape[1]
        a_off.append(ao)
        b_off.append(bo)
        ao += (n * n + 1) // 2 * 2 + 2
        bo += (n * r + 1) // 2 * 2 + 2
    Af = np.zeros(max(ao, 2))
    Bf = np.zeros(max(bo, 2))
    ns, rs = [], []
    for A, B, o, q in zip(mats, rhss, a_off, b_off):
        n = A.shape[0]
        Bm = B.reshape(n, -1)
        Af[o:o + n * n] = A.T.reshape(-1)
        Bf[q:q + Bm.size] = Bm.T.reshape(-1)
        ns.append(n)
        rs.append(Bm.shape[1])
    t = lambda a, dt: torch.tensor(a, dtype=dt).cuda()
    return dict(count=len(mats), n=t(ns, torch.int64), nrhs=t(rs, torch.int64),
                a_off=t(a_off, torch.int64), b_off=t(b_off, torch.int64),
                A=torch.from_numpy(Af).cuda(), B=torch.from_numpy(Bf).cuda(),
                ns=ns, rs=rs, a_off_h=a_off, b_off_h=b_off)


def run_batch(ctx, pk, flags=0):
    from paper_2007_11208_gb300 import asolve
    X = torch.zeros_like(pk["B"])
    infos = torch.zeros(pk["count"] * asolve.INFO_BYTES, dtype=torch.uint8, device="cuda")
    rc = ctx.solve_batched(pk["count"], pk["n"], pk["nrhs"], pk["a_off"], pk["b_off"], pk["A"],
                           pk["B"], X, infos, flags | asolve.SYNC)
    assert rc == 0, rc
    Xh = X.cpu().numpy()
    out = []
    for s in range(pk["count"]):
        n, r, q = pk["ns"][s], pk["rs"][s], pk["b_off_h"][s]
        out.append(Xh[q:q + n * r].reshape(r, n).T)
    return out, asolve.infos_from_tensor(infos)
