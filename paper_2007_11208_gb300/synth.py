"""Seeded synthetic inputs shaped like the adaptive solver's workloads.

Harness code: it generates matrices and right-hand sides and nothing else.
It holds none of the solver's arithmetic, and the GPU library never calls
it.  The same bytes are handed to the GPU path and to the CPU oracle.

Every generator takes a ``torch.Generator`` (CPU or CUDA) and returns FP64
tensors in column-major layout (a matrix is stored as its transpose's
row-major buffer: ``A.t().contiguous()`` viewed as (n, n) holds A
column-major).  To keep that convention simple every function here returns
the *column-major buffer as a 2-D tensor M with M[j, i] = A[i, j]*; use
``colmajor_to_dense`` to see A itself.

Recipes (the paper's workloads are "random" matrices, Sec. 3; the
distributions below are the ones the benchmark configurations name):
  general      A ~ N(0,1)
  shifted      A ~ N(0,1) + 2 sqrt(n) I
  lower_tri    off-diagonal N(0,1), diagonal 1 + |N(0,1)|
  tri_dd       off-diagonal N(0,1), diagonal 1 + sum_j |a_ij| (row)
  spd          G ~ N(0,1), A = G^T G / n + I, upper mirrored from lower
  tridiag      off-diagonals N(0,1), diagonal 4 + |N(0,1)|
  banded_dd    band entries N(0,1), diagonal 1 + row sum of |off-diagonal|
  ill          U diag(logspace(0, -k, n)) V^T, U, V Haar (QR of a
               Gaussian with sign-corrected R)
  reflector    U, V products of 8 random Householder reflectors and random
               signs (exact spectrum at O(n^2) cost, for large n)
  tri_kappa    T = D (I + s N), N strictly triangular N(0,1), s = 1/n,
               D = diag(logspace(0, -log10 kappa))
  replica_*    the paper's evaluation (Sec. 3, Fig. 3): entries U[-0.5, 0.5]
               (Fig. 3's randu - 0.5); sympd R^T R + I (Fig. 3), mirrored;
               dense as drawn; lower triangle and 5-diagonal band with
               diagonal 1 + row sum of |off-diagonal| (the paper does not
               give these two recipes; dominance keeps them on their routes,
               since random triangles are exponentially ill-conditioned);
               right-hand side U[0, 1] (Fig. 3's fill::randu)
"""
from __future__ import annotations

import math

import torch

F64 = torch.float64


def gen(seed: int, device="cpu") -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return g


def _randn(shape, g, device):
    return torch.randn(*shape, generator=g, device=device, dtype=F64)


def colmajor(A: torch.Tensor) -> torch.Tensor:
    """Dense A (row-major tensor holding A[i, j]) -> column-major buffer."""
    return A.t().contiguous()


def colmajor_to_dense(M: torch.Tensor) -> torch.Tensor:
    return M.t()


def general(n, g, device="cpu"):
    return colmajor(_randn((n, n), g, device))


def shifted(n, g, device="cpu"):
    A = _randn((n, n), g, device)
    A.diagonal().add_(2.0 * math.sqrt(n))
    return colmajor(A)


def lower_tri(n, g, device="cpu"):
    A = torch.tril(_randn((n, n), g, device), -1)
    A.diagonal().copy_(1.0 + _randn((n,), g, device).abs())
    return colmajor(A)


def tri_dd(n, g, lower=True, device="cpu"):
    A = _randn((n, n), g, device)
    A = torch.tril(A, -1) if lower else torch.triu(A, 1)
    A.diagonal().copy_(1.0 + A.abs().sum(dim=1))
    return colmajor(A)


def mirror_lower(A):
    """Exactly symmetric copy of A built from its lower triangle."""
    L = torch.tril(A)
    return L + torch.tril(A, -1).t()


def spd(n, g, device="cpu"):
    G = _randn((n, n), g, device)
    A = G.t() @ G / n
    A.diagonal().add_(1.0)
    return colmajor(mirror_lower(A))


def tridiag(n, g, device="cpu"):
    A = torch.zeros((n, n), dtype=F64, device=device)
    if n > 1:
        idx = torch.arange(n - 1, device=device)
        A[idx + 1, idx] = _randn((n - 1,), g, device)
        A[idx, idx + 1] = _randn((n - 1,), g, device)
    A.diagonal().copy_(4.0 + _randn((n,), g, device).abs())
    return colmajor(A)


def banded_dd(n, kl, ku, g, device="cpu"):
    A = _randn((n, n), g, device)
    i = torch.arange(n, device=device)
    d = i[None, :] - i[:, None]  # column - row
    A = torch.where((d <= ku) & (-d <= kl), A, torch.zeros((), dtype=F64, device=device))
    A.diagonal().zero_()
    A.diagonal().copy_(1.0 + A.abs().sum(dim=1))
    return colmajor(A)


def haar(n, g, device="cpu"):
    """Haar-distributed orthogonal matrix (QR of a Gaussian, R signs fixed)."""
    Z = _randn((n, n), g, device)
    Q, R = torch.linalg.qr(Z.cpu())  # host LAPACK: no device linear-algebra library needed
    Q, R = Q.to(device), R.to(device)
    s = torch.sign(torch.diagonal(R))
    s[s == 0] = 1.0
    return Q * s[None, :]


def ill(n, g, k=14.0, device="cpu"):
    U = haar(n, g, device)
    V = haar(n, g, device)
    s = torch.logspace(0.0, -k, n, dtype=F64, device=device)
    return colmajor((U * s[None, :]) @ V.t())


def reflector_orth(n, g, nref=8, device="cpu"):
    """Q = D H_1 ... H_nref as a dense matrix (D random signs)."""
    Q = torch.diag(torch.where(torch.rand(n, generator=g, device=device, dtype=F64) < 0.5,
                               -1.0, 1.0).to(F64))
    for _ in range(nref):
        v = _randn((n,), g, device)
        v = v / torch.linalg.vector_norm(v)
        Q = Q - 2.0 * torch.outer(Q @ v, v)
    return Q


def spectrum_general(n, g, kappa, device="cpu", orth=reflector_orth):
    U = orth(n, g, device=device)
    V = orth(n, g, device=device)
    s = torch.logspace(0.0, -math.log10(kappa), n, dtype=F64, device=device)
    return colmajor((U * s[None, :]) @ V.t())


def spectrum_spd(n, g, kappa, device="cpu", orth=reflector_orth):
    U = orth(n, g, device=device)
    s = torch.logspace(0.0, -math.log10(kappa), n, dtype=F64, device=device)
    return colmajor(mirror_lower((U * s[None, :]) @ U.t()))


def _signs(n, g, device):
    return torch.where(torch.rand(n, generator=g, device=device, dtype=F64) < 0.5, -1.0, 1.0)


def _unit(n, g, device):
    v = _randn((n,), g, device)
    return v / torch.linalg.vector_norm(v)


def spectrum_fast(n, g, kappa, spd=False, nref=8, device="cpu"):
    """U diag(logspace(0, -log10 kappa, n)) V^T (V = U when spd) with U, V
    products of nref random reflectors and random signs, built by applying
    the reflectors to the diagonal one at a time: O(nref n^2) work and one
    n x n buffer, for the largest sizes.  Column-major buffer."""
    s = torch.logspace(0.0, -math.log10(kappa), n, dtype=F64, device=device)
    M = torch.diag(s)
    for _ in range(nref):
        v = _unit(n, g, device)
        M.addr_(v, v @ M, alpha=-2.0)          # H M
        w = v if spd else _unit(n, g, device)
        M.addr_(M @ w, w, alpha=-2.0)          # M H'
    d = _signs(n, g, device)
    e = d if spd else _signs(n, g, device)
    M.mul_(d[:, None]).mul_(e[None, :])
    if spd:
        M = mirror_lower(M)
    return colmajor(M)


def tri_kappa(n, g, kappa, lower=True, device="cpu"):
    """T = D (I + s N), N strictly triangular N(0,1), s = 1/n, D =
    diag(logspace(0, -log10 kappa, n)) in random order of rows."""
    N = _randn((n, n), g, device)
    N = torch.tril(N, -1) if lower else torch.triu(N, 1)
    T = N.mul_(1.0 / n)
    T.diagonal().add_(1.0)
    dd = torch.logspace(0.0, -math.log10(kappa), n, dtype=F64, device=device)
    dd = dd[torch.randperm(n, generator=g, device=device)]
    return colmajor(T * dd[:, None])


def banded_kappa(n, kl, ku, g, kappa, device="cpu"):
    """Diagonally dominant band matrix with rows scaled by
    logspace(0, -log10 kappa) in random order (same band, kappa grown)."""
    A = colmajor_to_dense(banded_dd(n, kl, ku, g, device))
    dd = torch.logspace(0.0, -math.log10(kappa), n, dtype=F64, device=device)
    dd = dd[torch.randperm(n, generator=g, device=device)]
    return colmajor(A * dd[:, None])


def rhs(n, nrhs, g, device="cpu"):
    """B ~ N(0,1), column-major buffer of shape (nrhs, n)."""
    return _randn((nrhs, n), g, device)


def band_storage_dd(n, kl, ku, g, device="cpu"):
    """Diagonally dominant band matrix directly in compact band storage:
    returns AB of shape (n, kl+ku+1) whose row j is column j of the
    LAPACK layout, i.e. AB[j, ku + i - j] = A[i, j] for max(0,j-ku) <= i <=
    min(n-1, j+kl).  Entries outside the matrix are zero.  Off-diagonal
    entries N(0,1); diagonal 1 + sum of |off-diagonal| in the row."""
    ld = kl + ku + 1
    AB = _randn((n, ld), g, device)
    j = torch.arange(n, device=device)[:, None]
    r = torch.arange(ld, device=device)[None, :]
    i = r - ku + j  # row index of each slot
    AB = torch.where((i >= 0) & (i < n), AB, torch.zeros((), dtype=F64, device=device))
    AB[:, ku] = 0.0
    # row sums of |off-diagonal|: slot (j, r) is A[i, j] with i = j + r - ku
    rowsum = torch.zeros(n, dtype=F64, device=device)
    rowsum.index_add_(0, i.clamp(0, n - 1).reshape(-1), AB.abs().reshape(-1))
    AB[:, ku] = 1.0 + rowsum
    return AB


# --------------------------------------------------------------------------
# The batched workload: a class mix of many systems of uneven size.
BATCH_MIX = (("general", 0.40), ("spd", 0.25), ("banded", 0.15), ("tri", 0.15),
             ("ill", 0.05))


def batch_specs(count, seed, nmin=16, nmax=512, rmin=1, rmax=8, kmax=16):
    """Per-system (kind, n, nrhs, kl, ku, lower) for the batched mix."""
    g = gen(seed)
    u = torch.rand(count, generator=g, dtype=F64)
    ns = torch.randint(nmin, nmax + 1, (count,), generator=g)
    rs = torch.randint(rmin, rmax + 1, (count,), generator=g)
    kls = torch.randint(1, kmax + 1, (count,), generator=g)
    kus = torch.randint(1, kmax + 1, (count,), generator=g)
    lows = torch.rand(count, generator=g) < 0.5
    edges, acc = [], 0.0
    for kind, p in BATCH_MIX:
        acc += p
        edges.append((kind, acc))
    specs = []
    for c in range(count):
        kind = next(k for k, e in edges if u[c].item() < e or k == edges[-1][0])
        specs.append((kind, int(ns[c]), int(rs[c]), int(kls[c]), int(kus[c]),
                      bool(lows[c])))
    return specs


def batch_matrix(spec, g, device="cpu"):
    kind, n, _, kl, ku, lower = spec
    if kind == "general":
        return shifted(n, g, device)
    if kind == "spd":
        return spd(n, g, device)
    if kind == "banded":
        return banded_dd(n, kl, ku, g, device)
    if kind == "tri":
        return tri_dd(n, g, lower=lower, device=device)
    if kind == "ill":
        return ill(n, g, k=13.0, device=device)
    raise ValueError(kind)


def align(x, a=32):
    return (x + a - 1) // a * a


def packed_batch(specs, seed, device="cpu"):
    """All systems of a batch packed into flat FP64 buffers.

    Returns dict with A, B (flat), n, nrhs, a_off, b_off (int64) -- each
    system's A starts at a multiple of 32 elements (256 bytes)."""
    g = gen(seed, device)
    a_off, b_off, ao, bo = [], [], 0, 0
    for (_, n, r, *_rest) in specs:
        a_off.append(ao)
        b_off.append(bo)
        ao += align(n * n)
        bo += align(n * r)
    A = torch.zeros(max(ao, 1), dtype=F64, device=device)
    B = torch.zeros(max(bo, 1), dtype=F64, device=device)
    for s, (spec, o, q) in enumerate(zip(specs, a_off, b_off)):
        n, r = spec[1], spec[2]
        A[o:o + n * n] = batch_matrix(spec, g, device).reshape(-1)
        B[q:q + n * r] = rhs(n, r, g, device).reshape(-1)
    return {"A": A, "B": B,
            "n": torch.tensor([s[1] for s in specs], dtype=torch.int64),
            "nrhs": torch.tensor([s[2] for s in specs], dtype=torch.int64),
            "a_off": torch.tensor(a_off, dtype=torch.int64),
            "b_off": torch.tensor(b_off, dtype=torch.int64)}


REPLICA_KINDS = ("band5", "lower", "sympd", "dense")


def replica_batch(kind, n, count, seed, device="cpu"):
    """`count` systems of order n for one row of the paper's Tables 1-4,
    packed like packed_batch (one right-hand side each)."""
    g = gen(seed, device)
    R = torch.rand((count, n, n), generator=g, device=device, dtype=F64) - 0.5
    i = torch.arange(n, device=device)
    if kind == "sympd":
        A = R.transpose(1, 2) @ R
        A.diagonal(dim1=1, dim2=2).add_(1.0)
        A = torch.tril(A) + torch.tril(A, -1).transpose(1, 2)
    elif kind == "dense":
        A = R
    elif kind in ("lower", "band5"):
        d = i[None, :] - i[:, None]  # column - row
        keep = (d < 0) if kind == "lower" else ((d != 0) & (d.abs() <= 2))
        A = torch.where(keep, R, torch.zeros((), dtype=F64, device=device))
        A.diagonal(dim1=1, dim2=2).copy_(1.0 + A.abs().sum(dim=2))
    else:
        raise ValueError(kind)
    del R
    sa, sb = align(n * n), align(n)
    Af = torch.zeros((count, sa), dtype=F64, device=device)
    Af[:, :n * n] = A.transpose(1, 2).reshape(count, n * n)  # column-major per system
    del A
    Bf = torch.zeros((count, sb), dtype=F64, device=device)
    Bf[:, :n] = torch.rand((count, n), generator=g, device=device, dtype=F64)
    idx = torch.arange(count, dtype=torch.int64)
    return {"A": Af.reshape(-1), "B": Bf.reshape(-1),
            "n": torch.full((count,), n, dtype=torch.int64),
            "nrhs": torch.ones(count, dtype=torch.int64),
            "a_off": idx * sa, "b_off": idx * sb}
