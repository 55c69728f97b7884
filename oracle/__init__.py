"""CPU oracle for the adaptive solver (Sanderson & Curtin, arXiv 2007.11208).

TEST INFRASTRUCTURE ONLY.  This package wraps ``asolve_oracle.c`` -- a plain,
slow, FP64 restatement of the paper's scan (Sec. 2.1, 2.2, Fig. 4), routing
(Sec. 2), solvers (Sec. 2.1-2.4), condition estimate and SVD fallback
(Sec. 2.5) -- through ctypes.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it; the GPU library never
does, and the two share no code.

Matrices are numpy float64 arrays in column-major (Fortran) order, as the
paper's storage (Sec. 1, Sec. 2.1).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "asolve_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CLS_NONE, CLS_BANDED, CLS_LOWER, CLS_UPPER, CLS_SYMPD, CLS_GENERAL = range(6)
(ROUTE_NONE, ROUTE_BAND_LU, ROUTE_TRI_LOWER, ROUTE_TRI_UPPER, ROUTE_CHOL,
 ROUTE_CHOL_FAIL_LU, ROUTE_LU, ROUTE_SVD, ROUTE_TRIDIAG, ROUTE_LDLT, ROUTE_CHOL_FAIL_LDLT) = range(11)
OK, W_APPROX, W_ILLCOND = 0, 1, 2
E_INVALID, E_NONFINITE, E_SINGULAR = -1, -2, -3
NO_APPROX, FORCE_LU, FORCE_SVD, NO_RCOND = 1, 2, 4, 8
TRIDIAG = 256  # tridiagonal specialisation (opt-in route for kl = ku = 1)
SYM_INDEF = 512  # symmetric-indefinite specialisation (opt-in LDL^T route, n <= LDLT_NMAX)
LDLT_NMAX = 1024


class Scan(C.Structure):
    _fields_ = [("kl", C.c_int64), ("ku", C.c_int64), ("lower", C.c_int32),
                ("upper", C.c_int32), ("sympd", C.c_int32), ("banded", C.c_int32),
                ("nonfinite", C.c_int32), ("cls", C.c_int32), ("norm1", C.c_double),
                ("norminf", C.c_double)]


class Info(C.Structure):
    _fields_ = [("cls", C.c_int32), ("route", C.c_int32), ("status", C.c_int32),
                ("svd_used", C.c_int32), ("kl", C.c_int64), ("ku", C.c_int64),
                ("rcond", C.c_double), ("svd_rank", C.c_int64)]


class Config(C.Structure):
    _fields_ = [("rcond_threshold", C.c_double), ("sympd_tol", C.c_double),
                ("band_frac", C.c_double), ("svd_trunc_rel", C.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared",
                                   "-ffp-contract=off", "-fno-fast-math", "-o", tmp,
                                   _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.POINTER
        d, i64, i32 = C.c_double, C.c_int64, C.c_int
        pd, pi64 = P(d), P(i64)
        L.or_default_config.argtypes = [P(Config)]
        L.or_scan.argtypes = [pd, i64, P(Config), P(Scan)]
        L.or_scan_many.argtypes = [pd, i64, i64, P(Config), P(Scan)]
        L.or_band_count.argtypes = [i64, i64, i64]
        L.or_band_count.restype = i64
        L.or_likely_sympd.argtypes = [pd, i64, d]
        L.or_lu_factor.argtypes = [pd, i64, pi64]
        L.or_lu_solve.argtypes = [pd, pi64, i64, pd, i64, i32]
        L.or_chol_factor.argtypes = [pd, i64]
        L.or_chol_solve.argtypes = [pd, i64, pd, i64]
        L.or_tri_solve.argtypes = [pd, i64, i32, pd, i64, i32]
        L.or_band_pack.argtypes = [pd, i64, i64, i64, pd, i64]
        L.or_band_lu_factor.argtypes = [pd, i64, i64, i64, i64, pi64]
        L.or_band_lu_solve.argtypes = [pd, i64, i64, i64, i64, pi64, pd, i64, i32]
        for f in ("or_norm1", "or_norminf"):
            getattr(L, f).argtypes = [pd, i64]
            getattr(L, f).restype = d
        L.or_est_inv_norm1_lu.argtypes = [pd, pi64, i64]
        L.or_est_inv_norm1_chol.argtypes = [pd, i64]
        L.or_est_inv_norm1_tri.argtypes = [pd, i64, i32]
        L.or_est_inv_norm1_band.argtypes = [pd, i64, i64, i64, i64, pi64]
        for f in ("or_est_inv_norm1_lu", "or_est_inv_norm1_chol", "or_est_inv_norm1_tri",
                  "or_est_inv_norm1_band", "or_rcond_from"):
            getattr(L, f).restype = d
        L.or_rcond_from.argtypes = [d, d]
        L.or_is_symmetric.argtypes = [pd, i64, d]
        L.or_ldlt_factor.argtypes = [pd, i64, pi64]
        L.or_ldlt_solve.argtypes = [pd, pi64, i64, pd, i64]
        L.or_est_inv_norm1_ldlt.argtypes = [pd, pi64, i64]
        L.or_est_inv_norm1_ldlt.restype = d
        L.or_gt_factor.argtypes = [pd, pd, pd, pd, pi64, i64]
        L.or_gt_solve.argtypes = [pd, pd, pd, pd, pi64, i64, pd, i64, i32]
        L.or_est_inv_norm1_gt.argtypes = [pd, pd, pd, pd, pi64, i64]
        L.or_est_inv_norm1_gt.restype = d
        L.or_jacobi_svd.argtypes = [pd, pd, pd, i64, i32]
        L.or_svd_solve.argtypes = [pd, i64, pd, i64, d, pd]
        L.or_svd_solve.restype = i64
        L.or_residual_dot2.argtypes = [pd, i64, pd, pd, i64, pd, pd]
        L.or_solve.argtypes = [pd, pd, i64, i64, C.c_uint32, P(Config), pd, P(Info)]
        L.or_solve_band.argtypes = [pd, i64, i64, i64, pd, i64, i64, C.c_uint32,
                                    P(Config), pd, P(Info)]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _pi(a):
    return a.ctypes.data_as(C.POINTER(C.c_int64))


def _f64(a):
    return np.asfortranarray(a, dtype=np.float64)


def config(rcond_threshold=None, sympd_tol=None, band_frac=None, svd_trunc_rel=None):
    c = Config()
    lib().or_default_config(C.byref(c))
    if rcond_threshold is not None:
        c.rcond_threshold = rcond_threshold
    if sympd_tol is not None:
        c.sympd_tol = sympd_tol
    if band_frac is not None:
        c.band_frac = band_frac
    if svd_trunc_rel is not None:
        c.svd_trunc_rel = svd_trunc_rel
    return c


def _asdict(s):
    return {k: getattr(s, k) for k, _ in s._fields_}


def scan(A, cfg=None):
    A = _f64(A)
    n = A.shape[0]
    s = Scan()
    lib().or_scan(_p(A), n, C.byref(cfg or config()), C.byref(s))
    return _asdict(s)


def scan_many(As, cfg=None):
    """As: (count, n, n) array; each matrix column-major."""
    As = np.ascontiguousarray(np.transpose(np.asarray(As, dtype=np.float64), (0, 2, 1)))
    count, n = As.shape[0], As.shape[1]
    out = (Scan * count)()
    lib().or_scan_many(_p(As), n, count, C.byref(cfg or config()), out)
    return out


def band_count(n, kl, ku):
    return lib().or_band_count(n, kl, ku)


def likely_sympd(A, tol=100 * np.finfo(np.float64).eps):
    A = _f64(A)
    return bool(lib().or_likely_sympd(_p(A), A.shape[0], tol))


def lu_factor(A):
    F = _f64(A).copy(order="F")
    n = F.shape[0]
    ipiv = np.zeros(max(n, 1), dtype=np.int64)
    info = lib().or_lu_factor(_p(F), n, _pi(ipiv))
    return F, ipiv[:n], info


def lu_solve(F, ipiv, B, trans=False):
    X = _f64(np.array(B, dtype=np.float64, ndmin=2).reshape(F.shape[0], -1)).copy(order="F")
    lib().or_lu_solve(_p(F), _pi(np.ascontiguousarray(ipiv, dtype=np.int64)), F.shape[0],
                      _p(X), X.shape[1], int(trans))
    return X


def chol_factor(A):
    F = _f64(A).copy(order="F")
    info = lib().or_chol_factor(_p(F), F.shape[0])
    return F, info


def chol_solve(F, B):
    X = _f64(np.array(B, dtype=np.float64, ndmin=2).reshape(F.shape[0], -1)).copy(order="F")
    lib().or_chol_solve(_p(F), F.shape[0], _p(X), X.shape[1])
    return X


def tri_solve(T, B, lower, trans=False):
    T = _f64(T)
    X = _f64(np.array(B, dtype=np.float64, ndmin=2).reshape(T.shape[0], -1)).copy(order="F")
    info = lib().or_tri_solve(_p(T), T.shape[0], int(lower), _p(X), X.shape[1], int(trans))
    return X, info


def band_pack(A, kl, ku):
    A = _f64(A)
    n = A.shape[0]
    ldab = 2 * kl + ku + 1
    AB = np.zeros((ldab, n), dtype=np.float64, order="F")
    lib().or_band_pack(_p(A), n, kl, ku, _p(AB), ldab)
    return AB


def band_lu_factor(AB, kl, ku):
    F = _f64(AB).copy(order="F")
    n = F.shape[1]
    ipiv = np.zeros(max(n, 1), dtype=np.int64)
    info = lib().or_band_lu_factor(_p(F), F.shape[0], n, kl, ku, _pi(ipiv))
    return F, ipiv[:n], info


def band_lu_solve(F, kl, ku, ipiv, B, trans=False):
    n = F.shape[1]
    X = _f64(np.array(B, dtype=np.float64, ndmin=2).reshape(n, -1)).copy(order="F")
    lib().or_band_lu_solve(_p(F), F.shape[0], n, kl, ku,
                           _pi(np.ascontiguousarray(ipiv, dtype=np.int64)), _p(X),
                           X.shape[1], int(trans))
    return X


def is_symmetric(A, tol=None):
    A = _f64(A)
    return lib().or_is_symmetric(_p(A), A.shape[0], config().sympd_tol if tol is None else tol)


def ldlt_factor(A):
    """Bunch-Kaufman LDL^T of A's lower triangle: (F, ipiv, info)."""
    F = _f64(A).copy(order="F")
    n = F.shape[0]
    ipiv = np.zeros(max(n, 1), dtype=np.int64)
    info = lib().or_ldlt_factor(_p(F), n, _pi(ipiv))
    return F, ipiv[:n], info


def ldlt_solve(F, ipiv, B):
    n = F.shape[0]
    X = _f64(np.array(B, dtype=np.float64, ndmin=2).reshape(n, -1)).copy(order="F")
    lib().or_ldlt_solve(_p(F), _pi(np.ascontiguousarray(ipiv, dtype=np.int64)), n, _p(X), X.shape[1])
    return X


def est_inv_norm1_ldlt(F, ipiv):
    return lib().or_est_inv_norm1_ldlt(_p(F), _pi(np.ascontiguousarray(ipiv, dtype=np.int64)), F.shape[0])


def gt_factor(dl, d, du):
    """Tridiagonal LU with partial pivoting (xGTTRF semantics) of the
    diagonals dl (n-1), d (n), du (n-1).  Returns (dl, d, du, du2, ipiv, info)."""
    d = np.array(d, dtype=np.float64)
    n = d.shape[0]
    dl = np.array(dl, dtype=np.float64).reshape(max(n - 1, 0))
    du = np.array(du, dtype=np.float64).reshape(max(n - 1, 0))
    dlp, dup = np.zeros(max(n - 1, 1)), np.zeros(max(n - 1, 1))
    dlp[:n - 1], dup[:n - 1] = dl, du
    du2 = np.zeros(max(n - 2, 1))
    ipiv = np.zeros(max(n, 1), dtype=np.int64)
    info = lib().or_gt_factor(_p(dlp), _p(d), _p(dup), _p(du2), _pi(ipiv), n)
    return dlp, d, dup, du2, ipiv[:n], info


def gt_solve(fac, B, trans=False):
    dl, d, du, du2, ipiv, _ = fac
    n = d.shape[0]
    X = _f64(np.array(B, dtype=np.float64, ndmin=2).reshape(n, -1)).copy(order="F")
    lib().or_gt_solve(_p(dl), _p(d), _p(du), _p(du2), _pi(np.ascontiguousarray(ipiv, dtype=np.int64)), n,
                      _p(X), X.shape[1], int(trans))
    return X


def est_inv_norm1_gt(fac):
    dl, d, du, du2, ipiv, _ = fac
    return lib().or_est_inv_norm1_gt(_p(dl), _p(d), _p(du), _p(du2),
                                     _pi(np.ascontiguousarray(ipiv, dtype=np.int64)), d.shape[0])


def norm1(A):
    A = _f64(A)
    return lib().or_norm1(_p(A), A.shape[0])


def norminf(A):
    A = _f64(A)
    return lib().or_norminf(_p(A), A.shape[0])


def est_inv_norm1_lu(F, ipiv):
    return lib().or_est_inv_norm1_lu(_p(F), _pi(np.ascontiguousarray(ipiv, dtype=np.int64)),
                                     F.shape[0])


def est_inv_norm1_chol(F):
    return lib().or_est_inv_norm1_chol(_p(F), F.shape[0])


def est_inv_norm1_tri(T, lower):
    T = _f64(T)
    return lib().or_est_inv_norm1_tri(_p(T), T.shape[0], int(lower))


def est_inv_norm1_band(F, kl, ku, ipiv):
    return lib().or_est_inv_norm1_band(_p(F), F.shape[0], F.shape[1], kl, ku,
                                       _pi(np.ascontiguousarray(ipiv, dtype=np.int64)))


def rcond_from(anorm, ainvnm):
    return lib().or_rcond_from(anorm, ainvnm)


def jacobi_svd(A, max_sweeps=30):
    G = _f64(A).copy(order="F")
    n = G.shape[0]
    V = np.zeros((n, n), dtype=np.float64, order="F")
    s = np.zeros(n, dtype=np.float64)
    sweeps = lib().or_jacobi_svd(_p(G), _p(V), _p(s), n, max_sweeps)
    return G, V, s, sweeps


def svd_solve(A, B, trunc_rel=0.0):
    A = _f64(A)
    n = A.shape[0]
    Bm = _f64(np.array(B, dtype=np.float64, ndmin=2).reshape(n, -1))
    X = np.zeros_like(Bm, order="F")
    rank = lib().or_svd_solve(_p(A), n, _p(Bm), Bm.shape[1], trunc_rel, _p(X))
    return X, rank


def residual_dot2(A, X, B):
    A = _f64(A)
    n = A.shape[0]
    Xm = _f64(np.array(X, dtype=np.float64, ndmin=2).reshape(n, -1))
    Bm = _f64(np.array(B, dtype=np.float64, ndmin=2).reshape(n, -1))
    R = np.zeros_like(Bm, order="F")
    berr = np.zeros(Bm.shape[1], dtype=np.float64)
    lib().or_residual_dot2(_p(A), n, _p(Xm), _p(Bm), Bm.shape[1], _p(R), _p(berr))
    return R, berr


def solve(A, B, flags=0, cfg=None):
    """The whole adaptive solve.  Returns (X, info dict)."""
    A = _f64(A)
    n = A.shape[0]
    Bm = _f64(np.array(B, dtype=np.float64, ndmin=2).reshape(n, -1) if n else
              np.zeros((0, 1)))
    X = np.zeros_like(Bm, order="F")
    info = Info()
    lib().or_solve(_p(A), _p(Bm), n, Bm.shape[1], flags, C.byref(cfg or config()),
                   _p(X), C.byref(info))
    return X, _asdict(info)


def solve_band(AB, kl, ku, B, flags=0, cfg=None):
    """AB: (ldab, n) compact band, A(i,j) at AB[ku+i-j, j]."""
    AB = _f64(AB)
    ldab, n = AB.shape
    Bm = _f64(np.array(B, dtype=np.float64, ndmin=2).reshape(n, -1))
    X = np.zeros_like(Bm, order="F")
    info = Info()
    lib().or_solve_band(_p(AB), ldab, kl, ku, _p(Bm), n, Bm.shape[1], flags,
                        C.byref(cfg or config()), _p(X), C.byref(info))
    return X, _asdict(info)
