"""Thin ctypes binding of libasolve.so (include/asolve.h).

Argument marshalling only: every step of the solve runs in the library's CUDA
kernels.  Device buffers are torch CUDA tensors (FP64, column-major buffers:
a matrix A is passed as a tensor whose memory holds A column by column).
If libasolve.so is missing the import fails loudly; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libasolve.so")

# ---- constants mirrored from include/asolve.h -----------------------------
OK, W_APPROX, W_ILLCOND, PENDING = 0, 1, 2, 3
E_INVALID, E_NONFINITE, E_SINGULAR, E_NOMEM, E_CUDA, E_TIMEOUT, E_IR_STALL, E_UNSUPPORTED = (
    -1, -2, -3, -4, -5, -6, -7, -8)
CLS_NONE, CLS_BANDED, CLS_LOWER, CLS_UPPER, CLS_SYMPD, CLS_GENERAL = range(6)
(ROUTE_NONE, ROUTE_BAND_LU, ROUTE_TRI_LOWER, ROUTE_TRI_UPPER, ROUTE_CHOL,
 ROUTE_CHOL_FAIL_LU, ROUTE_LU, ROUTE_SVD, ROUTE_TRIDIAG, ROUTE_LDLT, ROUTE_CHOL_FAIL_LDLT) = range(11)
PREC_FP64, PREC_MIXED, PREC_BF16, PREC_FP16, PREC_FP64_OZ, PREC_FP8 = 0, 1, 2, 3, 4, 5
GEMM_TF32, GEMM_TF32X3, GEMM_BF16, GEMM_FP16, GEMM_FP8 = 1, 3, 16, 17, 18
NO_APPROX, FORCE_LU, FORCE_SVD, NO_RCOND, SYNC, HOST_BUFFERS, BERR, RESIDENT, TRIDIAG, SYM_INDEF = (
    0x01, 0x02, 0x04, 0x08, 0x10, 0x20, 0x40, 0x80, 0x100, 0x200)


class Config(C.Structure):
    _fields_ = [("rcond_threshold", C.c_double), ("sympd_tol", C.c_double),
                ("band_frac", C.c_double), ("svd_trunc_rel", C.c_double),
                ("precision", C.c_int32), ("ir_max_iter", C.c_int32),
                ("ir_target_berr", C.c_double), ("ir_kappa_limit", C.c_double),
                ("hbm_budget", C.c_size_t), ("stream", C.c_void_p), ("device", C.c_int32),
                ("reserved", C.c_int32)]


class Info(C.Structure):
    _fields_ = [("cls", C.c_int32), ("route", C.c_int32), ("status", C.c_int32),
                ("ir_iters", C.c_int32), ("kl", C.c_int64), ("ku", C.c_int64),
                ("rcond", C.c_double), ("berr", C.c_double), ("svd_rank", C.c_int64),
                ("precision", C.c_int32), ("detail", C.c_int32)]


class ScanResult(C.Structure):
    _fields_ = [("kl", C.c_int64), ("ku", C.c_int64), ("lower", C.c_int32),
                ("upper", C.c_int32), ("sympd", C.c_int32), ("banded", C.c_int32),
                ("nonfinite", C.c_int32), ("cls", C.c_int32), ("norm1", C.c_double),
                ("norminf", C.c_double)]


class ServeStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("rejected", C.c_int64), ("queued", C.c_int64), ("rounds", C.c_int64),
                ("batches", C.c_int64), ("large_solves", C.c_int64), ("budget", C.c_size_t),
                ("charged_bytes", C.c_size_t), ("peak_charged_bytes", C.c_size_t),
                ("busy_ms", C.c_double), ("wall_ms", C.c_double)]


class _ProfEntry(C.Structure):
    _fields_ = [("name", C.c_char * 40), ("launches", C.c_int64), ("total_ms", C.c_double)]


class Profile(C.Structure):
    _fields_ = [("count", C.c_int32), ("reserved", C.c_int32), ("k", _ProfEntry * 24)]


INFO_BYTES = C.sizeof(Info)
assert INFO_BYTES == 64

_lib = None

# Every symbol include/asolve.h declares.
EXPORTS = ("asolve_version", "asolve_strerror", "asolve_default_config", "asolve_create",
           "asolve_destroy", "asolve_stream", "asolve_scan", "asolve_solve",
           "asolve_solve_band", "asolve_solve_batched", "asolve_set_profiling",
           "asolve_get_profile", "asolve_reset_profile", "asolve_scan_noalloc",
           "asolve_gemm_sub", "asolve_solve_batched_ptrs", "asolve_submit", "asolve_poll",
           "asolve_get_serve_stats", "asolve_set_panel_widths", "asolve_pipe_peak",
           "asolve_gemm_oz_ws_bytes", "asolve_gemm_oz")
PIPE_FFMA, PIPE_DFMA, PIPE_DMMA = 1, 2, 3


def lib():
    """Load libasolve.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2007_11208_gb300/build.py "
                          "(no CPU fallback exists)")
    L = C.CDLL(LIB_PATH)
    P, vp, i64, i32, u32 = C.POINTER, C.c_void_p, C.c_int64, C.c_int, C.c_uint32
    L.asolve_version.restype = C.c_char_p
    L.asolve_strerror.argtypes = [i32]
    L.asolve_strerror.restype = C.c_char_p
    L.asolve_default_config.argtypes = [P(Config)]
    L.asolve_create.argtypes = [P(vp), P(Config)]
    L.asolve_destroy.argtypes = [vp]
    L.asolve_stream.argtypes = [vp]
    L.asolve_stream.restype = vp
    L.asolve_scan.argtypes = [vp, vp, i64, P(ScanResult)]
    L.asolve_solve.argtypes = [vp, vp, vp, i64, i64, u32, vp, P(Info)]
    L.asolve_solve_band.argtypes = [vp, vp, i64, i64, i64, vp, i64, i64, u32, vp, P(Info)]
    L.asolve_solve_batched.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, u32, vp]
    L.asolve_set_profiling.argtypes = [vp, i32]
    L.asolve_get_profile.argtypes = [vp, P(Profile)]
    L.asolve_reset_profile.argtypes = [vp]
    L.asolve_scan_noalloc.argtypes = [vp, i64, vp, vp]
    L.asolve_gemm_sub.argtypes = [vp, i64, vp, i64, vp, i64, i64, i64, i64, i32, vp, vp]
    L.asolve_solve_batched_ptrs.argtypes = [vp, i64, vp, vp, vp, vp, vp, u32, vp]
    L.asolve_submit.argtypes = [vp, vp, vp, i64, i64, u32, vp, P(C.c_uint64)]
    L.asolve_poll.argtypes = [vp, C.c_uint64, i64, P(Info), P(C.c_double)]
    L.asolve_get_serve_stats.argtypes = [vp, P(ServeStats)]
    L.asolve_set_panel_widths.argtypes = [vp, i32, vp, i32]
    L.asolve_pipe_peak.argtypes = [i32, i32, P(C.c_double), P(C.c_double)]
    L.asolve_gemm_oz_ws_bytes.argtypes = [i64, i64, i64]
    L.asolve_gemm_oz_ws_bytes.restype = C.c_size_t
    for f in EXPORTS:
        if f not in ("asolve_version", "asolve_strerror", "asolve_stream", "asolve_gemm_oz_ws_bytes"):
            getattr(L, f).restype = i32
    _lib = L
    return L


def strerror(code: int) -> str:
    return lib().asolve_strerror(code).decode()


def default_config(**kw) -> Config:
    c = Config()
    lib().asolve_default_config(C.byref(c))
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return C.c_void_p(t.data_ptr())
    return C.c_void_p(t)


def _need(t, count: int, name: str):
    """A tensor argument must hold at least `count` FP64 elements and be
    contiguous (the library reads and writes exactly that extent)."""
    if isinstance(t, torch.Tensor):
        if t.dtype != torch.float64 or not t.is_contiguous():
            raise ValueError(f"{name}: expected a contiguous float64 tensor")
        if t.numel() < count:
            raise ValueError(f"{name}: {t.numel()} elements, the call needs {count}")


def info_dict(i: Info) -> dict:
    return {k: getattr(i, k) for k, _ in Info._fields_}


def infos_from_tensor(t: torch.Tensor) -> list:
    """Decode a uint8/byte tensor holding count asolve_info records."""
    raw = t.detach().cpu().contiguous().numpy().tobytes()
    n = len(raw) // INFO_BYTES
    return [info_dict(Info.from_buffer_copy(raw[k * INFO_BYTES:(k + 1) * INFO_BYTES]))
            for k in range(n)]


class Context:
    """Owns an asolve_ctx (one CUDA stream, workspaces, captured graphs).

    The library's stream is non-blocking, so it is not ordered after work
    queued on torch's streams.  Every call below first makes the context
    stream wait for torch's current stream (inputs written there are
    complete before the library reads them) and afterwards makes torch's
    current stream wait for the context stream (outputs are complete before
    later torch work reads them).  Both are device-side waits on events."""

    def __init__(self, tuning=None, **cfg):
        """tuning: path of a panel-width table written by autotune.py (optional)."""
        self._h = C.c_void_p()
        c = default_config(**cfg)
        rc = lib().asolve_create(C.byref(self._h), C.byref(c))
        if rc != OK:
            raise RuntimeError(f"asolve_create: {strerror(rc)}")
        self._dev = None
        if torch.cuda.is_available():
            d = int(c.device)
            self._dev = torch.device("cuda", d if d >= 0 else torch.cuda.current_device())
        self._ext = None
        if tuning is not None:
            self.load_tuning(tuning)

    def _lib_stream(self):
        if self._ext is None:
            self._ext = torch.cuda.ExternalStream(self.stream, device=self._dev)
        return self._ext

    def _order_in(self):
        """Context stream waits for torch's current stream."""
        if self._dev is not None:
            self._lib_stream().wait_stream(torch.cuda.current_stream(self._dev))

    def _order_out(self):
        """torch's current stream waits for the context stream."""
        if self._dev is not None:
            torch.cuda.current_stream(self._dev).wait_stream(self._lib_stream())

    def set_panel_widths(self, kind: int, widths) -> int:
        arr = (C.c_int32 * len(widths))(*[int(x) for x in widths])
        return lib().asolve_set_panel_widths(self._h, kind, C.cast(arr, C.c_void_p), len(widths))

    def load_tuning(self, path: str):
        import json
        with open(path) as f:
            t = json.load(f)
        for kind, key in enumerate(("lu32", "chol32", "lu64", "chol64")):
            if key in t.get("nb", {}):
                rc = self.set_panel_widths(kind, t["nb"][key])
                if rc != OK:
                    raise RuntimeError(f"asolve_set_panel_widths: {strerror(rc)}")

    def close(self):
        self._ext = None
        if self._h:
            lib().asolve_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    @property
    def stream(self) -> int:
        return lib().asolve_stream(self._h)

    def scan(self, A: torch.Tensor, n: int) -> dict:
        r = ScanResult()
        self._order_in()
        rc = lib().asolve_scan(self._h, _ptr(A), n, C.byref(r))
        if rc != OK:
            raise RuntimeError(f"asolve_scan: {strerror(rc)}")
        return {k: getattr(r, k) for k, _ in ScanResult._fields_}

    def solve(self, A, B, n: int, nrhs: int, X, flags: int = 0):
        """A, B, X: CUDA tensors (or host pointers with HOST_BUFFERS)."""
        _need(A, n * n, "A")
        _need(B, n * nrhs, "B")
        _need(X, n * nrhs, "X")
        inf = Info()
        self._order_in()
        rc = lib().asolve_solve(self._h, _ptr(A), _ptr(B), n, nrhs, flags, _ptr(X), C.byref(inf))
        self._order_out()
        return rc, info_dict(inf)

    def solve_band(self, AB, ldab: int, kl: int, ku: int, B, n: int, nrhs: int, X, flags: int = 0):
        _need(AB, ldab * n, "AB")
        _need(B, n * nrhs, "B")
        _need(X, n * nrhs, "X")
        inf = Info()
        self._order_in()
        rc = lib().asolve_solve_band(self._h, _ptr(AB), ldab, kl, ku, _ptr(B), n, nrhs, flags,
                                     _ptr(X), C.byref(inf))
        self._order_out()
        return rc, info_dict(inf)

    def solve_batched(self, count, n, nrhs, a_off, b_off, A, B, X, infos, flags: int = 0) -> int:
        self._order_in()
        rc = lib().asolve_solve_batched(self._h, count, _ptr(n), _ptr(nrhs), _ptr(a_off),
                                        _ptr(b_off), _ptr(A), _ptr(B), _ptr(X), flags,
                                        _ptr(infos))
        self._order_out()
        return rc

    def solve_batched_ptrs(self, count, n, nrhs, A_ptrs, B_ptrs, X_ptrs, infos, flags: int = 0) -> int:
        """n, nrhs: int64 device tensors; *_ptrs: int64 device tensors of addresses."""
        self._order_in()
        rc = lib().asolve_solve_batched_ptrs(self._h, count, _ptr(n), _ptr(nrhs), _ptr(A_ptrs),
                                             _ptr(B_ptrs), _ptr(X_ptrs), flags, _ptr(infos))
        self._order_out()
        return rc

    def submit(self, A, B, n: int, nrhs: int, X, flags: int = 0):
        """Queue one request; returns (rc, ticket).  The buffers must outlive it."""
        _need(A, n * n, "A")
        _need(B, n * nrhs, "B")
        _need(X, n * nrhs, "X")
        t = C.c_uint64(0)
        # the server's lanes run on streams of their own: inputs written on
        # torch's current stream must be complete before they are queued
        if self._dev is not None and not (flags & HOST_BUFFERS):
            torch.cuda.current_stream(self._dev).synchronize()
        rc = lib().asolve_submit(self._h, _ptr(A), _ptr(B), n, nrhs, flags, _ptr(X), C.byref(t))
        return rc, t.value

    def poll(self, ticket: int, wait_us: int = -1):
        """Returns (status, info dict, latency_ms) once the request completed
        (status = info["status"]), else (PENDING or E_INVALID, None, None)."""
        inf = Info()
        lat = C.c_double(0.0)
        rc = lib().asolve_poll(self._h, ticket, wait_us, C.byref(inf), C.byref(lat))
        if rc != OK:
            return rc, None, None
        return inf.status, info_dict(inf), lat.value

    def serve_stats(self) -> dict:
        st = ServeStats()
        lib().asolve_get_serve_stats(self._h, C.byref(st))
        return {k: getattr(st, k) for k, _ in ServeStats._fields_}

    def set_profiling(self, on: bool):
        lib().asolve_set_profiling(self._h, int(on))

    def reset_profile(self):
        lib().asolve_reset_profile(self._h)

    def profile(self) -> dict:
        p = Profile()
        lib().asolve_get_profile(self._h, C.byref(p))
        return {p.k[i].name.decode(): (p.k[i].launches, p.k[i].total_ms) for i in range(p.count)}


def pipe_peak(pipe: int, iters: int = 4096):
    """(TFLOP/s, ms) of one arithmetic pipe's issue-rate probe on the current device."""
    tf, ms = C.c_double(0.0), C.c_double(0.0)
    rc = lib().asolve_pipe_peak(pipe, iters, C.byref(tf), C.byref(ms))
    if rc != OK:
        raise RuntimeError(f"asolve_pipe_peak: {strerror(rc)}")
    return tf.value, ms.value
