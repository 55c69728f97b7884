/*
 * asolve.h -- C ABI of a GB300-native (sm_103a) adaptive solver for A X = B.
 *
 * The method is the adaptive solver of Sanderson & Curtin, "An Adaptive
 * Solver for Systems of Linear Equations" (arXiv 2007.11208): a property scan
 * of A (Sec. 2.1 bandwidths, Sec. 2.2 triangularity, Sec. 2.3 / Fig. 4
 * likely-sympd), a solver chosen by the detection order of Sec. 2 (banded
 * LU, triangular substitution, Cholesky with fallback to LU, LU with partial
 * pivoting), a reciprocal condition estimate (Sec. 2, "each of the solvers
 * estimates the reciprocal condition number"), and a minimum-norm SVD solve
 * when a solver fails or rcond < 0.5 eps (Sec. 2.5).  Every step runs in the
 * library's own CUDA kernels on one GPU.
 *
 * Conventions shared by every entry point:
 *  - Matrices are FP64, dense, column-major with leading dimension n (the
 *    paper's storage, Sec. 1 and Sec. 2.1).  B and X are n x nrhs, ld = n.
 *  - Unless ASOLVE_HOST_BUFFERS is given, every matrix/vector pointer is a
 *    DEVICE pointer owned by the caller, 16-byte aligned.  A and B are never
 *    modified (like the paper's solve(A, B), Fig. 3); X may alias nothing.
 *  - The context owns its CUDA stream (or the stream given in the config),
 *    its workspaces and its CUDA graphs.  A context is not thread-safe; use
 *    one context per host thread.
 *  - Return codes: 0 = OK; > 0 = warning, X holds an answer; < 0 = error.
 *  - Work is ordered on the context stream.  Calls returning an
 *    asolve_info through a host pointer synchronise that stream before they
 *    return; the *_async / batched calls do not unless ASOLVE_SYNC is set.
 *    A stream the context creates is non-blocking: it is not ordered after
 *    work on other streams, so inputs written there must be complete (or
 *    the context stream made to wait on an event) before the call.
 *  - Test hooks for the error paths, read from the environment at each
 *    call (no GPU fault is involved): ASOLVE_FAIL_ALLOC=1 makes the
 *    context's workspace allocations fail as an out-of-memory would (the
 *    call returns E_NOMEM, the context stays usable); ASOLVE_WAIT_LIMIT=p
 *    caps the polls of the tensor-core GEMM's stage waits at p (a wait that
 *    runs out makes a solve return E_TIMEOUT and sets asolve_gemm_sub's err
 *    flag; the kernel still drains its tensor-core work before it exits).
 */
#ifndef ASOLVE_H
#define ASOLVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return / status codes ------------------------------------------- */
#define ASOLVE_OK              0
#define ASOLVE_W_APPROX        1   /* SVD fallback used (Sec. 2.5): approximate solution */
#define ASOLVE_W_ILLCOND       2   /* rcond below threshold, SVD disabled: X from the solver */
#define ASOLVE_PENDING         3   /* asolve_poll: request still in flight */
#define ASOLVE_E_INVALID      -1   /* bad argument (null pointer, n < 0, nrhs < 1, ...) */
#define ASOLVE_E_NONFINITE    -2   /* Inf or NaN in A or B */
#define ASOLVE_E_SINGULAR     -3   /* solver failed and SVD disabled; X zeroed */
#define ASOLVE_E_NOMEM        -4   /* device allocation failed / over the HBM budget */
#define ASOLVE_E_CUDA         -5   /* a CUDA call failed */
#define ASOLVE_E_TIMEOUT      -6   /* a device-side wait gave up */
#define ASOLVE_E_IR_STALL     -7   /* refinement stalled and FP64 fallback disabled */
#define ASOLVE_E_UNSUPPORTED  -8   /* size or option outside what this build supports */

/* ---- detected class (Sec. 2 detection order) ------------------------- */
#define ASOLVE_CLS_NONE     0
#define ASOLVE_CLS_BANDED   1
#define ASOLVE_CLS_LOWER    2
#define ASOLVE_CLS_UPPER    3
#define ASOLVE_CLS_SYMPD    4
#define ASOLVE_CLS_GENERAL  5

/* ---- route taken (the primary solver; SVD use is reported by status) -- */
#define ASOLVE_ROUTE_NONE          0
#define ASOLVE_ROUTE_BAND_LU       1   /* Sec. 2.1 (xGBTRF/xGBTRS/xGBCON) */
#define ASOLVE_ROUTE_TRI_LOWER     2   /* Sec. 2.2, Eq. 3 forward substitution */
#define ASOLVE_ROUTE_TRI_UPPER     3   /* Sec. 2.2 back substitution */
#define ASOLVE_ROUTE_CHOL          4   /* Sec. 2.3 (xPOTRF/xPOTRS/xPOCON) */
#define ASOLVE_ROUTE_CHOL_FAIL_LU  5   /* Sec. 2.3: Cholesky failed -> general solver */
#define ASOLVE_ROUTE_LU            6   /* Sec. 2.4, Eq. 4 (xGETRF/xGETRS/xGECON) */
#define ASOLVE_ROUTE_SVD           7   /* ASOLVE_FORCE_SVD only */
#define ASOLVE_ROUTE_TRIDIAG       8   /* with ASOLVE_TRIDIAG: a banded system with kl = ku = 1
                                          (the paper's closing remarks name tridiagonal
                                          matrices for specialised handling; xGTTRF/xGTTRS/
                                          xGTCON semantics) */
#define ASOLVE_ROUTE_LDLT          9   /* with ASOLVE_SYM_INDEF: symmetric (Fig. 4 tolerance), not
                                          likely_sympd: Bunch-Kaufman LDL^T (xSYTRF/xSYTRS/xSYCON
                                          semantics; the paper names plain symmetric matrices) */
#define ASOLVE_ROUTE_CHOL_FAIL_LDLT 10 /* with ASOLVE_SYM_INDEF: Cholesky failed -> LDL^T */

/* ---- precision of the dense factorisations --------------------------- */
#define ASOLVE_PREC_FP64    0   /* FP64 factorisations (DMMA tensor path) */
#define ASOLVE_PREC_MIXED   1   /* FP32 factors + FP64 iterative refinement; large dense
                                   systems: trailing updates as 3xTF32 tensor products
                                   (FP32-level accuracy) */
#define ASOLVE_PREC_BF16    2   /* as MIXED, but the trailing updates of large dense systems
                                   (n > 1024) are single BF16 tensor products with FP32
                                   accumulation; the refinement gate is the kappa limit of
                                   BF16 (ir_kappa_limit capped at 1e3).  Systems with
                                   n <= 1024 factor in FP32 as with MIXED */
#define ASOLVE_PREC_FP16    3   /* as BF16 with FP16 operands (per-tile power-of-two
                                   scaling); gate ir_kappa_limit capped at 1e4 */
#define ASOLVE_PREC_FP64_OZ 4   /* FP64 factorisations as ASOLVE_PREC_FP64, but on large dense
                                   systems (n > 1024) the trailing updates and the blocked
                                   triangular-solve updates are FP64-accurate Ozaki-split
                                   products on the BF16 tensor cores (asolve_gemm_oz); the
                                   FP64 re-factorisations of the mixed modes' large systems
                                   use the same products.  asolve_info.precision reports
                                   ASOLVE_PREC_FP64 and detail bit 6 (64) */
#define ASOLVE_PREC_FP8     5   /* the FP8 experiment: as FP16 with FP8 E4M3 operands
                                   (kind::f8f6f4, per-tile power-of-two scaling) in the
                                   large path's trailing updates; classical refinement
                                   gate 1e1 (unit roundoff 2^-4), GMRES-IR to kappa 1e3,
                                   else the FP64 re-factorisation */

/* ---- flags ----------------------------------------------------------- */
#define ASOLVE_NO_APPROX     0x01u  /* disable the SVD fallback (Sec. 2.5 option) */
#define ASOLVE_FORCE_LU      0x02u  /* skip structure-based routing: always LU */
#define ASOLVE_FORCE_SVD     0x04u  /* go straight to the SVD solver */
#define ASOLVE_NO_RCOND      0x08u  /* skip the condition estimate (and its SVD test) */
#define ASOLVE_SYNC          0x10u  /* synchronise the stream before returning */
#define ASOLVE_HOST_BUFFERS  0x20u  /* A, B, X (and batched arrays) are host memory */
#define ASOLVE_BERR          0x40u  /* FP64 path: also compute the backward error */
#define ASOLVE_RESIDENT      0x80u  /* request server: keep A and its factorisation on the device;
                                       a later resident request with the same A pointer (A
                                       unchanged) solves with them (systems above n = 1024 or
                                       8 right-hand sides) */
#define ASOLVE_TRIDIAG       0x100u /* tridiagonal specialisation (opt-in; the paper names it as
                                       a further improvement): banded systems with kl = ku = 1
                                       take ASOLVE_ROUTE_TRIDIAG -- elimination with partial
                                       pivoting on the three diagonals (the pivots and
                                       operations of xGTTRF), or, for long diagonally dominant
                                       systems (n >= 4096), the partitioned route */
#define ASOLVE_SYM_INDEF     0x200u /* symmetric-indefinite specialisation (opt-in; the paper names
                                       it as a further improvement), n <= 1024 and at most 8
                                       right-hand sides: a system symmetric within the Fig. 4
                                       tolerance but not likely_sympd, or whose Cholesky fails,
                                       takes Bunch-Kaufman LDL^T in FP64 (ASOLVE_ROUTE_LDLT /
                                       ASOLVE_ROUTE_CHOL_FAIL_LDLT).  With more right-hand sides
                                       and n <= 1024 the call returns E_UNSUPPORTED; above
                                       n = 1024 the flag has no effect */

typedef struct asolve_ctx asolve_ctx;

typedef struct {
  double  rcond_threshold; /* SVD if rcond < this (strict); default 0.5*DBL_EPSILON (Sec. 2.5) */
  double  sympd_tol;       /* Fig. 4 symmetry tolerance; default 100*DBL_EPSILON */
  double  band_frac;       /* Sec. 2.1: not banded if band positions > band_frac*n^2; 0.25 */
  double  svd_trunc_rel;   /* SVD keeps sigma_i > svd_trunc_rel*sigma_max; <= 0 means n*eps */
  int32_t precision;       /* ASOLVE_PREC_*; default ASOLVE_PREC_MIXED */
  int32_t ir_max_iter;     /* refinement steps before falling back to FP64; default 10 */
  double  ir_target_berr;  /* stop refining when berr <= this; default 1e-13 */
  double  ir_kappa_limit;  /* mixed: rcond < 1/limit from the FP32 factors -> FP64; default 1e9 */
  size_t  hbm_budget;      /* serving admission budget in bytes; default 120 GB */
  void*   stream;          /* cudaStream_t to run on; NULL: the context creates one */
  int32_t device;          /* CUDA device ordinal; < 0: the current device */
  int32_t reserved;
} asolve_config;

typedef struct {           /* 64 bytes, one per system */
  int32_t cls;             /* ASOLVE_CLS_* detected by the scan */
  int32_t route;           /* ASOLVE_ROUTE_* primary solver taken */
  int32_t status;          /* ASOLVE_OK / W_* / E_* for this system */
  int32_t ir_iters;        /* refinement steps taken (mixed precision) */
  int64_t kl, ku;          /* exact sub/super-diagonal counts (Sec. 2.1) */
  double  rcond;           /* estimate from the primary solver; NaN if none */
  double  berr;            /* max over columns of ||b-Ax||inf/(||A||inf||x||inf+||b||inf); NaN if not
                              computed.  Mixed precision: the backward error verified by the last FP64
                              residual; the returned X is that iterate plus the correction computed
                              from the same residual. */
  int64_t svd_rank;        /* singular values kept by the SVD solve; -1 if not used */
  int32_t precision;       /* ASOLVE_PREC_* the final answer came from */
  int32_t detail;          /* bit 0: FP32 factor rejected by the rcond gate,
                              bit 1: refinement stalled, bit 2: FP32 Cholesky failed,
                              bit 3: factorisation reused from an earlier resident request,
                              bit 4: band system solved by the partitioned route for
                              diagonally dominant bands (the default for n >= 4096;
                              environment ASOLVE_BAND_SPIKE=0 turns it off),
                              bit 5: refined by GMRES-IR (large path, BF16 / FP16 modes),
                              bit 6: large path, FP64 updates as Ozaki-split tensor-core
                              products (ASOLVE_PREC_FP64_OZ, or a mixed mode's FP64
                              re-factorisation),
                              bit 7: band system of n >= 2048 whose partitioned sweeps'
                              answer missed a backward error of 2^-46 and was refined
                              in FP64 with the same sweeps,
                              bit 8: ... and re-solved by the sequential kernels when
                              that refinement did not reach 2^-46 either */
} asolve_info;

typedef struct {           /* result of the property scan alone (Sec. 2.1, 2.2, Fig. 4) */
  int64_t kl, ku;
  int32_t lower, upper, sympd, banded;
  int32_t nonfinite, cls;
  double  norm1, norminf;  /* ||A||_1 and ||A||_inf, to 2^-17 relative (FP32 partial sums) */
} asolve_scan_result;

typedef struct {           /* per-kernel CUDA-event timing, enabled by asolve_set_profiling */
  int32_t count;           /* number of kernel kinds filled below */
  int32_t reserved;
  struct {
    char     name[40];
    int64_t  launches;
    double   total_ms;
  } k[24];
} asolve_profile;

typedef struct {           /* request-server counters (asolve_get_serve_stats) */
  int64_t submitted;       /* requests accepted (tickets issued) */
  int64_t completed;       /* requests finished, any status */
  int64_t failed;          /* finished with an error status (< 0) */
  int64_t rejected;        /* refused at submission: alone over the HBM budget */
  int64_t queued;          /* waiting for admission now */
  int64_t rounds;          /* lane rounds: batches plus large solves */
  int64_t batches;         /* batched launches of small requests */
  int64_t large_solves;    /* large systems solved */
  size_t  budget;          /* the context's hbm_budget */
  size_t  charged_bytes;   /* bytes admitted and not yet released */
  size_t  peak_charged_bytes;
  double  busy_ms;         /* wall time with at least one lane at work */
  double  wall_ms;         /* first submission to last completion */
} asolve_serve_stats;

/* Version string of this library. */
const char* asolve_version(void);
/* Text for a status code. */
const char* asolve_strerror(int code);
/* Fill *cfg with the defaults listed above.  Returns ASOLVE_E_INVALID on NULL. */
int asolve_default_config(asolve_config* cfg);

/* Create a context on cfg->device (NULL cfg: defaults).  On success *out
 * owns a stream (unless cfg->stream was given), device workspaces that grow
 * on demand, and graph caches.  Errors: E_INVALID, E_CUDA, E_NOMEM. */
int asolve_create(asolve_ctx** out, const asolve_config* cfg);
/* Release everything the context owns (waits for its stream first). */
int asolve_destroy(asolve_ctx* ctx);
/* The stream the context runs on (a cudaStream_t). */
void* asolve_stream(asolve_ctx* ctx);

/* Property scan of one n x n matrix (Sec. 2.1, 2.2, Fig. 4, plus norms);
 * A is a device pointer; *out is host memory.  Synchronous. */
int asolve_scan(asolve_ctx* ctx, const double* A, int64_t n, asolve_scan_result* out);

/* The adaptive solve of one system A X = B (Sec. 2, Fig. 2):
 *   A: n x n, B: n x nrhs, X: n x nrhs (device unless ASOLVE_HOST_BUFFERS);
 *   info: host pointer (may be NULL).  Synchronous.  n = 0 returns OK.
 * When the routed solver fails or its rcond is below the threshold, X is
 * the minimum-norm solution through the SVD (Sec. 2.5, status W_APPROX)
 * for n <= 8192; above that order the SVD fallback is not available (a
 * dense one-sided Jacobi SVD of a larger matrix is not offered): a failed
 * solver returns E_SINGULAR with X zeroed, a low rcond W_ILLCOND with the
 * solver's X, and FORCE_SVD returns E_UNSUPPORTED.  With NO_APPROX the
 * same two codes are returned at any order.
 * Returns the system's status (the value also stored in info->status). */
int asolve_solve(asolve_ctx* ctx, const double* A, const double* B, int64_t n,
                 int64_t nrhs, uint32_t flags, double* X, asolve_info* info);

/* Same, for a matrix given in band storage (Sec. 2.1 compact format):
 * AB is ldab x n column-major with A(i,j) at AB[(ku+i-j) + j*ldab],
 * ldab >= kl+ku+1, for the declared bandwidths kl, ku.  The system always
 * takes the banded route, with the true bandwidths found inside the band.
 * The SVD fallback runs on a dense copy of A, for n <= 8192; above that
 * a failure returns E_SINGULAR and a low rcond W_ILLCOND.  Synchronous. */
int asolve_solve_band(asolve_ctx* ctx, const double* AB, int64_t ldab, int64_t kl,
                      int64_t ku, const double* B, int64_t n, int64_t nrhs,
                      uint32_t flags, double* X, asolve_info* info);

/* Batched adaptive solve of `count` independent systems of uneven size,
 * packed in flat buffers: system s has A_s at A + a_off[s] (n[s] x n[s]),
 * B_s at B + b_off[s] and X_s at X + b_off[s] (n[s] x nrhs[s]).  Offsets
 * are in elements and must be even (16-byte alignment).  n[s] <= 1024.
 * n, nrhs, a_off, b_off and infos are device arrays (host arrays with
 * ASOLVE_HOST_BUFFERS, which also makes the call synchronous).  Systems
 * are scanned in one launch, routed by class on the device, and solved by
 * one persistent launch per class, replayed from a CUDA graph.  Returns
 * the launch status (per-system status is in infos[s].status). */
int asolve_solve_batched(asolve_ctx* ctx, int64_t count, const int64_t* n,
                         const int64_t* nrhs, const int64_t* a_off,
                         const int64_t* b_off, const double* A, const double* B,
                         double* X, uint32_t flags, asolve_info* infos);

/* Batched adaptive solve over per-system pointers (the paper has no batched
 * call; this is asolve_solve applied to `count` independent systems, Sec. 2
 * per system): system s solves A[s] X[s] = B[s] with A[s] n[s] x n[s] and
 * B[s], X[s] n[s] x nrhs[s], all column-major with ld = n[s], n[s] <= 1024,
 * nrhs[s] <= 8.  n, nrhs, A, B, X (arrays of device pointers) and infos are
 * DEVICE arrays; every matrix pointer must be 8-byte aligned.  Otherwise as
 * asolve_solve_batched (ASOLVE_HOST_BUFFERS is not accepted here). */
int asolve_solve_batched_ptrs(asolve_ctx* ctx, int64_t count, const int64_t* n,
                              const int64_t* nrhs, const double* const* A,
                              const double* const* B, double* const* X, uint32_t flags,
                              asolve_info* infos);

/* Request server with continuous batching (the paper has no counterpart:
 * it serves many asolve_solve calls, Sec. 2 per request, from one context).
 * asolve_submit queues one request and returns at once with a ticket.  The
 * first submission starts two server lanes, each a host thread with its own
 * stream: the batch lane solves all queued small requests (n <= 1024,
 * nrhs <= 8, same solver flags) as one class-routed batch, the large lane
 * the oldest larger request; the two overlap on the device, and requests
 * that arrive meanwhile join the next batch.  A request is admitted only
 * while the device bytes it holds fit cfg.hbm_budget with everything in
 * flight.  A, B, X: device pointers, or host pointers with
 * ASOLVE_HOST_BUFFERS (the server stages them in device memory it charges
 * to the budget); they must stay valid, and A and B unchanged, until the
 * request completes.  Allowed flags: NO_APPROX, FORCE_LU, FORCE_SVD, TRIDIAG, SYM_INDEF,
 * NO_RCOND, BERR, HOST_BUFFERS, RESIDENT (one large request's device block
 * is kept, charged to the budget, until another resident request replaces
 * it or the budget needs it).  Errors: E_INVALID, E_UNSUPPORTED
 * (n > 32768 or nrhs > 256), E_NOMEM (the request alone needs more than the
 * budget; no ticket is issued), E_CUDA.  n = 0 completes at once.
 * The server runs on its own streams and workspaces: synchronous calls on
 * the same context may run meanwhile.  asolve_destroy waits for every
 * submitted request to complete. */
int asolve_submit(asolve_ctx* ctx, const double* A, const double* B, int64_t n, int64_t nrhs,
                  uint32_t flags, double* X, uint64_t* ticket);
/* Wait up to wait_us microseconds (< 0: without limit, 0: do not wait) for
 * a ticket.  Returns ASOLVE_PENDING while the request runs.  Once it has
 * completed, returns ASOLVE_OK, fills *info (the request's own status is
 * info->status) and the submission-to-completion latency in milliseconds
 * (either pointer may be NULL), and forgets the ticket.  An unknown or
 * already returned ticket: ASOLVE_E_INVALID. */
int asolve_poll(asolve_ctx* ctx, uint64_t ticket, int64_t wait_us, asolve_info* info,
                double* latency_ms);
/* Counters of the context's request server (all zero before the first
 * submission, except budget). */
int asolve_get_serve_stats(asolve_ctx* ctx, asolve_serve_stats* out);

/* Property scan that allocates nothing (the paper has no counterpart: this
 * entry point exists for callers that may not allocate device memory --
 * code that must not enter the allocator, hosts that own every device byte
 * through their own pool, or callers without an asolve context).
 *   A:      device pointer, n x n column-major, n <= 2048.
 *   out:    DEVICE pointer to one asolve_scan_result, written on `stream`
 *           (read it after synchronising that stream).
 *   stream: cudaStream_t to run on; NULL is the legacy default stream.
 * Uses the paper's default band fraction (0.25) and symmetry tolerance
 * (100 eps).  The workspace is a fixed 1.125 MiB device array inside the
 * library, held by every GPU that loads it until the process exits and
 * shared by all calls: calls that overlap on the GPU race and must be
 * ordered by the caller.  The first call on each device looks up that
 * array's device address (make it before any stream capture).
 * Returns E_UNSUPPORTED for n > 2048, E_INVALID for bad arguments,
 * E_CUDA if a launch fails; never allocates. */
int asolve_scan_noalloc(const double* A, int64_t n, asolve_scan_result* out, void* stream);

/* The trailing-update GEMM of the large dense factorisations (Sec. 2.3/2.4
 * blocked Cholesky/LU updates), exposed so it can be verified on its own:
 *   C (M x N) -= A (M x K) * B (K x N), FP32, column-major, device pointers,
 * computed on the tcgen05 tensor cores with FP32 accumulation.  passes:
 * ASOLVE_GEMM_TF32X3 (3) splits every operand into a TF32 head and
 * remainder (three products, FP32-level accuracy), ASOLVE_GEMM_TF32 (1) is
 * plain TF32, ASOLVE_GEMM_BF16 / ASOLVE_GEMM_FP16 round every operand once
 * to the 16-bit type (FP16 tiles scaled by powers of two from each tile's
 * largest magnitude), ASOLVE_GEMM_FP8 to FP8 E4M3 (kind::f8f6f4, per-tile
 * power-of-two scales as FP16; the configuration's FP8 experiment).  err: optional device int set to 1 if a device-side
 * wait gave up.  Asynchronous on `stream`.  Errors: E_INVALID for another
 * `passes` value. */
#define ASOLVE_GEMM_TF32    1
#define ASOLVE_GEMM_TF32X3  3
#define ASOLVE_GEMM_BF16    16
#define ASOLVE_GEMM_FP16    17
#define ASOLVE_GEMM_FP8     18
int asolve_gemm_sub(float* C, int64_t ldc, const float* A, int64_t lda, const float* B, int64_t ldb,
                    int64_t M, int64_t N, int64_t K, int passes, int* err, void* stream);

/* The FP64 product of the large path's FP64 trailing updates, blocked
 * triangular-solve updates and many-right-hand-side residuals (Sec. 2.2-2.4
 * in FP64), exposed so it can be verified on its own:
 *   C (M x N) -= A (M x K) * op(B), FP64, column-major, device pointers,
 * op(B) = B (K x N, ldb >= K) or, with transb != 0, B^T for B stored N x K
 * (ldb >= N).  Computed by the Ozaki splitting (Ozaki, Ogita, Oishi, Rump
 * 2012; the paper has no counterpart): each operand becomes seven exact
 * BF16 slices (per-row / per-column power-of-two scales over each K chunk
 * of 128), the 28 significant slice products accumulate exactly in FP32 on
 * the tcgen05 tensor cores, and each chunk is added to C in FP64; the error
 * is about 2^-48 (max_k |A(i,k)|) (max_k |op(B)(k,j)|) per chunk of 128,
 * that of an FP64 GEMM.  A or B non-finite in a chunk: C(i,j) becomes NaN.
 * ws: device workspace of asolve_gemm_oz_ws_bytes(M, N, K) bytes, 256-byte
 * aligned, owned by the caller (its content is scratch).  err: optional
 * device int set to 1 if a device-side wait gave up.  Asynchronous on
 * `stream`.  Errors: E_INVALID (null pointer, leading dimension, workspace
 * too small or unaligned), E_UNSUPPORTED (a size above 2^31 - 1), E_CUDA. */
size_t asolve_gemm_oz_ws_bytes(int64_t M, int64_t N, int64_t K);
int asolve_gemm_oz(double* C, int64_t ldc, const double* A, int64_t lda, const double* B, int64_t ldb,
                   int64_t M, int64_t N, int64_t K, int transb, void* ws, size_t ws_bytes, int* err,
                   void* stream);

/* Panel widths of the batched dense factorisations, one per size bucket
 * (bucket i holds n in [32 i + 1, 32 i + 32]), as chosen by the autotuner
 * (paper_2007_11208_gb300/autotune.py; the paper has no counterpart: it is
 * a tuning knob of this implementation).  kind: 0 LU FP32, 1 Cholesky FP32,
 * 2 LU FP64, 3 Cholesky FP64.  Each value is 0 (built-in rule) or 4, 8, 16,
 * 32; a value wider than what fits the kernel's shared memory is narrowed.
 * Buckets past `count` revert to the built-in rule.  Applies to calls made
 * after it returns.  Errors: E_INVALID. */
int asolve_set_panel_widths(asolve_ctx* ctx, int kind, const int32_t* nb, int count);

/* Issue-rate probe of one arithmetic pipe on the current device (the paper
 * has no counterpart: it measures the roofline denominators of this
 * implementation's FP32-factor and FP64-refinement kernels, which no copy
 * or library-GEMM measurement bounds).  pipe: ASOLVE_PIPE_FFMA (FP32 fused
 * multiply-add), ASOLVE_PIPE_DFMA (FP64 fused multiply-add) or
 * ASOLVE_PIPE_DMMA (the FP64 tensor instruction mma.sync m8n8k4).  Runs a
 * grid of 8 CTAs x 256 threads per SM, each thread (each warp for DMMA)
 * with 8 independent accumulator chains, `iters` rounds of 16 FMAs (4 DMMA)
 * per chain, after a shorter warm-up launch, and returns the rate in
 * *tflops (2 flops per FMA, 512 per m8n8k4) and the timed launch's duration
 * in *ms (may be NULL), measured with CUDA events on the legacy default
 * stream.  Allocates and frees a small device buffer.  Errors: E_INVALID
 * (unknown pipe, iters < 1, tflops NULL), E_NOMEM, E_CUDA. */
#define ASOLVE_PIPE_FFMA  1
#define ASOLVE_PIPE_DFMA  2
#define ASOLVE_PIPE_DMMA  3
int asolve_pipe_peak(int pipe, int iters, double* tflops, double* ms);

/* Per-kernel timing with CUDA events on the context stream (off by default). */
int asolve_set_profiling(asolve_ctx* ctx, int on);
int asolve_get_profile(asolve_ctx* ctx, asolve_profile* out);
int asolve_reset_profile(asolve_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* ASOLVE_H */
