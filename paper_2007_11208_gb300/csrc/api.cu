// api.cu -- the C ABI (include/asolve.h): contexts, workspaces, the captured
// class-routed pipeline, and the single-system / batched entry points.
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <stdint.h>

#include "asolve_internal.cuh"

namespace asv {
cudaError_t launch_scan_batched(const BatchDesc* d, int grid, cudaStream_t st);
cudaError_t launch_route(const BatchDesc* d, cudaStream_t st);
cudaError_t launch_band(const BatchDesc* d, int grid, cudaStream_t st);
cudaError_t launch_tri(const BatchDesc* d, int grid, cudaStream_t st);
cudaError_t launch_chol(const BatchDesc* d, int grid, cudaStream_t st);
cudaError_t launch_lu(const BatchDesc* d, int grid, cudaStream_t st);
cudaError_t launch_svd(const BatchDesc* d, int grid, cudaStream_t st);
cudaError_t set_class_attrs();
size_t dense_slot_bytes(int nmax);
size_t scan_slot_bytes(int nmax);
size_t scan_large_workspace(int64_t n);
cudaError_t launch_scan_large(const double* A, int64_t n, const double* B, int64_t nb, double band_frac,
                              double tol, void* ws, ScanRes* out, int num_sms, cudaStream_t st);
cudaError_t launch_gemm_tc(float* C, int ldc, const float* A, int lda, const float* B, int ldb, int M, int N,
                           int K, int passes, int* err, cudaStream_t st, bool trans_b, bool lower);
void serve_shutdown(asolve_ctx* c);
}  // namespace asv

using namespace asv;

namespace {

enum KernelId { K_SCAN = 0, K_ROUTE, K_BAND, K_TRI, K_CHOL, K_LU, K_SVD, K_COUNT };
const char* kKernelNames[K_COUNT] = {"k_scan_batched", "k_route", "k_band_class", "k_tri_class",
                                     "k_chol_class", "k_lu_class", "k_svd_class"};

// Allocation-failure injection for tests of the error paths (no GPU fault
// involved): while the environment variable ASOLVE_FAIL_ALLOC is 1, every
// workspace allocation below fails as an out-of-memory would; the call
// returns E_NOMEM and the context stays usable.
bool alloc_fault_injected() {
  const char* e = getenv("ASOLVE_FAIL_ALLOC");
  return e && e[0] == '1' && e[1] == 0;
}

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t need) {
    if (need <= bytes) return cudaSuccess;
    if (alloc_fault_injected()) return cudaErrorMemoryAllocation;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    cudaError_t e = cudaMalloc(&p, need);
    if (e == cudaSuccess) bytes = need;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
};

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t memcpy_node = nullptr;
};

}  // namespace

struct asolve_ctx {
  asolve_config cfg;
  int device = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // batched pipeline state
  int64_t capacity = 0;
  DevBuf scan, lists, small;  // small: list_len[8] + work_ctr[32] + err
  DevBuf slots;
  size_t slot_bytes = 0;
  int slot_count = 0;
  BatchDesc* d_desc = nullptr;
  BatchDesc* h_desc = nullptr;  // pinned
  std::map<int64_t, GraphEntry> graphs;
  // single-system staging
  DevBuf single;       // n, nrhs, a_off, b_off, info (device)
  int64_t* h_single = nullptr;  // pinned: 4 int64 + asolve_info
  DevBuf hostA, hostB, hostX, hostMeta;  // device copies for ASOLVE_HOST_BUFFERS
  DevBuf large;        // large-system / banded workspace
  DevBuf bandDense;    // dense copy of a band-stored matrix (SVD fallback)
  ScanRes* h_scan = nullptr;  // pinned
  int8_t nb_tab[4][32] = {};  // tuned panel widths (0: built-in rule)
  // request server (created by the first asolve_submit)
  void* serve = nullptr;
  // profiling
  bool profiling = false;
  cudaEvent_t ev[K_COUNT + 1] = {};
  double prof_ms[K_COUNT] = {};
  int64_t prof_launches[K_COUNT] = {};
};

namespace asv {
// Accessors for the request server (serve.cu).
const asolve_config* ctx_config(asolve_ctx* c) { return &c->cfg; }
int ctx_device(asolve_ctx* c) { return c->device; }
int ctx_num_sms(asolve_ctx* c) { return c->num_sms; }
void** ctx_serve_slot(asolve_ctx* c) { return &c->serve; }
}  // namespace asv

static int cuda_fail(cudaError_t e) {
  if (e == cudaErrorMemoryAllocation) return ASOLVE_E_NOMEM;
  return ASOLVE_E_CUDA;
}
#define CK(x)                                  \
  do {                                         \
    cudaError_t _e = (x);                      \
    if (_e != cudaSuccess) return cuda_fail(_e); \
  } while (0)

extern "C" const char* asolve_version(void) { return "asolve 0.1 (sm_103a)"; }

extern "C" const char* asolve_strerror(int code) {
  switch (code) {
    case ASOLVE_OK: return "ok";
    case ASOLVE_W_APPROX: return "approximate solution (SVD fallback)";
    case ASOLVE_W_ILLCOND: return "ill-conditioned (rcond below threshold)";
    case ASOLVE_PENDING: return "pending";
    case ASOLVE_E_INVALID: return "invalid argument";
    case ASOLVE_E_NONFINITE: return "non-finite input";
    case ASOLVE_E_SINGULAR: return "singular (solver failed, SVD disabled)";
    case ASOLVE_E_NOMEM: return "out of device memory";
    case ASOLVE_E_CUDA: return "CUDA error";
    case ASOLVE_E_TIMEOUT: return "device wait timed out";
    case ASOLVE_E_IR_STALL: return "refinement stalled";
    case ASOLVE_E_UNSUPPORTED: return "unsupported size or option";
    default: return "unknown status";
  }
}

extern "C" int asolve_default_config(asolve_config* c) {
  if (!c) return ASOLVE_E_INVALID;
  memset(c, 0, sizeof(*c));
  c->rcond_threshold = 0.5 * DBL_EPSILON;
  c->sympd_tol = 100.0 * DBL_EPSILON;
  c->band_frac = 0.25;
  c->svd_trunc_rel = 0.0;
  c->precision = ASOLVE_PREC_MIXED;
  c->ir_max_iter = 10;
  c->ir_target_berr = 1e-13;
  c->ir_kappa_limit = 1e9;
  c->hbm_budget = (size_t)120 << 30;
  c->stream = nullptr;
  c->device = -1;
  return ASOLVE_OK;
}

extern "C" int asolve_create(asolve_ctx** out, const asolve_config* cfg) {
  if (!out) return ASOLVE_E_INVALID;
  *out = nullptr;
  asolve_ctx* c = new (std::nothrow) asolve_ctx();
  if (!c) return ASOLVE_E_NOMEM;
  if (cfg) c->cfg = *cfg;
  else asolve_default_config(&c->cfg);
  if (c->cfg.precision < ASOLVE_PREC_FP64 || c->cfg.precision > ASOLVE_PREC_FP8) {
    delete c;
    return ASOLVE_E_INVALID;
  }
  int dev = c->cfg.device;
  if (dev < 0) {
    if (cudaGetDevice(&dev) != cudaSuccess) { delete c; return ASOLVE_E_CUDA; }
  }
  c->device = dev;
  if (cudaSetDevice(dev) != cudaSuccess) { delete c; return ASOLVE_E_CUDA; }
  if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    delete c;
    return ASOLVE_E_CUDA;
  }
  if (c->cfg.stream) {
    c->stream = (cudaStream_t)c->cfg.stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return ASOLVE_E_CUDA;
    }
    c->own_stream = true;
  }
  if (cudaMalloc(&c->d_desc, sizeof(BatchDesc)) != cudaSuccess ||
      cudaMallocHost(&c->h_desc, sizeof(BatchDesc)) != cudaSuccess ||
      cudaMallocHost(&c->h_single, 4 * sizeof(int64_t) + sizeof(asolve_info)) != cudaSuccess ||
      cudaMallocHost(&c->h_scan, sizeof(ScanRes)) != cudaSuccess) {
    asolve_destroy(c);
    return ASOLVE_E_NOMEM;
  }
  for (int k = 0; k <= K_COUNT; ++k) cudaEventCreate(&c->ev[k]);
  if (set_class_attrs() != cudaSuccess) {
    asolve_destroy(c);
    return ASOLVE_E_CUDA;
  }
  *out = c;
  return ASOLVE_OK;
}

extern "C" int asolve_destroy(asolve_ctx* c) {
  if (!c) return ASOLVE_E_INVALID;
  serve_shutdown(c);  // waits for every submitted request
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (auto& kv : c->graphs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  c->graphs.clear();
  c->scan.release();
  c->lists.release();
  c->small.release();
  c->slots.release();
  c->single.release();
  c->hostA.release();
  c->hostB.release();
  c->hostX.release();
  c->hostMeta.release();
  c->large.release();
  c->bandDense.release();
  if (c->d_desc) cudaFree(c->d_desc);
  if (c->h_desc) cudaFreeHost(c->h_desc);
  if (c->h_single) cudaFreeHost(c->h_single);
  if (c->h_scan) cudaFreeHost(c->h_scan);
  for (int k = 0; k <= K_COUNT; ++k)
    if (c->ev[k]) cudaEventDestroy(c->ev[k]);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
  return ASOLVE_OK;
}

extern "C" void* asolve_stream(asolve_ctx* c) { return c ? (void*)c->stream : nullptr; }

// Grow the pipeline state to hold `count` systems; (re)allocates slots once.
static int ensure_pipeline(asolve_ctx* c, int64_t count) {
  if (count > c->capacity) {
    int64_t cap = 1;
    while (cap < count) cap <<= 1;
    CK(c->scan.ensure(sizeof(ScanRes) * cap));
    CK(c->lists.ensure(sizeof(int32_t) * L_COUNT * cap));
    c->capacity = cap;
    // graphs captured with the old capacity are stale
    for (auto& kv : c->graphs)
      if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    c->graphs.clear();
  }
  CK(c->small.ensure(64 * sizeof(int32_t)));
  if (!c->slots.p) {
    size_t sb = dense_slot_bytes(kBatchNMax);
    size_t ss = scan_slot_bytes(kBatchNMax);
    if (ss > sb) sb = ss;
    int ns = c->num_sms * 2;
    CK(c->slots.ensure(sb * (size_t)ns));
    c->slot_bytes = sb;
    c->slot_count = ns;
  }
  return ASOLVE_OK;
}

static void fill_desc(asolve_ctx* c, BatchDesc* h, int64_t count, const int64_t* n, const int64_t* nrhs,
                      const int64_t* a_off, const int64_t* b_off, const double* A, const double* B,
                      double* X, asolve_info* info, uint32_t flags) {
  memset(h, 0, sizeof(*h));
  h->count = count;
  h->n = n;
  h->nrhs = nrhs;
  h->a_off = a_off;
  h->b_off = b_off;
  h->A = A;
  h->B = B;
  h->X = X;
  h->info = info;
  h->flags = flags;
  h->precision = c->cfg.precision;
  h->rcond_threshold = c->cfg.rcond_threshold;
  h->sympd_tol = c->cfg.sympd_tol;
  h->band_frac = c->cfg.band_frac;
  h->svd_trunc_rel = c->cfg.svd_trunc_rel;
  h->ir_max_iter = c->cfg.ir_max_iter;
  h->ir_target_berr = c->cfg.ir_target_berr;
  h->ir_kappa_limit = c->cfg.ir_kappa_limit;
  h->scan = (ScanRes*)c->scan.p;
  h->lists = (int32_t*)c->lists.p;
  h->list_len = (int32_t*)c->small.p;
  h->work_ctr = (int32_t*)c->small.p + 8;
  h->err_flag = (int32_t*)c->small.p + 40;
  h->capacity = c->capacity;
  h->slot_base = (char*)c->slots.p;
  h->slot_bytes = (int64_t)c->slot_bytes;
  h->slot_count = c->slot_count;
  memcpy(h->nb_tab, c->nb_tab, sizeof(h->nb_tab));
}

// Enqueue the pipeline kernels (used both for capture and for profiling).
static cudaError_t enqueue_kernels(asolve_ctx* c, int grid, bool prof) {
  cudaStream_t st = c->stream;
  cudaError_t e;
  const BatchDesc* d = c->d_desc;
  if (prof) cudaEventRecord(c->ev[0], st);
  int gscan = grid;
  if ((e = launch_scan_batched(d, gscan, st)) != cudaSuccess) return e;
  if (prof) cudaEventRecord(c->ev[1], st);
  if ((e = launch_route(d, st)) != cudaSuccess) return e;
  if (prof) cudaEventRecord(c->ev[2], st);
  if ((e = launch_band(d, grid, st)) != cudaSuccess) return e;
  if (prof) cudaEventRecord(c->ev[3], st);
  if ((e = launch_tri(d, grid, st)) != cudaSuccess) return e;
  if (prof) cudaEventRecord(c->ev[4], st);
  if ((e = launch_chol(d, grid, st)) != cudaSuccess) return e;
  if (prof) cudaEventRecord(c->ev[5], st);
  if ((e = launch_lu(d, grid, st)) != cudaSuccess) return e;
  if (prof) cudaEventRecord(c->ev[6], st);
  if ((e = launch_svd(d, grid, st)) != cudaSuccess) return e;
  if (prof) cudaEventRecord(c->ev[7], st);
  return cudaSuccess;
}

static int grid_for(asolve_ctx* c, int64_t count) {
  int64_t g = 1;
  while (g < count && g < c->slot_count) g <<= 1;
  if (g > c->slot_count) g = c->slot_count;
  return (int)g;
}

// Run the pipeline for the descriptor already in c->h_desc.
static int run_pipeline(asolve_ctx* c, int64_t count) {
  cudaStream_t st = c->stream;
  const int grid = grid_for(c, count);
  if (c->profiling) {
    CK(cudaMemcpyAsync(c->d_desc, c->h_desc, sizeof(BatchDesc), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(c->small.p, 0, 64 * sizeof(int32_t), st));
    CK(enqueue_kernels(c, grid, true));
    CK(cudaStreamSynchronize(st));
    for (int k = 0; k < K_COUNT; ++k) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, c->ev[k], c->ev[k + 1]);
      c->prof_ms[k] += ms;
      c->prof_launches[k] += 1;
    }
    return ASOLVE_OK;
  }
  auto it = c->graphs.find(grid);
  if (it == c->graphs.end()) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    cudaError_t e1 = cudaMemcpyAsync(c->d_desc, c->h_desc, sizeof(BatchDesc), cudaMemcpyHostToDevice, st);
    cudaError_t e2 = cudaMemsetAsync(c->small.p, 0, 64 * sizeof(int32_t), st);
    cudaError_t e3 = enqueue_kernels(c, grid, false);
    cudaError_t e4 = cudaStreamEndCapture(st, &g);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || e4 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return ASOLVE_E_CUDA;
    }
    GraphEntry ge;
    cudaError_t e5 = cudaGraphInstantiate(&ge.exec, g, 0);
    cudaGraphDestroy(g);
    if (e5 != cudaSuccess) return ASOLVE_E_CUDA;
    it = c->graphs.emplace(grid, ge).first;
  }
  CK(cudaGraphLaunch(it->second.exec, st));
  // the graph's first node reads h_desc: do not let the host overwrite it
  // before that copy has run
  CK(cudaStreamSynchronize(st));
  return ASOLVE_OK;
}

extern "C" int asolve_solve_batched(asolve_ctx* c, int64_t count, const int64_t* n, const int64_t* nrhs,
                                    const int64_t* a_off, const int64_t* b_off, const double* A,
                                    const double* B, double* X, uint32_t flags, asolve_info* infos) {
  if (!c || count < 0) return ASOLVE_E_INVALID;
  if (count == 0) return ASOLVE_OK;
  if (!n || !nrhs || !a_off || !b_off || !A || !B || !X || !infos) return ASOLVE_E_INVALID;
  CK(cudaSetDevice(c->device));
  int rc = ensure_pipeline(c, count);
  if (rc) return rc;
  if (flags & ASOLVE_HOST_BUFFERS) {
    // sizes from the host arrays
    int64_t na = 0, nb = 0;
    for (int64_t s = 0; s < count; ++s) {
      if (n[s] < 0 || nrhs[s] < 1 || a_off[s] < 0 || b_off[s] < 0 || (a_off[s] & 1) || (b_off[s] & 1))
        return ASOLVE_E_INVALID;
      int64_t ea = a_off[s] + n[s] * n[s], eb = b_off[s] + n[s] * nrhs[s];
      if (ea > na) na = ea;
      if (eb > nb) nb = eb;
    }
    CK(c->hostA.ensure(sizeof(double) * (size_t)(na > 0 ? na : 1)));
    CK(c->hostB.ensure(sizeof(double) * (size_t)(nb > 0 ? nb : 1)));
    CK(c->hostX.ensure(sizeof(double) * (size_t)(nb > 0 ? nb : 1)));
    CK(c->hostMeta.ensure((4 * sizeof(int64_t) + sizeof(asolve_info)) * (size_t)count));
    int64_t* dm = (int64_t*)c->hostMeta.p;
    asolve_info* dinf = (asolve_info*)(dm + 4 * count);
    cudaStream_t st = c->stream;
    CK(cudaMemcpyAsync(dm, n, sizeof(int64_t) * count, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(dm + count, nrhs, sizeof(int64_t) * count, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(dm + 2 * count, a_off, sizeof(int64_t) * count, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(dm + 3 * count, b_off, sizeof(int64_t) * count, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->hostA.p, A, sizeof(double) * (size_t)na, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->hostB.p, B, sizeof(double) * (size_t)nb, cudaMemcpyHostToDevice, st));
    fill_desc(c, c->h_desc, count, dm, dm + count, dm + 2 * count, dm + 3 * count,
              (const double*)c->hostA.p, (const double*)c->hostB.p, (double*)c->hostX.p, dinf, flags);
    rc = run_pipeline(c, count);
    if (rc) return rc;
    CK(cudaMemcpyAsync(X, c->hostX.p, sizeof(double) * (size_t)nb, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(infos, dinf, sizeof(asolve_info) * count, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return ASOLVE_OK;
  }
  fill_desc(c, c->h_desc, count, n, nrhs, a_off, b_off, A, B, X, infos, flags);
  rc = run_pipeline(c, count);
  if (rc) return rc;
  if (flags & ASOLVE_SYNC) CK(cudaStreamSynchronize(c->stream));
  return ASOLVE_OK;
}

extern "C" int asolve_solve_batched_ptrs(asolve_ctx* c, int64_t count, const int64_t* n,
                                         const int64_t* nrhs, const double* const* A,
                                         const double* const* B, double* const* X, uint32_t flags,
                                         asolve_info* infos) {
  if (!c || count < 0) return ASOLVE_E_INVALID;
  if (count == 0) return ASOLVE_OK;
  if (!n || !nrhs || !A || !B || !X || !infos) return ASOLVE_E_INVALID;
  if (flags & ASOLVE_HOST_BUFFERS) return ASOLVE_E_UNSUPPORTED;
  CK(cudaSetDevice(c->device));
  int rc = ensure_pipeline(c, count);
  if (rc) return rc;
  fill_desc(c, c->h_desc, count, n, nrhs, nullptr, nullptr, nullptr, nullptr, nullptr, infos, flags);
  c->h_desc->Ap = A;
  c->h_desc->Bp = B;
  c->h_desc->Xp = X;
  rc = run_pipeline(c, count);
  if (rc) return rc;
  if (flags & ASOLVE_SYNC) CK(cudaStreamSynchronize(c->stream));
  return ASOLVE_OK;
}

extern "C" int asolve_solve(asolve_ctx* c, const double* A, const double* B, int64_t n, int64_t nrhs,
                            uint32_t flags, double* X, asolve_info* info) {
  if (!c || n < 0 || nrhs < 1) return ASOLVE_E_INVALID;
  if (n == 0) {
    if (info) {
      memset(info, 0, sizeof(*info));
      info->rcond = NAN;
      info->berr = NAN;
      info->svd_rank = -1;
    }
    return ASOLVE_OK;
  }
  if (!A || !B || !X) return ASOLVE_E_INVALID;
  CK(cudaSetDevice(c->device));
  if (n > kBatchNMax || nrhs > kBatchRhsMax) {
    // one large system: blocked factorisations over the whole GPU
    if (n > 32768 || nrhs > 256) return ASOLVE_E_UNSUPPORTED;
    cudaStream_t st = c->stream;
    const double *dA = A, *dB = B;
    double* dX = X;
    if (flags & ASOLVE_HOST_BUFFERS) {
      CK(c->hostA.ensure(sizeof(double) * (size_t)(n * n)));
      CK(c->hostB.ensure(sizeof(double) * (size_t)(n * nrhs)));
      CK(c->hostX.ensure(sizeof(double) * (size_t)(n * nrhs)));
      CK(cudaMemcpyAsync(c->hostA.p, A, sizeof(double) * (size_t)(n * n), cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(c->hostB.p, B, sizeof(double) * (size_t)(n * nrhs), cudaMemcpyHostToDevice, st));
      dA = (const double*)c->hostA.p;
      dB = (const double*)c->hostB.p;
      dX = (double*)c->hostX.p;
    }
    const size_t wsb = large_ws_bytes(n, nrhs);
    CK(c->large.ensure(wsb));
    LargeArgs la{dA, dB, dX, n, nrhs, flags, c->cfg.precision, c->cfg.rcond_threshold, c->cfg.sympd_tol,
                 c->cfg.band_frac, c->cfg.ir_target_berr, c->cfg.ir_kappa_limit, c->cfg.ir_max_iter,
                 c->num_sms, st, nullptr, c->cfg.svd_trunc_rel};
    asolve_info li;
    const int rc = large_solve(la, c->large.p, c->large.bytes, &li);
    if (rc < 0 && rc != li.status) {  // an error before the solve produced a status
      li.status = rc;
      if (info) *info = li;
      return rc;
    }
    if (flags & ASOLVE_HOST_BUFFERS) {
      CK(cudaMemcpyAsync(X, dX, sizeof(double) * (size_t)(n * nrhs), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
    }
    if (info) *info = li;
    return li.status;
  }
  int rc = ensure_pipeline(c, 1);
  if (rc) return rc;
  CK(c->single.ensure(4 * sizeof(int64_t) + sizeof(asolve_info)));
  cudaStream_t st = c->stream;
  const double *dA = A, *dB = B;
  double* dX = X;
  if (flags & ASOLVE_HOST_BUFFERS) {
    CK(c->hostA.ensure(sizeof(double) * (size_t)(n * n)));
    CK(c->hostB.ensure(sizeof(double) * (size_t)(n * nrhs)));
    CK(c->hostX.ensure(sizeof(double) * (size_t)(n * nrhs)));
    CK(cudaMemcpyAsync(c->hostA.p, A, sizeof(double) * (size_t)(n * n), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->hostB.p, B, sizeof(double) * (size_t)(n * nrhs), cudaMemcpyHostToDevice, st));
    dA = (const double*)c->hostA.p;
    dB = (const double*)c->hostB.p;
    dX = (double*)c->hostX.p;
  }
  int64_t* hs = c->h_single;
  hs[0] = n;
  hs[1] = nrhs;
  hs[2] = 0;
  hs[3] = 0;
  int64_t* ds = (int64_t*)c->single.p;
  asolve_info* dinf = (asolve_info*)(ds + 4);
  CK(cudaMemcpyAsync(ds, hs, 4 * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  fill_desc(c, c->h_desc, 1, ds, ds + 1, ds + 2, ds + 3, dA, dB, dX, dinf, flags);
  rc = run_pipeline(c, 1);
  if (rc) return rc;
  asolve_info* hinf = (asolve_info*)(c->h_single + 4);
  CK(cudaMemcpyAsync(hinf, dinf, sizeof(asolve_info), cudaMemcpyDeviceToHost, st));
  if (flags & ASOLVE_HOST_BUFFERS)
    CK(cudaMemcpyAsync(X, dX, sizeof(double) * (size_t)(n * nrhs), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (info) *info = *hinf;
  return hinf->status;
}

extern "C" int asolve_scan(asolve_ctx* c, const double* A, int64_t n, asolve_scan_result* out) {
  if (!c || !out || n < 0 || (n > 0 && !A)) return ASOLVE_E_INVALID;
  memset(out, 0, sizeof(*out));
  if (n == 0) return ASOLVE_OK;
  CK(cudaSetDevice(c->device));
  cudaStream_t st = c->stream;
  size_t ws = scan_large_workspace(n);
  CK(c->large.ensure(ws + sizeof(ScanRes) + 256));
  ScanRes* d_out = (ScanRes*)((char*)c->large.p + ((ws + 255) & ~(size_t)255));
  CK(launch_scan_large(A, n, A, 0, c->cfg.band_frac, c->cfg.sympd_tol, c->large.p, d_out, c->num_sms, st));
  CK(cudaMemcpyAsync(c->h_scan, d_out, sizeof(ScanRes), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const ScanRes& r = *c->h_scan;
  out->kl = r.kl;
  out->ku = r.ku;
  out->lower = (r.flags & SF_LOWER) != 0;
  out->upper = (r.flags & SF_UPPER) != 0;
  out->sympd = (r.flags & SF_SYMPD) != 0;
  out->banded = (r.flags & SF_BANDED) != 0;
  out->nonfinite = (r.flags & SF_NONFINITE) != 0;
  out->cls = r.cls;
  out->norm1 = r.norm1;
  out->norminf = r.norminf;
  return ASOLVE_OK;
}

extern "C" int asolve_solve_band(asolve_ctx* c, const double* AB, int64_t ldab, int64_t kl, int64_t ku,
                                 const double* B, int64_t n, int64_t nrhs, uint32_t flags, double* X,
                                 asolve_info* info) {
  if (!c || n < 0 || nrhs < 1 || kl < 0 || ku < 0 || ldab < kl + ku + 1) return ASOLVE_E_INVALID;
  if (n == 0) {
    if (info) {
      memset(info, 0, sizeof(*info));
      info->rcond = NAN;
      info->berr = NAN;
      info->svd_rank = -1;
    }
    return ASOLVE_OK;
  }
  if (!AB || !B || !X) return ASOLVE_E_INVALID;
  if (n > INT32_MAX / 2 || nrhs > 256) return ASOLVE_E_UNSUPPORTED;
  // the true bandwidths never exceed n - 1
  const int64_t kle = kl < n - 1 ? kl : n - 1, kue = ku < n - 1 ? ku : n - 1;
  if (!band_window_fits(kle, kue)) return ASOLVE_E_UNSUPPORTED;
  CK(cudaSetDevice(c->device));
  cudaStream_t st = c->stream;
  const double* dAB = AB;
  const double* dB = B;
  double* dX = X;
  if (flags & ASOLVE_HOST_BUFFERS) {
    CK(c->hostA.ensure(sizeof(double) * (size_t)(ldab * n)));
    CK(c->hostB.ensure(sizeof(double) * (size_t)(n * nrhs)));
    CK(c->hostX.ensure(sizeof(double) * (size_t)(n * nrhs)));
    CK(cudaMemcpyAsync(c->hostA.p, AB, sizeof(double) * (size_t)(ldab * n), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->hostB.p, B, sizeof(double) * (size_t)(n * nrhs), cudaMemcpyHostToDevice, st));
    dAB = (const double*)c->hostA.p;
    dB = (const double*)c->hostB.p;
    dX = (double*)c->hostX.p;
  }
  CK(c->large.ensure(band_ws_bytes(n, kle, kue, nrhs)));
  BandArgs ba{dAB, ldab, kl, ku, nullptr, dB, dX, n, nrhs, flags, c->cfg.rcond_threshold, 0, 0, 0.0, 0.0, st};
  asolve_info li;
  int rc = band_solve(ba, c->large.p, c->large.bytes, &li);
  if (rc == ASOLVE_PENDING) {
    // solver failed or rcond below the threshold: the SVD fallback of
    // Sec. 2.5 on a dense copy (n <= kSvdLargeMax here)
    CK(c->bandDense.ensure(sizeof(double) * (size_t)(n * n)));
    int r2 = band_to_dense(dAB, ldab, kl, ku, n, (double*)c->bandDense.p, st);
    if (r2 != ASOLVE_OK) return r2;
    asolve_info si;
    r2 = asolve_solve(c, (const double*)c->bandDense.p, dB, n, nrhs,
                      (flags & ~(ASOLVE_HOST_BUFFERS | ASOLVE_FORCE_LU)) | ASOLVE_FORCE_SVD, dX, &si);
    if (r2 < 0 && si.status >= 0) si.status = r2;
    li.status = si.status;
    li.svd_rank = si.svd_rank;
    li.berr = si.berr;
    rc = li.status;
  }
  if (flags & ASOLVE_HOST_BUFFERS) {
    CK(cudaMemcpyAsync(X, dX, sizeof(double) * (size_t)(n * nrhs), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  if (info) *info = li;
  return li.status;
}

extern "C" int asolve_gemm_sub(float* C, int64_t ldc, const float* A, int64_t lda, const float* B, int64_t ldb,
                               int64_t M, int64_t N, int64_t K, int passes, int* err, void* stream) {
  if (!C || !A || !B || M < 0 || N < 0 || K < 0 ||
      (passes != ASOLVE_GEMM_TF32 && passes != ASOLVE_GEMM_TF32X3 && passes != ASOLVE_GEMM_BF16 &&
       passes != ASOLVE_GEMM_FP16 && passes != ASOLVE_GEMM_FP8))
    return ASOLVE_E_INVALID;
  if (ldc < (M > 0 ? M : 1) || lda < (M > 0 ? M : 1) || ldb < (K > 0 ? K : 1)) return ASOLVE_E_INVALID;
  if (M > INT32_MAX || N > INT32_MAX || K > INT32_MAX || ldc > INT32_MAX || lda > INT32_MAX || ldb > INT32_MAX)
    return ASOLVE_E_UNSUPPORTED;
  if (M == 0 || N == 0 || K == 0) return ASOLVE_OK;
  cudaError_t e = launch_gemm_tc(C, (int)ldc, A, (int)lda, B, (int)ldb, (int)M, (int)N, (int)K, passes, err,
                                 (cudaStream_t)stream, false, false);
  return e == cudaSuccess ? ASOLVE_OK : ASOLVE_E_CUDA;
}

extern "C" size_t asolve_gemm_oz_ws_bytes(int64_t M, int64_t N, int64_t K) {
  if (M <= 0 || N <= 0 || K <= 0 || M > INT32_MAX || N > INT32_MAX || K > INT32_MAX) return 0;
  return gemm_oz_ws_bytes((int)M, (int)N, (int)K);
}

extern "C" int asolve_gemm_oz(double* C, int64_t ldc, const double* A, int64_t lda, const double* B, int64_t ldb,
                              int64_t M, int64_t N, int64_t K, int transb, void* ws, size_t ws_bytes, int* err,
                              void* stream) {
  if (!C || !A || !B || M < 0 || N < 0 || K < 0) return ASOLVE_E_INVALID;
  if (ldc < (M > 0 ? M : 1) || lda < (M > 0 ? M : 1) || ldb < (transb ? (N > 0 ? N : 1) : (K > 0 ? K : 1)))
    return ASOLVE_E_INVALID;
  if (M > INT32_MAX || N > INT32_MAX || K > INT32_MAX || ldc > INT32_MAX || lda > INT32_MAX || ldb > INT32_MAX)
    return ASOLVE_E_UNSUPPORTED;
  if (M == 0 || N == 0 || K == 0) return ASOLVE_OK;
  if (!ws || ((uintptr_t)ws & 255) || ws_bytes < gemm_oz_ws_bytes((int)M, (int)N, (int)K)) return ASOLVE_E_INVALID;
  cudaError_t e = gemm_oz(C, (int)ldc, A, (int)lda, B, (int)ldb, (int)M, (int)N, (int)K, transb != 0, false, ws, err,
                          (cudaStream_t)stream);
  return e == cudaSuccess ? ASOLVE_OK : ASOLVE_E_CUDA;
}

extern "C" int asolve_set_panel_widths(asolve_ctx* c, int kind, const int32_t* nb, int count) {
  if (!c || kind < 0 || kind > 3 || count < 0 || count > 32 || (count > 0 && !nb)) return ASOLVE_E_INVALID;
  for (int i = 0; i < count; ++i)
    if (!(nb[i] == 0 || nb[i] == 4 || nb[i] == 8 || nb[i] == 16 || nb[i] == 32)) return ASOLVE_E_INVALID;
  for (int i = 0; i < 32; ++i) c->nb_tab[kind][i] = (int8_t)(i < count ? nb[i] : 0);
  return ASOLVE_OK;
}

extern "C" int asolve_set_profiling(asolve_ctx* c, int on) {
  if (!c) return ASOLVE_E_INVALID;
  c->profiling = on != 0;
  return ASOLVE_OK;
}

extern "C" int asolve_reset_profile(asolve_ctx* c) {
  if (!c) return ASOLVE_E_INVALID;
  for (int k = 0; k < K_COUNT; ++k) {
    c->prof_ms[k] = 0.0;
    c->prof_launches[k] = 0;
  }
  return ASOLVE_OK;
}

extern "C" int asolve_get_profile(asolve_ctx* c, asolve_profile* out) {
  if (!c || !out) return ASOLVE_E_INVALID;
  memset(out, 0, sizeof(*out));
  out->count = K_COUNT;
  for (int k = 0; k < K_COUNT; ++k) {
    strncpy(out->k[k].name, kKernelNames[k], sizeof(out->k[k].name) - 1);
    out->k[k].launches = c->prof_launches[k];
    out->k[k].total_ms = c->prof_ms[k];
  }
  return ASOLVE_OK;
}
