// serve.cu -- a request server with continuous batching on top of the
// adaptive solver (asolve_submit / asolve_poll / asolve_get_serve_stats).
//
// The paper solves one system per call.  A server takes a stream of such
// calls from many producers and keeps the GPU busy with them: requests wait
// in a FIFO queue and two lanes, each a host thread with its own CUDA
// stream, take work from it as soon as they are free:
//   * the batch lane takes every queued small request (n <= 1024,
//     nrhs <= 8) with the same solver flags, in arrival order, and solves
//     them as one class-routed batch (scan, device routing, one persistent
//     launch per class, replayed from a CUDA graph);
//   * the large lane takes the oldest larger request and runs the blocked
//     whole-GPU path.
// The lanes overlap on the device: small requests that arrive while a large
// system is being factored are solved meanwhile.  Admission is by HBM
// budget: a request is admitted only while the bytes it holds on the device
// (staging of host buffers, the workspace of a large system) fit the
// context's budget together with everything in flight; a large request that
// does not fit yet reserves its bytes so that small ones cannot starve it,
// and one that alone exceeds the budget is refused at submission with
// ASOLVE_E_NOMEM.  Each request's status, asolve_info and latency
// (submission to completion, host steady clock) are published for
// asolve_poll.
//
// The server owns a second asolve context (its streams and workspaces), so
// synchronous calls on the owner context may go on meanwhile.  Staging
// memory and large-system workspaces come from a stream-ordered memory pool
// private to the server.
#include <cuda_runtime.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "asolve_internal.cuh"

namespace asv {
const asolve_config* ctx_config(asolve_ctx* c);
int ctx_device(asolve_ctx* c);
int ctx_num_sms(asolve_ctx* c);
void** ctx_serve_slot(asolve_ctx* c);
void serve_shutdown(asolve_ctx* c);
}  // namespace asv

extern "C" int asolve_solve_batched_ptrs(asolve_ctx* c, int64_t count, const int64_t* n,
                                         const int64_t* nrhs, const double* const* A,
                                         const double* const* B, double* const* X, uint32_t flags,
                                         asolve_info* infos);

using namespace asv;

namespace {

using Clock = std::chrono::steady_clock;

constexpr int64_t kServeMaxBatch = 8192;  // systems per batched round
constexpr int64_t kLargeNMax = 32768;
constexpr int64_t kLargeRhsMax = 256;
constexpr size_t kMetaBytes = 5 * sizeof(int64_t) + sizeof(asolve_info);  // per small request
// flags that change how a system is solved (requests in one batch share them)
constexpr uint32_t kSolverFlags =
    ASOLVE_NO_APPROX | ASOLVE_FORCE_LU | ASOLVE_FORCE_SVD | ASOLVE_NO_RCOND | ASOLVE_BERR | ASOLVE_TRIDIAG | ASOLVE_SYM_INDEF;

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

struct Request {
  uint64_t ticket;
  const double* A;
  const double* B;
  double* X;
  int64_t n, nrhs;
  uint32_t flags;
  bool large;
  size_t charge;  // bytes held against the budget while the request runs
  Clock::time_point t_submit;
};

struct Done {
  int status;
  asolve_info info;
  double latency_ms;
};

bool host_mode(const Request& r) { return (r.flags & ASOLVE_HOST_BUFFERS) != 0; }

size_t staging_bytes(int64_t n, int64_t nrhs) {
  return round256(sizeof(double) * (size_t)(n * n)) + 2 * round256(sizeof(double) * (size_t)(n * nrhs));
}

struct Server {
  asolve_ctx* owner = nullptr;
  asolve_ctx* w = nullptr;  // worker context (own stream)
  cudaStream_t st = nullptr;
  cudaMemPool_t pool = nullptr;
  int device = 0;
  int num_sms = 0;
  asolve_config cfg;
  size_t budget = 0;

  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request> queue;
  std::unordered_set<uint64_t> pending;  // queued or running
  std::unordered_map<uint64_t, Done> done;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread th_small, th_large;
  // one kept large request (ASOLVE_RESIDENT): its device block holds the
  // workspace with the factorisation and, for host buffers, the staged A
  void* kept_blk = nullptr;
  size_t kept_bytes = 0, kept_ws = 0;
  const double* kept_key = nullptr;  // the caller's A pointer
  int64_t kept_n = 0, kept_nrhs = 0;
  bool kept_host = false;
  LargeReuse kept{};
  bool evict_pending = false;
  void evict_kept();  // large-lane thread only
  cudaStream_t stl = nullptr;  // stream of the large lane
  size_t reserved = 0;         // held for a large request waiting for budget
  int active = 0;              // lanes busy on the device
  Clock::time_point busy_since;

  // statistics (under mu)
  asolve_serve_stats stats = {};
  bool any_submit = false;
  Clock::time_point t_first, t_last_done;

  // host staging of the per-request metadata (server thread only)
  char* h_meta = nullptr;
  size_t h_meta_bytes = 0;

  void lane_small();
  void lane_large();
  bool pick_small(std::vector<Request>& batch);
  bool pick_large(Request& r);
  bool any_queued(bool large) const;
  void begin_busy();
  void end_busy();
  void solve_small(std::vector<Request>& batch);
  void solve_large(Request& r);
  void complete(const Request& r, int status, const asolve_info* info);
  void fail_all(std::vector<Request>& rs, int status);
};

int cuda_code(cudaError_t e) { return e == cudaErrorMemoryAllocation ? ASOLVE_E_NOMEM : ASOLVE_E_CUDA; }

void blank_info(asolve_info* i, int status) {
  memset(i, 0, sizeof(*i));
  i->status = status;
  i->rcond = NAN;
  i->berr = NAN;
  i->svd_rank = -1;
}

void Server::complete(const Request& r, int status, const asolve_info* info) {
  const Clock::time_point t = Clock::now();
  Done d;
  d.status = status;
  if (info) d.info = *info;
  else blank_info(&d.info, status);
  d.info.status = status;
  d.latency_ms = std::chrono::duration<double, std::milli>(t - r.t_submit).count();
  std::lock_guard<std::mutex> lk(mu);
  pending.erase(r.ticket);
  done[r.ticket] = d;
  stats.completed += 1;
  if (status < 0) stats.failed += 1;
  stats.charged_bytes -= r.charge;
  t_last_done = t;
  cv_done.notify_all();
  cv_work.notify_all();  // budget freed
}

void Server::fail_all(std::vector<Request>& rs, int status) {
  for (const Request& r : rs) complete(r, status, nullptr);
}

// One batched round: all admitted small requests with identical solver flags.
void Server::solve_small(std::vector<Request>& b) {
  const int64_t m = (int64_t)b.size();
  // device block: [n | nrhs | Ap | Bp | Xp | infos | staging...]
  size_t meta = round256(kMetaBytes * (size_t)m);
  size_t total = meta;
  for (const Request& r : b)
    if (host_mode(r)) total += staging_bytes(r.n, r.nrhs);
  void* dblk = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync(&dblk, total, pool, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail_all(b, cuda_code(e));
    return;
  }
  if (meta > h_meta_bytes) {
    if (h_meta) cudaFreeHost(h_meta);
    h_meta = nullptr;
    h_meta_bytes = 0;
    size_t want = meta * 2;
    if (cudaMallocHost(&h_meta, want) != cudaSuccess) {
      h_meta = nullptr;
      cudaGetLastError();
      cudaFreeAsync(dblk, st);
      cudaStreamSynchronize(st);
      fail_all(b, ASOLVE_E_NOMEM);
      return;
    }
    h_meta_bytes = want;
  }
  // the previous round's copies out of h_meta have completed (the stream
  // was synchronised at the end of that round)
  int64_t* hn = reinterpret_cast<int64_t*>(h_meta);
  int64_t* hr = hn + m;
  const double** hA = reinterpret_cast<const double**>(hr + m);
  const double** hB = reinterpret_cast<const double**>(hr + 2 * m);
  double** hX = reinterpret_cast<double**>(hr + 3 * m);
  char* d0 = static_cast<char*>(dblk);
  asolve_info* dinf = reinterpret_cast<asolve_info*>(d0 + 5 * sizeof(int64_t) * (size_t)m);
  char* stage = d0 + meta;
  bool ok = true;
  for (int64_t k = 0; k < m; ++k) {
    const Request& r = b[k];
    hn[k] = r.n;
    hr[k] = r.nrhs;
    if (host_mode(r)) {
      const size_t ba = sizeof(double) * (size_t)(r.n * r.n), bb = sizeof(double) * (size_t)(r.n * r.nrhs);
      double* sA = reinterpret_cast<double*>(stage);
      double* sB = reinterpret_cast<double*>(stage + round256(ba));
      double* sX = reinterpret_cast<double*>(stage + round256(ba) + round256(bb));
      stage += staging_bytes(r.n, r.nrhs);
      ok = ok && cudaMemcpyAsync(sA, r.A, ba, cudaMemcpyHostToDevice, st) == cudaSuccess;
      ok = ok && cudaMemcpyAsync(sB, r.B, bb, cudaMemcpyHostToDevice, st) == cudaSuccess;
      hA[k] = sA;
      hB[k] = sB;
      hX[k] = sX;
    } else {
      hA[k] = r.A;
      hB[k] = r.B;
      hX[k] = r.X;
    }
  }
  ok = ok && cudaMemcpyAsync(d0, h_meta, 5 * sizeof(int64_t) * (size_t)m, cudaMemcpyHostToDevice, st) ==
                 cudaSuccess;
  int rc = ASOLVE_E_CUDA;
  if (ok) {
    const int64_t* dn = reinterpret_cast<const int64_t*>(d0);
    rc = asolve_solve_batched_ptrs(w, m, dn, dn + m, reinterpret_cast<const double* const*>(dn + 2 * m),
                                   reinterpret_cast<const double* const*>(dn + 3 * m),
                                   reinterpret_cast<double* const*>(dn + 4 * m), b[0].flags & kSolverFlags,
                                   dinf);
  }
  std::vector<asolve_info> infos((size_t)m);
  if (rc == ASOLVE_OK) {
    // results back: X of host-mode requests, then every info record
    for (int64_t k = 0; k < m && ok; ++k)
      if (host_mode(b[k]))
        ok = cudaMemcpyAsync(b[k].X, hX[k], sizeof(double) * (size_t)(b[k].n * b[k].nrhs),
                             cudaMemcpyDeviceToHost, st) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(infos.data(), dinf, sizeof(asolve_info) * (size_t)m, cudaMemcpyDeviceToHost,
                               st) == cudaSuccess;
  }
  cudaFreeAsync(dblk, st);
  const bool synced = cudaStreamSynchronize(st) == cudaSuccess;
  if (rc == ASOLVE_OK && (!ok || !synced)) rc = ASOLVE_E_CUDA;
  if (rc != ASOLVE_OK) {
    cudaGetLastError();
    fail_all(b, rc);
    return;
  }
  {
    std::lock_guard<std::mutex> lk(mu);
    stats.batches += 1;
  }
  for (int64_t k = 0; k < m; ++k) complete(b[k], infos[k].status, &infos[k]);
}

// One large system on the blocked whole-GPU path.
void Server::evict_kept() {
  if (!kept_blk) return;
  cudaFreeAsync(kept_blk, stl);
  cudaStreamSynchronize(stl);
  kept_blk = nullptr;
  kept.valid = 0;
  std::lock_guard<std::mutex> lk(mu);
  stats.charged_bytes -= kept_bytes;
  kept_bytes = 0;
  cv_work.notify_all();
}

// One large system on the blocked whole-GPU path.  With ASOLVE_RESIDENT the
// request's device block is kept afterwards, and a later resident request
// with the same A (same pointer, unchanged contents) solves with the kept
// factorisation (and, for host buffers, the A already staged).
void Server::solve_large(Request& r) {
  const bool hm = host_mode(r);
  const bool resident = (r.flags & ASOLVE_RESIDENT) != 0;
  const bool hit = resident && kept_blk && kept.valid && kept_key == r.A && kept_n == r.n && kept_host == hm &&
                   r.nrhs <= kept_nrhs;
  if (resident && !hit) evict_kept();
  const size_t ws = hit ? kept_ws : round256(large_ws_bytes(r.n, r.nrhs));
  const size_t total = ws + (hm ? staging_bytes(r.n, hit ? kept_nrhs : r.nrhs) : 0);
  void* dblk = hit ? kept_blk : nullptr;
  if (!hit) {
    cudaError_t e = cudaMallocFromPoolAsync(&dblk, total, pool, stl);
    if (e != cudaSuccess) {
      cudaGetLastError();
      complete(r, cuda_code(e), nullptr);
      return;
    }
  }
  const double* A = r.A;
  const double* B = r.B;
  double* X = r.X;
  bool ok = true;
  if (hm) {
    char* stage = static_cast<char*>(dblk) + ws;
    const size_t ba = sizeof(double) * (size_t)(r.n * r.n), bb = sizeof(double) * (size_t)(r.n * r.nrhs);
    const size_t bcap = sizeof(double) * (size_t)(r.n * (hit ? kept_nrhs : r.nrhs));
    double* sA = reinterpret_cast<double*>(stage);
    double* sB = reinterpret_cast<double*>(stage + round256(ba));
    double* sX = reinterpret_cast<double*>(stage + round256(ba) + round256(bcap));
    if (!hit) ok = cudaMemcpyAsync(sA, r.A, ba, cudaMemcpyHostToDevice, stl) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(sB, r.B, bb, cudaMemcpyHostToDevice, stl) == cudaSuccess;
    A = sA;
    B = sB;
    X = sX;
  }
  asolve_info info;
  blank_info(&info, ASOLVE_E_CUDA);
  int rc = ASOLVE_E_CUDA;
  if (ok) {
    LargeArgs la{A, B, X, r.n, r.nrhs, r.flags & kSolverFlags, cfg.precision, cfg.rcond_threshold,
                 cfg.sympd_tol, cfg.band_frac, cfg.ir_target_berr, cfg.ir_kappa_limit, cfg.ir_max_iter,
                 num_sms, stl, resident ? &kept : nullptr, cfg.svd_trunc_rel};
    rc = large_solve(la, dblk, ws, &info);
    if (rc < 0 && rc != info.status) info.status = rc;
    if (hm && info.status >= 0)
      ok = cudaMemcpyAsync(r.X, X, sizeof(double) * (size_t)(r.n * r.nrhs), cudaMemcpyDeviceToHost, stl) ==
           cudaSuccess;
  }
  const bool keep = resident && ok && info.status >= 0 && kept.valid;
  if (!keep) {
    if (hit) {
      kept_blk = nullptr;  // the kept block goes with this request
      kept.valid = 0;
      std::lock_guard<std::mutex> lk(mu);
      stats.charged_bytes -= kept_bytes;
      kept_bytes = 0;
    }
    cudaFreeAsync(dblk, stl);
  }
  const bool synced = cudaStreamSynchronize(stl) == cudaSuccess;
  if (keep && !hit) {
    kept_blk = dblk;
    kept_bytes = total;
    kept_ws = ws;
    kept_key = r.A;
    kept_n = r.n;
    kept_nrhs = r.nrhs;
    kept_host = hm;
    std::lock_guard<std::mutex> lk(mu);
    stats.charged_bytes += kept_bytes;
    if (stats.charged_bytes > stats.peak_charged_bytes) stats.peak_charged_bytes = stats.charged_bytes;
  }
  if (!ok || !synced) {
    cudaGetLastError();
    complete(r, ASOLVE_E_CUDA, nullptr);
    return;
  }
  {
    std::lock_guard<std::mutex> lk(mu);
    stats.large_solves += 1;
  }
  complete(r, info.status, &info);
}

// Admission (mu held).  Small requests with the solver flags of the oldest
// one, in arrival order, while the budget allows (minus what a waiting large
// request has reserved).
bool Server::pick_small(std::vector<Request>& batch) {
  size_t used = 0;
  uint32_t f0 = 0;
  bool have = false;
  for (auto it = queue.begin(); it != queue.end();) {
    if (it->large) {
      ++it;
      continue;
    }
    const uint32_t f = it->flags & kSolverFlags;
    if (have && f != f0) {
      ++it;
      continue;
    }
    if (stats.charged_bytes + reserved + used + it->charge > budget) break;
    if ((int64_t)batch.size() >= kServeMaxBatch) break;
    f0 = f;
    have = true;
    used += it->charge;
    batch.push_back(*it);
    it = queue.erase(it);
  }
  if (batch.empty()) return false;
  stats.charged_bytes += used;
  if (stats.charged_bytes > stats.peak_charged_bytes) stats.peak_charged_bytes = stats.charged_bytes;
  stats.queued = (int64_t)queue.size();
  return true;
}

// The oldest large request, if it fits; otherwise its bytes are reserved.
bool Server::pick_large(Request& r) {
  for (auto it = queue.begin(); it != queue.end(); ++it) {
    if (!it->large) continue;
    if (stats.charged_bytes + it->charge > budget) {
      if (kept_blk && (stats.charged_bytes - kept_bytes) + it->charge <= budget) {
        // the kept factorisation gives way (freed by the caller, outside the lock)
        evict_pending = true;
        return false;
      }
      reserved = it->charge;
      return false;
    }
    reserved = 0;
    r = *it;
    queue.erase(it);
    stats.charged_bytes += r.charge;
    if (stats.charged_bytes > stats.peak_charged_bytes) stats.peak_charged_bytes = stats.charged_bytes;
    stats.queued = (int64_t)queue.size();
    return true;
  }
  reserved = 0;
  return false;
}

bool Server::any_queued(bool large) const {
  for (const Request& q : queue)
    if (q.large == large) return true;
  return false;
}

void Server::begin_busy() {
  if (active++ == 0) busy_since = Clock::now();
}
void Server::end_busy() {
  if (--active == 0) stats.busy_ms += std::chrono::duration<double, std::milli>(Clock::now() - busy_since).count();
  stats.rounds += 1;
}

void Server::lane_small() {
  cudaSetDevice(device);
  for (;;) {
    std::vector<Request> batch;
    {
      std::unique_lock<std::mutex> lk(mu);
      for (;;) {
        if (pick_small(batch)) break;
        if (stop && !any_queued(false)) return;
        cv_work.wait(lk);
      }
      begin_busy();
    }
    solve_small(batch);
    std::lock_guard<std::mutex> lk(mu);
    end_busy();
    cv_work.notify_all();
  }
}

void Server::lane_large() {
  cudaSetDevice(device);
  for (;;) {
    Request r{};
    {
      std::unique_lock<std::mutex> lk(mu);
      for (;;) {
        if (pick_large(r)) break;
        if (evict_pending) {
          evict_pending = false;
          lk.unlock();
          evict_kept();
          lk.lock();
          continue;
        }
        if (stop && !any_queued(true)) return;
        cv_work.wait(lk);
      }
      begin_busy();
    }
    solve_large(r);
    std::lock_guard<std::mutex> lk(mu);
    end_busy();
    cv_work.notify_all();
  }
}

Server* server_of(asolve_ctx* c) { return static_cast<Server*>(*ctx_serve_slot(c)); }

// Guards the creation of servers (first submissions may race).
std::mutex g_create_mu;

// Create the server of context c on first use.
int ensure_server(asolve_ctx* c, Server** out) {
  std::lock_guard<std::mutex> create_lk(g_create_mu);
  Server* s = server_of(c);
  if (s) {
    *out = s;
    return ASOLVE_OK;
  }
  s = new (std::nothrow) Server();
  if (!s) return ASOLVE_E_NOMEM;
  s->owner = c;
  s->cfg = *ctx_config(c);
  s->device = ctx_device(c);
  s->num_sms = ctx_num_sms(c);
  s->budget = s->cfg.hbm_budget;
  s->stats.budget = s->budget;
  asolve_config wc = s->cfg;
  wc.stream = nullptr;
  wc.device = s->device;
  int rc = asolve_create(&s->w, &wc);
  if (rc != ASOLVE_OK) {
    delete s;
    return rc;
  }
  s->st = (cudaStream_t)asolve_stream(s->w);
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = s->device;
  if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess) {
    cudaGetLastError();
    asolve_destroy(s->w);
    delete s;
    return ASOLVE_E_CUDA;
  }
  // keep freed blocks for the next rounds instead of returning them
  uint64_t keep = s->budget;
  cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  if (cudaStreamCreateWithFlags(&s->stl, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    cudaMemPoolDestroy(s->pool);
    asolve_destroy(s->w);
    delete s;
    return ASOLVE_E_CUDA;
  }
  s->th_small = std::thread([s] { s->lane_small(); });
  s->th_large = std::thread([s] { s->lane_large(); });
  *ctx_serve_slot(c) = s;
  *out = s;
  return ASOLVE_OK;
}

}  // namespace

namespace asv {
void serve_shutdown(asolve_ctx* c) {
  Server* s = server_of(c);
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->th_small.joinable()) s->th_small.join();
  if (s->th_large.joinable()) s->th_large.join();
  if (s->kept_blk) {
    cudaSetDevice(s->device);
    cudaFreeAsync(s->kept_blk, s->stl);
    s->kept_blk = nullptr;
  }
  cudaSetDevice(s->device);
  if (s->st) cudaStreamSynchronize(s->st);
  if (s->stl) {
    cudaStreamSynchronize(s->stl);
    cudaStreamDestroy(s->stl);
  }
  if (s->pool) cudaMemPoolDestroy(s->pool);
  if (s->h_meta) cudaFreeHost(s->h_meta);
  asolve_destroy(s->w);
  delete s;
  *ctx_serve_slot(c) = nullptr;
}
}  // namespace asv

extern "C" int asolve_submit(asolve_ctx* c, const double* A, const double* B, int64_t n, int64_t nrhs,
                             uint32_t flags, double* X, uint64_t* ticket) {
  if (!c || !ticket || n < 0 || nrhs < 1) return ASOLVE_E_INVALID;
  if (n > 0 && (!A || !B || !X)) return ASOLVE_E_INVALID;
  if (flags & ~(kSolverFlags | ASOLVE_HOST_BUFFERS | ASOLVE_SYNC | ASOLVE_RESIDENT)) return ASOLVE_E_INVALID;
  if (n > kLargeNMax || nrhs > kLargeRhsMax) return ASOLVE_E_UNSUPPORTED;
  Server* s = nullptr;
  int rc = ensure_server(c, &s);
  if (rc != ASOLVE_OK) return rc;
  Request r;
  r.A = A;
  r.B = B;
  r.X = X;
  r.n = n;
  r.nrhs = nrhs;
  r.flags = flags;
  r.large = n > kBatchNMax || nrhs > kBatchRhsMax;
  const bool hm = (flags & ASOLVE_HOST_BUFFERS) != 0;
  if (r.large) r.charge = round256(large_ws_bytes(n, nrhs)) + (hm ? staging_bytes(n, nrhs) : 0);
  else r.charge = kMetaBytes + (hm ? staging_bytes(n, nrhs) : 0);
  r.t_submit = Clock::now();
  std::unique_lock<std::mutex> lk(s->mu);
  if (!s->any_submit) {
    s->any_submit = true;
    s->t_first = r.t_submit;
  }
  if (r.charge > s->budget) {
    s->stats.rejected += 1;
    return ASOLVE_E_NOMEM;
  }
  r.ticket = s->next_ticket++;
  *ticket = r.ticket;
  s->stats.submitted += 1;
  if (n == 0) {  // nothing to solve: done at once
    Done d;
    d.status = ASOLVE_OK;
    blank_info(&d.info, ASOLVE_OK);
    d.latency_ms = 0.0;
    s->done[r.ticket] = d;
    s->stats.completed += 1;
    s->cv_done.notify_all();
    return ASOLVE_OK;
  }
  s->pending.insert(r.ticket);
  s->queue.push_back(r);
  s->stats.queued = (int64_t)s->queue.size();
  lk.unlock();
  s->cv_work.notify_all();  // both lanes wait on this condition
  return ASOLVE_OK;
}

extern "C" int asolve_poll(asolve_ctx* c, uint64_t ticket, int64_t wait_us, asolve_info* info,
                           double* latency_ms) {
  if (!c) return ASOLVE_E_INVALID;
  Server* s = server_of(c);
  if (!s) return ASOLVE_E_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  auto ready = [&] { return s->done.count(ticket) != 0 || s->pending.count(ticket) == 0; };
  if (wait_us < 0) s->cv_done.wait(lk, ready);
  else if (wait_us > 0) s->cv_done.wait_for(lk, std::chrono::microseconds(wait_us), ready);
  auto it = s->done.find(ticket);
  if (it == s->done.end()) return s->pending.count(ticket) ? ASOLVE_PENDING : ASOLVE_E_INVALID;
  const Done d = it->second;
  s->done.erase(it);
  if (info) *info = d.info;
  if (latency_ms) *latency_ms = d.latency_ms;
  return ASOLVE_OK;
}

extern "C" int asolve_get_serve_stats(asolve_ctx* c, asolve_serve_stats* out) {
  if (!c || !out) return ASOLVE_E_INVALID;
  memset(out, 0, sizeof(*out));
  Server* s = server_of(c);
  if (!s) {
    out->budget = ctx_config(c)->hbm_budget;
    return ASOLVE_OK;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  if (s->any_submit && s->stats.completed > 0)
    out->wall_ms = std::chrono::duration<double, std::milli>(s->t_last_done - s->t_first).count();
  return ASOLVE_OK;
}
