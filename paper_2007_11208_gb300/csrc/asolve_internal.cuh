// asolve_internal.cuh -- definitions shared by the library's translation units.
//
// Everything here belongs to the GPU library (libasolve.so); none of it is
// shared with the CPU oracle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

#include "asolve.h"

namespace asv {

// Kernel attributes such as a raised dynamic shared memory limit belong to
// one device.  PerDeviceOnce runs a setup step once per device, from any
// host thread: the first caller on a device runs it under a mutex, later
// callers only read the device's flag.  A failed setup is tried again by
// the next call; devices beyond the table run it on every call.
struct PerDeviceOnce {
  static constexpr int kMaxDevices = 64;
  std::atomic<int> done[kMaxDevices];
  std::mutex mu;
  template <class F>
  cudaError_t run(F&& setup) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return setup();
    if (done[dev].load(std::memory_order_acquire)) return cudaSuccess;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev].load(std::memory_order_relaxed)) return cudaSuccess;
    e = setup();
    if (e == cudaSuccess) done[dev].store(1, std::memory_order_release);
    return e;
  }
};

// Raise one kernel's dynamic shared memory limit on the current device
// (once per device and call site).
#define ASV_SMEM_LIMIT_ONCE(kernel, bytes)                                                      \
  ([&]() -> cudaError_t {                                                                      \
    static ::asv::PerDeviceOnce once_;                                                         \
    return once_.run([&]() {                                                                   \
      return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(bytes)); \
    });                                                                                        \
  }())

constexpr int kWarp = 32;
constexpr int kBatchNMax = 1024;   // largest n handled by the per-CTA batched path
constexpr int kBatchRhsMax = 8;    // largest nrhs handled by the per-CTA batched path
constexpr int kCtaThreads = 256;   // threads of the per-system (class) kernels
constexpr double kEps = 2.220446049250313080847e-16;  // 2^-52, machine epsilon
constexpr int kGemmBf16 = ASOLVE_GEMM_BF16;  // operand modes of launch_gemm_tc
constexpr int kGemmFp16 = ASOLVE_GEMM_FP16;
constexpr int kGemmFp8 = ASOLVE_GEMM_FP8;
// kappa limits of refinement with 16-bit trailing updates (unit roundoff
// 2^-8 for BF16, 2^-11 for FP16, times a margin for the growth of |L||U|)
constexpr double kKappaLimitBf16 = 1e3;
constexpr double kKappaLimitFp16 = 1e4;
// kappa limits of GMRES-IR with the same factors as preconditioner (the
// large path's 16-bit modes): GMRES on inv(LU) A absorbs the factors' error
// far beyond the classical refinement's limit
constexpr double kKappaLimitGmresBf16 = 1e7;
constexpr double kKappaLimitGmresFp16 = 1e8;
// FP8 E4M3 trailing updates (unit roundoff 2^-4): classical refinement only
// for the best-conditioned systems; GMRES-IR to kappa 1e3
constexpr double kKappaLimitFp8 = 1e1;
constexpr double kKappaLimitGmresFp8 = 1e3;

// Scan flags (Sec. 2.1, 2.2, Fig. 4).
enum : int32_t {
  SF_NONFINITE = 1 << 0,   // Inf/NaN in A
  SF_SYMPD = 1 << 1,       // likely_sympd (Fig. 4)
  SF_LOWER = 1 << 2,       // all elements above the diagonal are zero
  SF_UPPER = 1 << 3,       // all elements below the diagonal are zero
  SF_BANDED = 1 << 4,      // band positions <= band_frac * n^2
  SF_NORM_FP64 = 1 << 5,   // norms had to be summed in FP64 (FP32 range exceeded)
  SF_B_NONFINITE = 1 << 6, // Inf/NaN in B
};

struct ScanRes {           // 32 bytes, one per system
  int32_t kl, ku;
  int32_t flags;
  int32_t cls;
  double norm1, norminf;
};

// Work lists of the class-routed batched pipeline.
enum : int { L_BAND = 0, L_TRI = 1, L_CHOL = 2, L_LU = 3, L_SVD = 4, L_COUNT = 5 };

// Device-resident description of one batched call.  The host writes it into
// pinned memory; the captured graph copies it to the device first.
struct BatchDesc {
  int64_t count;
  const int64_t* n;        // [count]
  const int64_t* nrhs;     // [count]
  const int64_t* a_off;    // [count]
  const int64_t* b_off;    // [count]
  const double* A;
  const double* B;
  double* X;
  // optional per-system base pointers [count]; when set they replace
  // A + a_off[s], B + b_off[s] and X + b_off[s]
  const double* const* Ap;
  const double* const* Bp;
  double* const* Xp;
  asolve_info* info;       // [count]
  uint32_t flags;
  int32_t precision;
  double rcond_threshold, sympd_tol, band_frac, svd_trunc_rel;
  int32_t ir_max_iter;
  int32_t pad0;
  double ir_target_berr, ir_kappa_limit;
  // pipeline state (context-owned device memory)
  ScanRes* scan;           // [capacity]
  int32_t* lists;          // [L_COUNT][capacity]
  int32_t* list_len;       // [L_COUNT] (zeroed per call)
  int32_t* work_ctr;       // [16]      (zeroed per call)
  int64_t capacity;
  // per-CTA scratch slots of the class kernels
  char* slot_base;
  int64_t slot_bytes;
  int32_t slot_count;
  int32_t pad1;
  int32_t* err_flag;       // device-side error (e.g. a scratch slot too small)
  // panel widths of the dense class kernels chosen by the autotuner:
  // [LU FP32, Cholesky FP32, LU FP64, Cholesky FP64][(n - 1) / 32];
  // 0 keeps the built-in rule
  int8_t nb_tab[4][32];
};

// A dense route's factorisation kept for later solves with the same A
// (request server, ASOLVE_RESIDENT).  Filled by large_solve after a dense
// route succeeded; a later call with the same key solves with the kept
// factor (which stays in the workspace it was computed in).
struct LargeReuse {
  int valid;
  const double* A;       // key: the caller's A, its order and routing flags
  int64_t n;
  uint32_t flags;
  int cls, route, precision, lu, detail;
  int64_t kl, ku;
  double rcond, norm1, norminf;
};

// One large dense system (large.cu).
struct LargeArgs {
  const double* A;
  const double* B;
  double* X;
  int64_t n, nrhs;
  uint32_t flags;
  int precision;
  double rcond_threshold, sympd_tol, band_frac, ir_target_berr, ir_kappa_limit;
  int ir_max_iter;
  int num_sms;
  cudaStream_t st;
  LargeReuse* reuse;       // optional
  double svd_trunc_rel;    // SVD fallback cut-off: sigma <= svd_trunc_rel * sigma_max dropped (0: n eps)
};
// The SVD fallback for one large system (svd_large.cu), up to this order.
constexpr int64_t kSvdLargeMax = 8192;
size_t large_svd_ws_bytes(int64_t n, int64_t nrhs);
int large_svd(const double* A, int64_t n, const double* B, double* X, int64_t nrhs, double trunc_rel,
              double* G, void* ws, int64_t* rank, int* sweeps, cudaStream_t st);
size_t large_ws_bytes(int64_t n, int64_t nrhs);
int large_solve(const LargeArgs& a, void* ws, size_t ws_bytes, asolve_info* info);
// FP64 C (M x N) -= A (M x K) op(B) by the Ozaki splitting on the BF16
// tensor cores (gemm_oz.cu); ws: gemm_oz_ws_bytes(M, N, K) bytes.
size_t gemm_oz_ws_bytes(int M, int N, int K);
cudaError_t gemm_oz(double* C, int ldc, const double* A, int lda, const double* B, int ldb, int M, int N, int K,
                    bool tb, bool lower, void* ws, int* err, cudaStream_t st);

// One system for the banded route (band_large.cu): band storage input
// (AB, ldab, declared kld/kud) or a dense matrix A with its scan results.
struct BandArgs {
  const double* AB;
  int64_t ldab;
  int64_t kld, kud;
  const double* A;
  const double* B;
  double* X;
  int64_t n, nrhs;
  uint32_t flags;
  double rcond_threshold;
  int64_t kl, ku;          // dense input: the scan's bandwidths and norms
  double norm1, norminf;
  cudaStream_t st;
};
size_t band_ws_bytes(int64_t n, int64_t kl, int64_t ku, int64_t nrhs);
bool band_window_fits(int64_t kl, int64_t ku);
int band_solve(const BandArgs& a, void* ws, size_t ws_bytes, asolve_info* info);
int band_to_dense(const double* AB, int64_t ldab, int64_t kld, int64_t kud, int64_t n, double* A, cudaStream_t st);

// Column-major A, B and X of system s of a batch.
__device__ __forceinline__ const double* sys_A(const BatchDesc& d, int64_t s) {
  return d.Ap ? d.Ap[s] : d.A + d.a_off[s];
}
__device__ __forceinline__ const double* sys_B(const BatchDesc& d, int64_t s) {
  return d.Bp ? d.Bp[s] : d.B + d.b_off[s];
}
__device__ __forceinline__ double* sys_X(const BatchDesc& d, int64_t s) {
  return d.Xp ? d.Xp[s] : d.X + d.b_off[s];
}

// --------------------------------------------------------------------------
// Small device helpers.
__device__ __forceinline__ uint64_t dbits(double x) { return (uint64_t)__double_as_longlong(x); }
__device__ __forceinline__ bool is_nonzero_bits(uint64_t b) { return (b << 1) != 0; }
__device__ __forceinline__ bool is_nonfinite_bits(uint64_t b) {
  return ((b >> 52) & 0x7ff) == 0x7ff;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// Largest value, ties (and the order of NaN-free equal values) resolved to
// the smallest index: the first-maximum rule of partial pivoting.
template <typename T>
__device__ __forceinline__ void warp_argmax_first(T& v, int& idx) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T w = __shfl_xor_sync(0xffffffffu, v, o);
    int j = __shfl_xor_sync(0xffffffffu, idx, o);
    if (w > v || (w == v && j < idx)) { v = w; idx = j; }
  }
}

// Pivot search of partial pivoting on a warp.  abs_key(v): the bit pattern
// of |v| plus one (non-negative doubles order as unsigned integers), 0 for
// NaN, which is never a pivot.  warp_first_max_key: the first lane holding
// the largest non-zero key (high words reduced first, then low words among
// the lanes that hold the largest high word), -1 if no lane has one; kmax
// gets the key.
__device__ __forceinline__ unsigned long long abs_key(double v) {
  const double a = fabs(v);
  return (a == a) ? (unsigned long long)__double_as_longlong(a) + 1ull : 0ull;
}
__device__ __forceinline__ int warp_first_max_key(unsigned long long key, unsigned long long& kmax) {
  const unsigned hi = (unsigned)(key >> 32), lo = (unsigned)key;
  const unsigned mhi = __reduce_max_sync(0xffffffffu, hi);
  const unsigned mlo = __reduce_max_sync(0xffffffffu, hi == mhi ? lo : 0u);
  kmax = ((unsigned long long)mhi << 32) | mlo;
  const unsigned ball = __ballot_sync(0xffffffffu, key != 0ull && hi == mhi && lo == mlo);
  return ball ? __ffs(ball) - 1 : -1;
}

__device__ __forceinline__ int64_t ldg_i64(const int64_t* p) { return __ldg(p); }

}  // namespace asv
