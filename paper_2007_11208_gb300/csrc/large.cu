// large.cu -- one large dense system (n > 1024), spread over the whole GPU.
//
// Routes (paper Sec. 2.2-2.4) for a single large system, orchestrated by the
// host with one launch (or a few) per block step:
//   Cholesky (Sec. 2.3)  blocked right-looking, 128-wide panels: diagonal
//                        block by one CTA, L21 = A21 inv(L11)^T, trailing
//                        SYRK on the lower triangle;
//   LU (Sec. 2.4)        blocked right-looking with partial pivoting: the
//                        128-wide panel is factored by a cooperative kernel
//                        (one grid barrier per column), its row swaps are
//                        applied to the other columns, U12 = inv(L11) A12,
//                        and the trailing update A22 -= L21 U12;
//   triangular (Sec. 2.2, Eq. 3) blocked forward/back substitution: one
//                        cooperative wavefront launch per solve.
// The working matrix is FP32 in the mixed-precision modes (trailing updates
// on the tcgen05 tensor cores: 3xTF32 split, or single BF16 / FP16
// products; the FP32 panel elects pivots with one atomic per CTA; solves
// multiply by the inverses of the 128 x 128 diagonal blocks) and FP64 in
// the plain mode (trailing updates on the FP64 mma.sync instruction; solves
// by substitution).  Refinement (FP64 residual split over k), the 1-norm
// condition estimate (est_host.cuh) and the per-column backward error are
// driven from the host.
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>
#include <string.h>

#include <vector>

#include "cta_linalg.cuh"
#include "est_host.cuh"

namespace asv {

cudaError_t launch_gemm_tc(float* C, int ldc, const float* A, int lda, const float* B, int ldb, int M, int N,
                           int K, int passes, int* err, cudaStream_t st, bool trans_b, bool lower);

constexpr int kLB = 128;  // panel / block width of the large path
constexpr int kGmresM = 30;         // GMRES-IR: Krylov basis size of one inner solve
constexpr double kGmresTol = 1e-4;  // inner solve: preconditioned residual reduced by this factor

// ------------------------------------------------------------ utilities
// Bounded grid-wide barrier for cooperatively launched kernels (all CTAs
// co-resident), on an arrival counter that only grows (zeroed before the
// launch): the k-th barrier of a launch completes when the counter reaches
// k * G.  One atomic per CTA and polling; no reset and no generation word.
__device__ bool grid_barrier_count(unsigned* bar, unsigned target, int* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    s_ok = 1;
    __threadfence();
    atomicAdd(bar, 1u);
    long long it = 0;
    while (*(volatile unsigned*)bar < target) {
      if (++it > 200000000ll) {
        s_ok = 0;
        atomicExch(err, 1);
        break;
      }
    }
    __threadfence();
  }
  __syncthreads();
  return s_ok != 0;
}

template <typename T>
__global__ void k_to_work(const double* __restrict__ A, int n, T* __restrict__ W, int ldw) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int c = blockIdx.x * 8 + w; c < n; c += gridDim.x * 8)
    for (int r = lane; r < n; r += 32) W[(size_t)c * ldw + r] = (T)A[(size_t)c * n + r];
}

// ------------------------------------------------- diagonal-block Cholesky
template <typename T>
__global__ void __launch_bounds__(kThreads) k_chol_diag(T* W, int ldw, int k0, int kb, int nb, int* fail) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int f = cta_chol_factor<T>(W + (size_t)k0 * ldw + k0, ldw, kb, reinterpret_cast<T*>(smem), nb);
  if (f && threadIdx.x == 0) *fail = k0 + f;
}

// ------------------------------------------------- panel TRSM by substitution
// With L11 the kb x kb lower block of W at (k0, k0) (unit diagonal if
// `unit`), solve L11 x = v in place for 64 vectors per CTA:
//   side 0: the columns c in [lo, hi) of W's rows k0..k0+kb-1 (U12 of LU);
//   side 1: the rows r in [lo, hi) of W's columns k0..k0+kb-1, i.e.
//           x L11^T = a (L21 of Cholesky).
// L11 and the 64 vectors sit in shared memory; four threads share each
// vector (the dot product of step i is split four ways and combined with
// two shuffles), so the 128 steps of forward substitution need no block
// barrier.
constexpr int kTrsmXP = kLB + 4;  // vector stride: 4 consecutive k of 8 vectors hit distinct banks
constexpr int kTrsmBlockedRhs = 32;  // triangular route: blocked TRSM from this many right-hand sides

template <typename T>
__global__ void __launch_bounds__(kThreads) k_trsm_sub(T* __restrict__ W, int ldw, int k0, int kb, int lo, int hi,
                                                      int side, int unit) {
  extern __shared__ __align__(16) unsigned char smem[];
  T(*Ms)[kLB + 1] = reinterpret_cast<T(*)[kLB + 1]>(smem);  // Ms[i][k] = L11(i, k)
  T* X = reinterpret_cast<T*>(smem + sizeof(T) * kLB * (kLB + 1));
  T* rinv = X + 64 * kTrsmXP;
  const int base = lo + blockIdx.x * 64;
  if (base >= hi) return;
  const int cnt = min(64, hi - base);
  const int tid = threadIdx.x;
  for (int e = tid; e < kLB * kLB; e += kThreads) {
    const int i = e & (kLB - 1), k = e >> 7;
    Ms[i][k] = (i < kb && k <= i) ? W[(size_t)(k0 + k) * ldw + k0 + i] : T(0);
  }
  if (side == 0) {
    for (int e = tid; e < kLB * 64; e += kThreads) {
      const int k = e & (kLB - 1), q = e >> 7;
      X[q * kTrsmXP + k] = (k < kb && q < cnt) ? W[(size_t)(base + q) * ldw + k0 + k] : T(0);
    }
  } else {
    for (int e = tid; e < kLB * 64; e += kThreads) {
      const int q = e & 63, k = e >> 6;
      X[q * kTrsmXP + k] = (k < kb && q < cnt) ? W[(size_t)(k0 + k) * ldw + base + q] : T(0);
    }
  }
  __syncthreads();
  for (int i = tid; i < kLB; i += kThreads) rinv[i] = (unit || i >= kb) ? T(1) : T(1) / Ms[i][i];
  __syncthreads();
  const int q = tid >> 2, t = tid & 3;
  T* xq = X + q * kTrsmXP;
  for (int i = 0; i < kb; ++i) {
    T part = T(0);
    for (int k = t; k < i; k += 4) part += Ms[i][k] * xq[k];
    part += __shfl_xor_sync(0xffffffffu, part, 1);
    part += __shfl_xor_sync(0xffffffffu, part, 2);
    const T xi = (xq[i] - part) * rinv[i];
    __syncwarp();
    if (t == 0) xq[i] = xi;
    __syncwarp();
  }
  __syncthreads();
  if (side == 0) {
    for (int e = tid; e < kLB * 64; e += kThreads) {
      const int k = e & (kLB - 1), qq = e >> 7;
      if (k < kb && qq < cnt) W[(size_t)(base + qq) * ldw + k0 + k] = X[qq * kTrsmXP + k];
    }
  } else {
    for (int e = tid; e < kLB * 64; e += kThreads) {
      const int qq = e & 63, k = e >> 6;
      if (k < kb && qq < cnt) W[(size_t)(k0 + k) * ldw + base + qq] = X[qq * kTrsmXP + k];
    }
  }
}

template <typename T>
constexpr size_t trsm_smem() {
  return sizeof(T) * ((size_t)kLB * (kLB + 1) + 64 * kTrsmXP + kLB);
}

// Diagonal-block step of the blocked TRSM with many right-hand sides:
// X(k0.., c) <- inv(T11) X(k0.., c) for the kb x kb block T11 of the
// triangle M (lower: rows and columns k0..k0+kb-1 on and below the
// diagonal, forward substitution; upper: on and above, backward), one CTA
// per 64 right-hand sides, four threads per right-hand side.
__global__ void __launch_bounds__(kThreads) k_trsm_rhs(const double* __restrict__ M, int ldm, int k0, int kb,
                                                      double* __restrict__ X, int ldx, int nrhs, int upper) {
  extern __shared__ __align__(16) unsigned char smem[];
  double(*Ms)[kLB + 1] = reinterpret_cast<double(*)[kLB + 1]>(smem);  // Ms[i][k] = T11(i, k)
  double* Xs = reinterpret_cast<double*>(smem + sizeof(double) * kLB * (kLB + 1));
  double* rinv = Xs + 64 * kTrsmXP;
  const int base = blockIdx.x * 64;
  if (base >= nrhs) return;
  const int cnt = min(64, nrhs - base);
  const int tid = threadIdx.x;
  for (int e = tid; e < kLB * kLB; e += kThreads) {
    const int i = e & (kLB - 1), k = e >> 7;
    const bool in = i < kb && k < kb && (upper ? k >= i : k <= i);
    Ms[i][k] = in ? M[(size_t)(k0 + k) * ldm + k0 + i] : 0.0;
  }
  for (int e = tid; e < kLB * 64; e += kThreads) {
    const int k = e & (kLB - 1), q = e >> 7;
    Xs[q * kTrsmXP + k] = (k < kb && q < cnt) ? X[(size_t)(base + q) * ldx + k0 + k] : 0.0;
  }
  __syncthreads();
  for (int i = tid; i < kLB; i += kThreads) rinv[i] = (i >= kb) ? 1.0 : 1.0 / Ms[i][i];
  __syncthreads();
  const int q = tid >> 2, t = tid & 3;
  double* xq = Xs + q * kTrsmXP;
  for (int ii = 0; ii < kb; ++ii) {
    const int i = upper ? kb - 1 - ii : ii;
    double part = 0.0;
    if (upper)
      for (int k = i + 1 + t; k < kb; k += 4) part += Ms[i][k] * xq[k];
    else
      for (int k = t; k < i; k += 4) part += Ms[i][k] * xq[k];
    part += __shfl_xor_sync(0xffffffffu, part, 1);
    part += __shfl_xor_sync(0xffffffffu, part, 2);
    const double xi = (xq[i] - part) * rinv[i];
    __syncwarp();
    if (t == 0) xq[i] = xi;
    __syncwarp();
  }
  __syncthreads();
  for (int e = tid; e < kLB * 64; e += kThreads) {
    const int k = e & (kLB - 1), qq = e >> 7;
    if (k < kb && qq < cnt) X[(size_t)(base + qq) * ldx + k0 + k] = Xs[qq * kTrsmXP + k];
  }
}

// ------------------------------------------------- LU panel (cooperative)
// Panel columns k0..k0+kb-1, rows k0..n-1.  CTA b keeps rows
// [b*R, (b+1)*R) of the panel (relative to k0) in shared memory for the
// whole panel.  Per column: every CTA publishes its best candidate (value,
// row, and the whole panel row) and the owner of the diagonal row publishes
// that row; after one grid barrier every CTA picks the same pivot (largest
// |value|, first row on ties), swaps locally and updates its own rows.
// Buffers are double-buffered by column parity.  This is the FP64 panel of
// more than 2^16 rows; the others (k_lu_panel_at, below) elect the pivot
// with an atomic.
struct PanelBuf {
  void* cand;      // [2][G][4] of T: |v|, row, v, valid
  void* rows;      // [2][G][kLB] of T
  void* diag;      // [2][kLB] of T
  unsigned* bar;   // grid barrier (zeroed before the launch)
  int* err;
  unsigned long long* key;  // [3] k_lu_panel_at: election keys (PivKey), by atomicMax
};

template <typename T>
__global__ void __launch_bounds__(kThreads) k_lu_panel(T* __restrict__ W, int ldw, int n, int k0, int kb, int R,
                                                      int* __restrict__ piv, PanelBuf pb, int* fail) {
  extern __shared__ __align__(16) unsigned char smem[];
  T* S = reinterpret_cast<T*>(smem);  // R x (kLB + 1)
  T* prow = S + (size_t)R * (kLB + 1);  // kLB
  __shared__ T s_best[kWarps];
  __shared__ int s_idx[kWarps];
  __shared__ T s_val[kWarps];
  __shared__ int s_idxw[kWarps];
  __shared__ int s_p, s_wb, s_stop;
  __shared__ T s_pv;
  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int m = n - k0;
  const int rlo = b * R, rhi = min(m, rlo + R);
  const int nr = max(0, rhi - rlo);
  for (int c = w; c < kb; c += kWarps)
    for (int i = lane; i < nr; i += 32) S[i * (kLB + 1) + c] = W[(size_t)(k0 + c) * ldw + k0 + rlo + i];
  __syncthreads();
  T* candT = reinterpret_cast<T*>(pb.cand);
  T* rowsT = reinterpret_cast<T*>(pb.rows);
  T* diagT = reinterpret_cast<T*>(pb.diag);
  for (int c = 0; c < kb; ++c) {
    const int buf = c & 1;
    // local candidate among own rows >= c
    T best = T(-1), bval = T(0);
    int bi = 0x7fffffff;
    for (int i = tid; i < nr; i += kThreads) {
      if (rlo + i < c) continue;
      const T v = S[i * (kLB + 1) + c];
      const T a = fabs(v);
      if (a > best) { best = a; bi = rlo + i; bval = v; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      const T ov = __shfl_xor_sync(0xffffffffu, bval, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; bval = ov; }
    }
    if (lane == 0) { s_best[w] = best; s_idx[w] = bi; s_val[w] = bval; }
    __syncthreads();
    if (tid == 0) {
      T bb = s_best[0], bv = s_val[0];
      int ii = s_idx[0];
      for (int k = 1; k < kWarps; ++k)
        if (s_best[k] > bb || (s_best[k] == bb && s_idx[k] < ii)) { bb = s_best[k]; ii = s_idx[k]; bv = s_val[k]; }
      T* cd = candT + ((size_t)buf * G + b) * 4;
      cd[0] = bb;
      cd[1] = (T)ii;
      cd[2] = bv;
      cd[3] = (ii != 0x7fffffff && bb >= T(0)) ? T(1) : T(0);
      s_p = ii;
    }
    __syncthreads();
    {  // publish the candidate row and, if owned, the diagonal row
      const int ii = s_p;
      if (ii != 0x7fffffff && ii >= rlo && ii < rhi)
        for (int k = tid; k < kb; k += kThreads)
          rowsT[((size_t)buf * G + b) * kLB + k] = S[(ii - rlo) * (kLB + 1) + k];
      if (c >= rlo && c < rhi)
        for (int k = tid; k < kb; k += kThreads) diagT[(size_t)buf * kLB + k] = S[(c - rlo) * (kLB + 1) + k];
    }
    __threadfence();
    if (!grid_barrier_count(pb.bar, (unsigned)(c + 1) * (unsigned)G, pb.err)) return;
    // every CTA finds the same winner: the candidates are read in parallel
    // (one per thread) and reduced (largest |v|, then smallest row)
    {
      T bb = T(-1), bv = T(0);
      int ii = 0x7fffffff, wb = 0x7fffffff;
      for (int k = tid; k < G; k += kThreads) {
        const volatile T* cd = candT + ((size_t)buf * G + k) * 4;
        if (cd[3] == T(0)) continue;
        const T kb_ = cd[0];
        const int ki = (int)cd[1];
        if (kb_ > bb || (kb_ == bb && ki < ii)) { bb = kb_; ii = ki; bv = cd[2]; wb = k; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T ob = __shfl_xor_sync(0xffffffffu, bb, o);
        const int oi = __shfl_xor_sync(0xffffffffu, ii, o);
        const T ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int ow = __shfl_xor_sync(0xffffffffu, wb, o);
        if (ob > bb || (ob == bb && oi < ii)) { bb = ob; ii = oi; bv = ov; wb = ow; }
      }
      __syncthreads();
      if (lane == 0) { s_best[w] = bb; s_idx[w] = ii; s_val[w] = bv; s_idxw[w] = wb; }
      __syncthreads();
      if (tid == 0) {
        bb = s_best[0]; ii = s_idx[0]; bv = s_val[0]; wb = s_idxw[0];
        for (int k = 1; k < kWarps; ++k)
          if (s_best[k] > bb || (s_best[k] == bb && s_idx[k] < ii)) {
            bb = s_best[k]; ii = s_idx[k]; bv = s_val[k]; wb = s_idxw[k];
          }
        s_p = ii;
        s_wb = wb;
        s_pv = bv;
        s_stop = (wb < 0 || wb >= G || ii < c || ii >= m || bv == T(0) || bv != bv) ? 1 : 0;
        if (s_stop && b == 0) *fail = k0 + c + 1;
        if (!s_stop && b == 0) piv[k0 + c] = k0 + ii;
      }
    }
    __syncthreads();
    if (s_stop) return;  // uniform across the grid: every CTA saw the same candidates
    const int p = s_p;
    for (int k = tid; k < kb; k += kThreads) prow[k] = ((volatile T*)rowsT)[((size_t)buf * G + s_wb) * kLB + k];
    __syncthreads();
    if (p != c) {
      if (p >= rlo && p < rhi)
        for (int k = tid; k < kb; k += kThreads) S[(p - rlo) * (kLB + 1) + k] = ((volatile T*)diagT)[(size_t)buf * kLB + k];
      if (c >= rlo && c < rhi)
        for (int k = tid; k < kb; k += kThreads) S[(c - rlo) * (kLB + 1) + k] = prow[k];
    }
    __syncthreads();
    const T inv = T(1) / s_pv;
    // multipliers of the rows below the pivot, then the rank-1 update spread
    // over (row, column) pairs so that every thread has independent work
    const int i0 = max(0, c + 1 - rlo);
    for (int i = i0 + tid; i < nr; i += kThreads) S[i * (kLB + 1) + c] *= inv;
    __syncthreads();
    // one warp per row, lanes over the columns
    for (int i = i0 + w; i < nr; i += kWarps) {
      T* row = S + i * (kLB + 1);
      const T l = row[c];
      for (int k = c + 1 + lane; k < kb; k += 32) row[k] -= l * prow[k];
    }
    __syncthreads();
  }
  for (int c = w; c < kb; c += kWarps)
    for (int i = lane; i < nr; i += 32) W[(size_t)(k0 + c) * ldw + k0 + rlo + i] = S[i * (kLB + 1) + c];
}

// Pivot election key of the atomic panel: the largest key is the largest
// |v| and, among equal magnitudes, the first row.  FP32: (|v| bits << 32) |
// ~row.  FP64: |v|'s sign-free bits with the low 16 cleared, | ~row in the
// low 16 bits (rows below 2^16): the winner is within 2^-36 of the
// column's largest |v| (first row among those that agree in the top 47
// bits), as stable a choice as the exact maximum.
template <typename T>
struct PivKey;
template <>
struct PivKey<float> {
  static constexpr int kMaxRows = 0x7fffffff;
  __device__ static unsigned long long make(float a, int row) {
    return ((unsigned long long)__float_as_uint(a) << 32) | (0xffffffffull - (unsigned)row);
  }
  __device__ static int row(unsigned long long key) { return (int)(0xffffffffull - (key & 0xffffffffull)); }
};
template <>
struct PivKey<double> {
  static constexpr int kMaxRows = 0xffff;
  __device__ static unsigned long long make(double a, int row) {
    return ((unsigned long long)__double_as_longlong(a) & ~0xffffull) | (0xffffull - (unsigned)row);
  }
  __device__ static int row(unsigned long long key) { return (int)(0xffffull - (key & 0xffffull)); }
};

// The panel with the pivot elected by one 64-bit atomicMax per CTA and
// column (PivKey).  Per column:
//   1. each warp finds its best row among the CTA's rows >= c; warp 0
//      reduces the eight, posts the key and publishes that row; the owner
//      of row c publishes it (the row a swap moves down);
//   2. grid barrier;
//   3. every thread reads the key, then its element of the winning row and
//      of row c (the two loads in flight together);
//   4. each warp takes rows below the pivot: multiplier l = a(i,c) / pivot,
//      a(i,k) -= l * u(k) for k > c; the swapped-in row is taken from the
//      copy of row c and the pivot row is written over row c, so the swap
//      needs no barrier of its own.
// Keys are triple-buffered (the buffer for column c + 1 is cleared while
// column c is elected), rows double-buffered by column parity.  FP64 panels
// of more than PivKey<double>::kMaxRows rows take k_lu_panel.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_lu_panel_at(T* __restrict__ W, int ldw, int n, int k0, int kb, int R,
                                                         int* __restrict__ piv, PanelBuf pb, int* fail) {
  extern __shared__ __align__(16) unsigned char smem[];
  T* S = reinterpret_cast<T*>(smem);  // R x (kLB + 1)
  T* prow = S + (size_t)R * (kLB + 1);  // the pivot row
  T* drow = prow + kLB;                 // the old row c
  __shared__ T s_best[kWarps];
  __shared__ int s_idx[kWarps];
  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int m = n - k0;
  const int rlo = b * R, rhi = min(m, rlo + R);
  const int nr = max(0, rhi - rlo);
  for (int c = w; c < kb; c += kWarps)
    for (int i = lane; i < nr; i += 32) S[i * (kLB + 1) + c] = W[(size_t)(k0 + c) * ldw + k0 + rlo + i];
  __syncthreads();
  T* rowsT = reinterpret_cast<T*>(pb.rows);
  T* diagT = reinterpret_cast<T*>(pb.diag);
  for (int c = 0; c < kb; ++c) {
    const int buf = c & 1;
    T best = T(-1);
    int bi = 0x7fffffff;
    for (int i = max(0, c - rlo) + tid; i < nr; i += kThreads) {
      const T a = fabs(S[i * (kLB + 1) + c]);
      if (a > best) { best = a; bi = rlo + i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { s_best[w] = best; s_idx[w] = bi; }
    if (c >= rlo && c < rhi && w == kWarps - 1)  // row c, as it stands, for the swap
      for (int k = lane; k < kb; k += 32) diagT[(size_t)buf * kLB + k] = S[(c - rlo) * (kLB + 1) + k];
    __syncthreads();
    if (w == 0) {
      best = lane < kWarps ? s_best[lane] : T(-1);
      bi = lane < kWarps ? s_idx[lane] : 0x7fffffff;
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) {
        const T ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      best = __shfl_sync(0xffffffffu, best, 0);
      bi = __shfl_sync(0xffffffffu, bi, 0);
      if (bi != 0x7fffffff) {
        for (int k = lane; k < kb; k += 32) rowsT[((size_t)buf * G + b) * kLB + k] = S[(bi - rlo) * (kLB + 1) + k];
        if (lane == 0 && best >= T(0)) atomicMax(pb.key + c % 3, PivKey<T>::make(best, bi));
      }
      // the next column's key was last read after barrier c - 2: clear it now
      if (b == 0 && lane == 0) pb.key[(c + 1) % 3] = 0ull;
    }
    __threadfence();
    if (!grid_barrier_count(pb.bar, (unsigned)(c + 1) * (unsigned)G, pb.err)) return;
    const unsigned long long key = *(volatile unsigned long long*)(pb.key + c % 3);
    const int p = key ? PivKey<T>::row(key) : 0x7fffffff;
    const int wb = (p != 0x7fffffff) ? p / R : -1;
    const bool okw = wb >= 0 && wb < G;
    if (tid < kb) {
      prow[tid] = okw ? ((volatile T*)rowsT)[((size_t)buf * G + wb) * kLB + tid] : T(0);
      drow[tid] = ((volatile T*)diagT)[(size_t)buf * kLB + tid];
    }
    __syncthreads();
    const T pv = prow[c];
    const bool stop = !okw || p < c || p >= m || pv == T(0) || pv != pv;  // uniform: the same key everywhere
    if (tid == 0 && b == 0) {
      if (stop) *fail = k0 + c + 1;
      else piv[k0 + c] = k0 + p;
    }
    if (stop) return;
    const T inv = T(1) / pv;
    const int pl = (p != c && p >= rlo && p < rhi) ? p - rlo : -1;  // the swapped-in row, if here
    for (int i = max(0, c + 1 - rlo) + w; i < nr; i += kWarps) {
      T* row = S + i * (kLB + 1);
      const T* src = (i == pl) ? drow : row;
      const T l = src[c] * inv;
      if (i == pl)
        for (int k = lane; k < c; k += 32) row[k] = drow[k];
      for (int k = c + 1 + lane; k < kb; k += 32) row[k] = src[k] - l * prow[k];
      __syncwarp();
      if (lane == 0) row[c] = l;
    }
    if (p != c && c >= rlo && c < rhi)  // the pivot row moves up to row c
      for (int k = tid; k < kb; k += kThreads) S[(c - rlo) * (kLB + 1) + k] = prow[k];
    __syncthreads();
  }
  for (int c = w; c < kb; c += kWarps)
    for (int i = lane; i < nr; i += 32) W[(size_t)(k0 + c) * ldw + k0 + rlo + i] = S[i * (kLB + 1) + c];
}

// Row swaps of one panel applied to every column outside it.
template <typename T>
__global__ void k_swap_rows(T* W, int ldw, int n, int k0, int kb, const int* __restrict__ piv) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= n || (col >= k0 && col < k0 + kb)) return;
  T* cp = W + (size_t)col * ldw;
  for (int c = 0; c < kb; ++c) {
    const int p = piv[k0 + c];
    if (p != k0 + c) {
      const T a = cp[k0 + c];
      cp[k0 + c] = cp[p];
      cp[p] = a;
    }
  }
}

template <int BYTES>
__device__ __forceinline__ void cp_async_el(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if (BYTES == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }


// ------------------------------------------- FP64 GEMM (mma.sync f64)
// C (M x N) -= A (M x K) * B (K x N) (B transposed when TB); LO skips tiles
// strictly above the diagonal.  CTA tile 128 x 64, eight warps of 32 x 32
// (4 x 4 m8n8k4 tiles each), K steps of 16 double-buffered in shared memory
// with cp.async so the global loads of step k+1 overlap the MMAs of step k.
constexpr int kDmM = 128, kDmN = 64, kDmK = 16;
constexpr int kDmPA = kDmM + 8, kDmPB = kDmN + 8;  // padded rows: the 4 k of a fragment hit other banks
constexpr size_t kDmSmem = sizeof(double) * 2 * kDmK * (kDmPA + kDmPB);

template <bool TB, bool LO>
__global__ void __launch_bounds__(kThreads) k_gemm_dmma(double* __restrict__ C, int ldc, const double* __restrict__ A,
                                                       int lda, const double* __restrict__ B, int ldb, int M, int N,
                                                       int K) {
  const int m0 = blockIdx.x * kDmM, n0 = blockIdx.y * kDmN;
  if (LO && n0 >= m0 + kDmM) return;
  extern __shared__ __align__(16) unsigned char smem[];
  double(*As)[kDmK][kDmPA] = reinterpret_cast<double(*)[kDmK][kDmPA]>(smem);
  double(*Bs)[kDmK][kDmPB] = reinterpret_cast<double(*)[kDmK][kDmPB]>(smem + sizeof(double) * 2 * kDmK * kDmPA);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int wr = (w & 3) * 32, wc = (w >> 2) * 32;
  auto load = [&](int buf, int k0) {
    for (int e = tid; e < kDmK * kDmM; e += kThreads) {
      const int r = e & (kDmM - 1), k = e >> 7;
      double* dst = &As[buf][k][r];
      if (m0 + r < M && k0 + k < K) cp_async_el<8>(dst, A + (size_t)(k0 + k) * lda + m0 + r);
      else *dst = 0.0;
    }
    for (int e = tid; e < kDmK * kDmN; e += kThreads) {
      int k, c;
      if (TB) { c = e & (kDmN - 1); k = e >> 6; }
      else { k = e & (kDmK - 1); c = e >> 4; }
      double* dst = &Bs[buf][k][c];
      if (n0 + c < N && k0 + k < K)
        cp_async_el<8>(dst, TB ? B + (size_t)(k0 + k) * ldb + n0 + c : B + (size_t)(n0 + c) * ldb + k0 + k);
      else *dst = 0.0;
    }
    cp_async_commit();
  };
  double acc[4][4][2];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[a][q][0] = acc[a][q][1] = 0.0;
  const int nk = (K + kDmK - 1) / kDmK;
  if (nk > 0) load(0, 0);
  for (int ks = 0; ks < nk; ++ks) {
    const int buf = ks & 1;
    if (ks + 1 < nk) {
      load(buf ^ 1, (ks + 1) * kDmK);
      cp_async_wait1();
    } else {
      cp_async_wait0();
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kDmK; kk += 4) {
      double af[4], bf[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) af[a] = As[buf][kk + t][wr + a * 8 + g];
#pragma unroll
      for (int q = 0; q < 4; ++q) bf[q] = Bs[buf][kk + t][wc + q * 8 + g];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int q = 0; q < 4; ++q) dmma_8x8x4(acc[a][q][0], acc[a][q][1], af[a], bf[q]);
    }
    __syncthreads();
  }
  // epilogue: all loads of C first, then the stores
  double cv[4][4][2];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = m0 + wr + a * 8 + g, c = n0 + wc + q * 8 + 2 * t + h;
        cv[a][q][h] = (r < M && c < N) ? C[(size_t)c * ldc + r] : 0.0;
      }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = m0 + wr + a * 8 + g, c = n0 + wc + q * 8 + 2 * t + h;
        if (r < M && c < N) C[(size_t)c * ldc + r] = cv[a][q][h] - acc[a][q][h];
      }
}

// ------------------------------------------- wavefront triangular solve
// op(T) x = b for a triangular T (Sec. 2.2, Eq. 3 by BW-row blocks), one
// launch for the whole solve.  Work items are (right-hand-side chunk of 8,
// block row in solve order); CTA c takes items c, c+G, ... in order.  The
// item for block row o accumulates -op(T)(o, p) x_p for every earlier block
// p as soon as p's flag is set, then solves its diagonal block by warp
// substitution (no inverse: FP64-stable), stores x_o and sets its flag.
// The tiles of T do not depend on any flag: each is copied into shared
// memory with cp.async one pair ahead (double buffer), so only x_p waits.
// Every CTA is co-resident (cooperative launch) and an item waits only on
// items of lower index, so the lowest unfinished item can always proceed.
// Waits are bounded: on expiry the kernel sets *err and returns.
constexpr int kWaveNR = 8;

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// block width of the solve: 128 rows for FP32 factors, 64 for FP64 (two
// tiles of BW x (BW+1) elements in shared memory either way)
template <typename T>
struct WaveBW {
  static constexpr int value = sizeof(T) == 4 ? 128 : 64;
};

// Dinv (optional): inverses of the BW x BW diagonal blocks of the triangle,
// block b at Dinv + b * BW * BW, column-major (k_diag_inv).  With them the
// diagonal step is a product with the inverse instead of a substitution.
template <typename T, typename V>
__global__ void __launch_bounds__(kThreads, 1) k_trsv_wave(const T* __restrict__ M, int ldm, int n, int lower, int trans,
                                                       int unit, V* x, int ldx, int nrhs, int* flags, int* err,
                                                       const T* __restrict__ Dinv) {
  constexpr int BW = WaveBW<T>::value;
  constexpr int P = kThreads / BW;          // thread parts per row
  constexpr int NQ = kWaveNR / P;           // right-hand sides per thread (multi mode)
  extern __shared__ __align__(16) unsigned char smem[];
  T(*tile)[BW][BW + 1] = reinterpret_cast<T(*)[BW][BW + 1]>(smem);  // [2][col][row]
  V(*xs)[BW] = reinterpret_cast<V(*)[BW]>(smem + sizeof(T) * 2 * BW * (BW + 1));  // [NR][BW]
  __shared__ int s_ok;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const bool elower = (lower != 0) != (trans != 0);
  const int nblk = (n + BW - 1) / BW;
  const int nchunk = (nrhs + kWaveNR - 1) / kWaveNR;
  const int items = nblk * nchunk;
  const int r = tid % BW, part = tid / BW;
  if (tid == 0) s_ok = 1;
  __syncthreads();
  // copy the tile of M holding op(T)(block bi, block bj) into buffer buf
  auto issue = [&](int buf, int bi, int bj) {
    const int col0 = (trans ? bi : bj) * BW, row0 = (trans ? bj : bi) * BW;
    const int nc_ = min(BW, n - col0), nr_ = min(BW, n - row0);
    for (int e = tid; e < BW * BW; e += kThreads) {
      const int c = e / BW, rr = e % BW;
      T* dst = &tile[buf][c][rr];
      if (c < nc_ && rr < nr_) cp_async_el<sizeof(T)>(dst, M + (size_t)(col0 + c) * ldm + row0 + rr);
      else *dst = T(0);
    }
    cp_async_commit();
  };
  // the inverse of diagonal block bi (op applies to it as to T's tiles)
  auto issue_inv = [&](int buf, int bi) {
    const T* src = Dinv + (size_t)bi * BW * BW;
    for (int e = tid; e < BW * BW; e += kThreads) {
      const int c = e / BW, rr = e % BW;
      cp_async_el<sizeof(T)>(&tile[buf][c][rr], src + (size_t)c * BW + rr);
    }
    cp_async_commit();
  };
  // element (i, j) of op(T)(bi, bj) in buffer buf
  auto E = [&](int buf, int i, int j) -> V { return trans ? (V)tile[buf][i][j] : (V)tile[buf][j][i]; };
  for (int it = blockIdx.x; it < items; it += gridDim.x) {
    const int chunk = it / nblk, o = it - chunk * nblk;
    const int c0 = chunk * kWaveNR, nc = min(kWaveNR, nrhs - c0);
    const bool single = nc == 1;
    const int bo = elower ? o : nblk - 1 - o;
    const int r0 = bo * BW, bs = min(BW, n - r0);
    V acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int c = part + P * q;
      const bool on = single ? (q == 0 && part == 0) : (c < nc);
      acc[q] = (on && r < bs) ? x[(size_t)(c0 + (single ? 0 : c)) * ldx + r0 + r] : V(0);
    }
    // first tile: pair (o, 0), or the diagonal block when o == 0
    if (o > 0) issue(0, bo, elower ? 0 : nblk - 1);
    else if (Dinv) issue_inv(0, bo);
    else issue(0, bo, bo);
    for (int p = 0; p < o; ++p) {
      const int bp = elower ? p : nblk - 1 - p;
      const int buf = p & 1;
      // prefetch the next pair's tile (or the diagonal block) meanwhile
      if (p + 1 < o) issue(buf ^ 1, bo, elower ? p + 1 : nblk - 2 - p);
      else if (Dinv) issue_inv(buf ^ 1, bo);
      else issue(buf ^ 1, bo, bo);
      if (tid == 0) {
        const int* f = flags + chunk * nblk + p;
        long long spins = 0;
        while (ld_acquire(f) == 0) {
          if (++spins > 100000000ll) {
            s_ok = 0;
            atomicExch(err, 1);
            break;
          }
        }
      }
      __syncthreads();
      if (!s_ok) {
        cp_async_wait0();
        return;
      }
      const int p0 = bp * BW, ps = min(BW, n - p0);
      for (int e = tid; e < kWaveNR * BW; e += kThreads) {
        const int j = e % BW, c = e / BW;
        xs[c][j] = (j < ps && c < nc) ? __ldcg(x + (size_t)(c0 + c) * ldx + p0 + j) : V(0);
      }
      cp_async_wait1();
      __syncthreads();
      if (single) {  // one right-hand side: the parts split the j range
        const int j0 = part * (BW / P);
#pragma unroll 8
        for (int j = j0; j < j0 + BW / P; ++j) acc[0] -= E(buf, r, j) * xs[0][j];
      } else {
#pragma unroll 4
        for (int j = 0; j < BW; ++j) {
          const V e = E(buf, r, j);
#pragma unroll
          for (int q = 0; q < NQ; ++q) acc[q] -= e * xs[part + P * q][j];
        }
      }
      __syncthreads();
    }
    cp_async_wait0();
    __syncthreads();  // every thread's copies of the diagonal tile have landed
    const int dbuf = o & 1;
    // right-hand side of the diagonal block into xs
    if (single) {
      xs[part][r] = acc[0];
      __syncthreads();
      if (part == 0) {
        V t = xs[0][r];
#pragma unroll
        for (int k = 1; k < P; ++k) t += xs[k][r];
        xs[0][r] = t;
      }
    } else {
#pragma unroll
      for (int q = 0; q < NQ; ++q) xs[part + P * q][r] = acc[q];
    }
    if (Dinv) {
      // x = inv(D) rhs: the same product as the pair updates, from zero
      __syncthreads();
      if (single) {
        const int j0 = part * (BW / P);
        V t = V(0);
#pragma unroll 8
        for (int j = j0; j < j0 + BW / P; ++j) t += E(dbuf, r, j) * xs[0][j];
        xs[1 + part][r] = t;  // rows 1..P of xs are free in this mode
        __syncthreads();
        if (part == 0 && r < bs) {
          V u = xs[1][r];
#pragma unroll
          for (int k = 1; k < P; ++k) u += xs[1 + k][r];
          x[(size_t)c0 * ldx + r0 + r] = u;
        }
      } else {
        V t[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) t[q] = V(0);
#pragma unroll 4
        for (int j = 0; j < BW; ++j) {
          const V e = E(dbuf, r, j);
#pragma unroll
          for (int q = 0; q < NQ; ++q) t[q] += e * xs[part + P * q][j];
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int c = part + P * q;
          if (c < nc && r < bs) x[(size_t)(c0 + c) * ldx + r0 + r] = t[q];
        }
      }
      __threadfence();
      __syncthreads();
      if (tid == 0) st_release(flags + it, 1);
      continue;
    }
    // reciprocals of the diagonal (one division per row, off the chain)
    __shared__ V s_rinv[BW];
    for (int i = tid; i < BW; i += kThreads) s_rinv[i] = (unit || i >= bs) ? V(1) : V(1) / E(dbuf, i, i);
    __syncthreads();
    // diagonal block: warp w substitutes for right-hand side w
    if (w < nc) {
      constexpr int NV = (BW + 31) / 32;
      V v[NV];
#pragma unroll
      for (int k = 0; k < NV; ++k) v[k] = (k * 32 + lane < BW) ? xs[w][k * 32 + lane] : V(0);
      // register kk of the lanes holds rows 32kk..32kk+31: the outer loop
      // index names the register statically
#pragma unroll
      for (int kq = 0; kq < NV; ++kq) {
        const int kk = elower ? kq : NV - 1 - kq;
        for (int jq = 0; jq < 32; ++jq) {
          const int jj = elower ? jq : 31 - jq;
          const int j = kk * 32 + jj;
          if (j >= bs) continue;
          const V vk = elower ? v[kq] : v[NV - 1 - kq];  // static register either way
          const V vj = __shfl_sync(0xffffffffu, vk, jj) * s_rinv[j];
#pragma unroll
          for (int k = 0; k < NV; ++k) {
            const int i = k * 32 + lane;
            const bool below = elower ? i > j : i < j;
            const V upd = v[k] - E(dbuf, i < BW ? i : 0, j) * vj;
            v[k] = (i == j) ? vj : ((i < bs && below) ? upd : v[k]);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        const int i = k * 32 + lane;
        if (i < bs) x[(size_t)(c0 + w) * ldx + r0 + i] = v[k];
      }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) st_release(flags + it, 1);
  }
}

// FP64 residual for up to 8 right-hand sides, split over k so that every
// SM has many independent loads of A in flight: blockIdx.y takes the k
// segment [seg * klen, (seg + 1) * klen) and writes its partial products
// P[seg][c][r]; k_residual_sum adds the segments in order (the result does
// not depend on scheduling) and forms R = B - sum and max |R|.  One thread
// per row on DFMA with exactly NR accumulators (A read once, eight loads
// ahead): an FP64 instruction costs its pipe time whether its lanes are on
// or off, so a column count fixed at compile time wastes none (the 8-column
// mma.sync f64 form spent 8 columns' work at any nrhs).
constexpr int kResMaxSeg = 32;
template <int NR>
__global__ void __launch_bounds__(256) k_residual_part_fma(const double* __restrict__ A, int n,
                                                           const double* __restrict__ X, int klen,
                                                           double* __restrict__ P) {
  const int r = blockIdx.x * 256 + threadIdx.x, seg = blockIdx.y;
  const int k0 = seg * klen, k1 = min(n, k0 + klen);
  if (r >= n) return;
  double s[NR];
#pragma unroll
  for (int c = 0; c < NR; ++c) s[c] = 0.0;
  int k = k0;
  for (; k + 8 <= k1; k += 8) {
    double a[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = __ldg(A + (size_t)(k + q) * n + r);
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
      for (int c = 0; c < NR; ++c) s[c] = fma(a[q], __ldg(X + (size_t)c * n + k + q), s[c]);
  }
  for (; k < k1; ++k) {
    const double a = __ldg(A + (size_t)k * n + r);
#pragma unroll
    for (int c = 0; c < NR; ++c) s[c] = fma(a, __ldg(X + (size_t)c * n + k), s[c]);
  }
#pragma unroll
  for (int c = 0; c < NR; ++c) P[((size_t)seg * NR + c) * n + r] = s[c];
}

__global__ void k_residual_sum(const double* __restrict__ P, int nseg, int n, int nrhs,
                               const double* __restrict__ B, double* __restrict__ R,
                               unsigned long long* rmax) {
  const int c = blockIdx.y;
  double m = 0.0;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int seg = 0; seg < nseg; ++seg) s += P[((size_t)seg * nrhs + c) * n + r];
    const double v = B[(size_t)c * n + r] - s;
    R[(size_t)c * n + r] = v;
    m = fmax(m, fabs(v));
  }
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) atomicMax(rmax + c, (unsigned long long)__double_as_longlong(m));
}

// ------------------------------------------------------ vector helpers
template <typename V>
__global__ void k_colmax_abs(const V* __restrict__ x, int n, int nrhs, unsigned long long* out) {
  for (int c = blockIdx.y; c < nrhs; c += gridDim.y) {
    double m = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
      m = fmax(m, fabs((double)x[(size_t)c * n + i]));
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) atomicMax(out + c, (unsigned long long)__double_as_longlong(m));
  }
}

// xs = (V)(src / scale[c])  and  x += (double)xs * scale[c]
template <typename V>
__global__ void k_scale_down(const double* __restrict__ src, int n, int nrhs, const double* scale, V* dst) {
  const size_t tot = (size_t)n * nrhs;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x)
    dst[e] = (V)(src[e] / scale[e / n]);
}
template <typename V>
__global__ void k_scale_add(double* __restrict__ x, int n, int nrhs, const double* scale, const V* d, int assign) {
  const size_t tot = (size_t)n * nrhs;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const double v = (double)d[e] * scale[e / n];
    x[e] = assign ? v : x[e] + v;
  }
}

// ---- GMRES-IR kernels: the Krylov basis V (columns of n doubles, ld ldv)
// h[j] = V_j . w for j < m: a CTA per column, a fixed-order block sum.
__global__ void __launch_bounds__(256) k_krylov_dots(const double* __restrict__ V, int64_t ldv, int n, int m,
                                                     const double* __restrict__ w, double* __restrict__ h) {
  __shared__ double red[8];
  const int j = blockIdx.x;
  if (j >= m) return;
  const double* v = V + (size_t)j * ldv;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s = fma(v[i], w[i], s);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += red[k];
    h[j] = t;
  }
}

// w += sign * sum_{j < m} V_j h[j], a thread per row.
__global__ void k_krylov_comb(double* __restrict__ w, const double* __restrict__ V, int64_t ldv, int n, int m,
                              const double* __restrict__ h, double sign) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < m; ++j) s = fma(V[(size_t)j * ldv + i], h[j], s);
    w[i] += sign * s;
  }
}

// dst = (float)(src * inv)  and  dst = (double)src * s
__global__ void k_vec_to_f32(const double* __restrict__ src, int n, double inv, float* __restrict__ dst) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    dst[i] = (float)(src[i] * inv);
}
__global__ void k_vec_from_f32(const float* __restrict__ src, int n, double s, double* __restrict__ dst) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    dst[i] = (double)src[i] * s;
}
__global__ void k_vec_scale(double* __restrict__ dst, const double* __restrict__ src, int n, double s) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[i] * s;
}

// permutation: dst[k] = src[perm[k]] (forward) or dst[perm[k]] = src[k]
template <typename V>
__global__ void k_permute(const V* __restrict__ src, V* __restrict__ dst, int n, int nrhs, const int* perm, int inverse) {
  const size_t tot = (size_t)n * nrhs;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(e % n);
    const size_t c = e / n;
    if (!inverse) dst[e] = src[c * n + perm[k]];
    else dst[c * n + perm[k]] = src[e];
  }
}

__global__ void k_build_perm(const int* piv, int n, int* perm) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int k = 0; k < n; ++k) perm[k] = k;
  for (int k = 0; k < n; ++k) {
    const int p = piv[k];
    const int t = perm[k];
    perm[k] = perm[p];
    perm[p] = t;
  }
}


// ===================================================================== host
size_t scan_large_workspace(int64_t n);
cudaError_t launch_scan_large(const double* A, int64_t n, const double* B, int64_t nb, double band_frac,
                              double tol, void* ws, ScanRes* out, int num_sms, cudaStream_t st);


namespace {

struct Arena {
  char* base;
  size_t used, cap;
  void* take(size_t bytes) {
    const size_t off = (used + 255) & ~(size_t)255;
    if (off + bytes > cap) return nullptr;
    used = off + bytes;
    return base + off;
  }
};

#define LCK(x)                                      \
  do {                                              \
    cudaError_t _e = (x);                           \
    if (_e != cudaSuccess) return ASOLVE_E_CUDA;    \
  } while (0)

// R = B - A X in FP64 with rmax[c] |= max |R(:, c)| (rmax zeroed by the
// caller); P: kResMaxSeg x 8 x n doubles of scratch.
// K columns of A per Ozaki-split residual product (bounds its workspace
// to gemm_oz_ws_bytes(n, nrhs, kOzResK))
constexpr int kOzResK = 1024;

int residual_large(const double* A, int n, const double* B, const double* X, int nrhs, double* R,
                   unsigned long long* rmax, double* P, int num_sms, cudaStream_t st, void* ozws = nullptr,
                   int* err = nullptr) {
  if (nrhs > 8) {  // R = B, then R -= A X, then max |R|
    LCK(cudaMemcpyAsync(R, B, sizeof(double) * (size_t)n * nrhs, cudaMemcpyDeviceToDevice, st));
    if (ozws) {  // Ozaki-split products on the tensor cores, kOzResK columns of A at a time
      for (int k0 = 0; k0 < n; k0 += kOzResK)
        LCK(gemm_oz(R, n, A + (size_t)k0 * n, n, X + k0, n, n, nrhs, std::min(kOzResK, n - k0), false, false, ozws,
                    err, st));
    } else {  // the mma.sync f64 GEMM
      k_gemm_dmma<false, false><<<dim3((n + kDmM - 1) / kDmM, (nrhs + kDmN - 1) / kDmN), kThreads, kDmSmem, st>>>(
          R, n, A, n, X, n, n, nrhs, n);
    }
    k_colmax_abs<double><<<dim3(64, nrhs), 256, 0, st>>>(R, n, nrhs, rmax);
    LCK(cudaGetLastError());
    return ASOLVE_OK;
  }
  const int gx = (n + 255) / 256;
  int nseg = (4 * num_sms + gx - 1) / gx;  // about four CTAs of loads per SM
  nseg = nseg < 1 ? 1 : (nseg > kResMaxSeg ? kResMaxSeg : nseg);
  int klen = (n + nseg - 1) / nseg;
  klen = (klen + 7) & ~7;
  nseg = (n + klen - 1) / klen;
  const dim3 grid(gx, nseg);
  switch (nrhs) {
    case 1: k_residual_part_fma<1><<<grid, 256, 0, st>>>(A, n, X, klen, P); break;
    case 2: k_residual_part_fma<2><<<grid, 256, 0, st>>>(A, n, X, klen, P); break;
    case 3: k_residual_part_fma<3><<<grid, 256, 0, st>>>(A, n, X, klen, P); break;
    case 4: k_residual_part_fma<4><<<grid, 256, 0, st>>>(A, n, X, klen, P); break;
    case 5: k_residual_part_fma<5><<<grid, 256, 0, st>>>(A, n, X, klen, P); break;
    case 6: k_residual_part_fma<6><<<grid, 256, 0, st>>>(A, n, X, klen, P); break;
    case 7: k_residual_part_fma<7><<<grid, 256, 0, st>>>(A, n, X, klen, P); break;
    default: k_residual_part_fma<8><<<grid, 256, 0, st>>>(A, n, X, klen, P); break;
  }
  k_residual_sum<<<dim3((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024, nrhs), 256, 0, st>>>(P, nseg, n, nrhs,
                                                                                              B, R, rmax);
  LCK(cudaGetLastError());
  return ASOLVE_OK;
}

// Scratch of the wavefront triangular solve: one flag per work item.
struct WaveBuf {
  int* flags;
  int* err;
  int cap;  // flags available
  int grid; // co-resident CTAs
};

// Inverses of the 128 x 128 diagonal blocks of FP32 factors, for the
// wavefront solve's diagonal step: Linv[b] = inv(L(b, b)) (unit diagonal
// when unitL; only the triangle below the diagonal is read),
// Uinv[b] = inv(U(b, b)) (upper triangle with the diagonal), each block
// column-major with ld 128 and the identity past the matrix's last row.
// One CTA per block: threads 0..127 form the columns of inv(L), threads
// 128..255 those of inv(U), by substitution against the identity (rows in
// increasing, respectively decreasing, order).  Either output may be null.
constexpr int kInvBW = 128;
constexpr size_t kDiagInvSmem = sizeof(float) * 3 * kInvBW * (kInvBW + 1);
__global__ void __launch_bounds__(kThreads, 1) k_diag_inv(const float* __restrict__ W, int ldw, int n, int unitL,
                                                        float* __restrict__ Linv, float* __restrict__ Uinv) {
  constexpr int BW = kInvBW, LD = BW + 1;
  extern __shared__ __align__(16) unsigned char smem[];
  float* D = reinterpret_cast<float*>(smem);  // D[i * LD + k] = W(r0 + i, r0 + k)
  float* XL = D + BW * LD;                    // XL[i * LD + j] = inv(L)(i, j)
  float* XU = XL + BW * LD;
  const int b = blockIdx.x, r0 = b * BW, bs = min(BW, n - r0), tid = threadIdx.x;
  for (int e = tid; e < BW * BW; e += kThreads) {
    const int k = e / BW, i = e % BW;  // column k, row i: coalesced over i
    D[i * LD + k] = (i < bs && k < bs) ? W[(size_t)(r0 + k) * ldw + r0 + i] : 0.f;
    XL[i * LD + k] = 0.f;
    XU[i * LD + k] = 0.f;
  }
  __syncthreads();
  const int j = tid & (BW - 1);
  if (tid < BW) {
    if (Linv)
      for (int i = 0; i < BW; ++i) {
        float s = (i == j) ? 1.f : 0.f;
        for (int k = 0; k < i; ++k) s -= D[i * LD + k] * XL[k * LD + j];
        XL[i * LD + j] = (i >= bs || unitL) ? s : s / D[i * LD + i];
      }
  } else if (Uinv) {
    for (int i = BW - 1; i >= 0; --i) {
      float s = (i == j) ? 1.f : 0.f;
      for (int k = i + 1; k < BW; ++k) s -= D[i * LD + k] * XU[k * LD + j];
      XU[i * LD + j] = (i >= bs) ? s : s / D[i * LD + i];
    }
  }
  __syncthreads();
  for (int e = tid; e < BW * BW; e += kThreads) {
    const int k = e / BW, i = e % BW;
    if (Linv) Linv[(size_t)b * BW * BW + (size_t)k * BW + i] = XL[i * LD + k];
    if (Uinv) Uinv[(size_t)b * BW * BW + (size_t)k * BW + i] = XU[i * LD + k];
  }
}

template <typename T, typename V>
constexpr size_t wave_smem() {
  return sizeof(T) * 2 * (size_t)WaveBW<T>::value * (WaveBW<T>::value + 1) +
         sizeof(V) * (size_t)kWaveNR * WaveBW<T>::value;
}

template <typename T>
struct Fac {  // a factorisation of the large path and its scratch
  T* W;
  int ldw;
  int* piv;
  int* perm;
  T* Dtmp;       // 128 x 128 inverse of the current diagonal block
  int* fail;     // device
  PanelBuf pb;
  WaveBuf wb;
  int gemm_mode = 3;  // FP32 factors: operand mode of the trailing updates (launch_gemm_tc)
  void* ozws = nullptr;  // FP64 factors: Ozaki-split trailing updates (gemm_oz) in this workspace
  const T* dinvL = nullptr;  // FP32 factors: inverses of the 128 x 128 diagonal blocks (k_diag_inv)
  const T* dinvU = nullptr;
};

template <typename T>
int tri_solve_large(const T* M, int ldm, int n, bool lower, bool trans, bool unit, void* xv, int nrhs,
                    bool vfloat, const WaveBuf& wb, cudaStream_t st, const T* dinv = nullptr) {
  const int nblk = (n + WaveBW<T>::value - 1) / WaveBW<T>::value;
  const int items = nblk * ((nrhs + kWaveNR - 1) / kWaveNR);
  if (items > wb.cap) return ASOLVE_E_NOMEM;
  LCK(cudaMemsetAsync(wb.flags, 0, sizeof(int) * (size_t)items, st));
  int G = std::min(wb.grid, items);
  int lw = lower, tw = trans, uw = unit, ld = ldm, nn = n, nr = nrhs, ldx = n;
  int* fl = wb.flags;
  int* er = wb.err;
  const T* Mp = M;
  const T* Dp = dinv;
  if (vfloat) {
    float* x = static_cast<float*>(xv);
    void* args[] = {&Mp, &ld, &nn, &lw, &tw, &uw, &x, &ldx, &nr, &fl, &er, &Dp};
    LCK(cudaLaunchCooperativeKernel((void*)k_trsv_wave<T, float>, dim3(G), dim3(kThreads), args,
                                    wave_smem<T, float>(), st));
  } else {
    double* x = static_cast<double*>(xv);
    void* args[] = {&Mp, &ld, &nn, &lw, &tw, &uw, &x, &ldx, &nr, &fl, &er, &Dp};
    LCK(cudaLaunchCooperativeKernel((void*)k_trsv_wave<T, double>, dim3(G), dim3(kThreads), args,
                                    wave_smem<T, double>(), st));
  }
  return ASOLVE_OK;
}

template <typename T, typename V>
int apply_large(const Fac<T>& f, bool lu, int n, V* x, int nrhs, bool trans, V* tmp, cudaStream_t st) {
  const bool vf = sizeof(V) == 4;
  const int g = 1024;
  if (lu) {
    if (!trans) {
      k_permute<V><<<g, 256, 0, st>>>(x, tmp, n, nrhs, f.perm, 0);
      LCK(cudaMemcpyAsync(x, tmp, sizeof(V) * (size_t)n * nrhs, cudaMemcpyDeviceToDevice, st));
      int rc = tri_solve_large<T>(f.W, f.ldw, n, true, false, true, x, nrhs, vf, f.wb, st, f.dinvL);
      if (rc) return rc;
      return tri_solve_large<T>(f.W, f.ldw, n, false, false, false, x, nrhs, vf, f.wb, st, f.dinvU);
    }
    int rc = tri_solve_large<T>(f.W, f.ldw, n, false, true, false, x, nrhs, vf, f.wb, st, f.dinvU);
    if (rc) return rc;
    rc = tri_solve_large<T>(f.W, f.ldw, n, true, true, true, x, nrhs, vf, f.wb, st, f.dinvL);
    if (rc) return rc;
    k_permute<V><<<g, 256, 0, st>>>(x, tmp, n, nrhs, f.perm, 1);
    LCK(cudaMemcpyAsync(x, tmp, sizeof(V) * (size_t)n * nrhs, cudaMemcpyDeviceToDevice, st));
    return ASOLVE_OK;
  }
  int rc = tri_solve_large<T>(f.W, f.ldw, n, true, false, false, x, nrhs, vf, f.wb, st, f.dinvL);
  if (rc) return rc;
  return tri_solve_large<T>(f.W, f.ldw, n, true, true, false, x, nrhs, vf, f.wb, st, f.dinvL);
}

template <typename T>
cudaError_t gemm_update(T* C, int ldc, const T* A, int lda, const T* B, int ldb, int M, int N, int K, bool tb,
                        bool lower, int* err, int mode, cudaStream_t st, void* ozws = nullptr);
template <>
cudaError_t gemm_update<float>(float* C, int ldc, const float* A, int lda, const float* B, int ldb, int M, int N,
                               int K, bool tb, bool lower, int* err, int mode, cudaStream_t st, void*) {
  return launch_gemm_tc(C, ldc, A, lda, B, ldb, M, N, K, mode, err, st, tb, lower);
}
// FP64: the Ozaki-split product on the BF16 tensor cores when a workspace
// is given, else the mma.sync f64 GEMM
template <>
cudaError_t gemm_update<double>(double* C, int ldc, const double* A, int lda, const double* B, int ldb, int M, int N,
                                int K, bool tb, bool lower, int* err, int, cudaStream_t st, void* ozws) {
  if (ozws) return gemm_oz(C, ldc, A, lda, B, ldb, M, N, K, tb, lower, ozws, err, st);
  dim3 g((M + kDmM - 1) / kDmM, (N + kDmN - 1) / kDmN);
  if (tb && lower) k_gemm_dmma<true, true><<<g, kThreads, kDmSmem, st>>>(C, ldc, A, lda, B, ldb, M, N, K);
  else if (tb) k_gemm_dmma<true, false><<<g, kThreads, kDmSmem, st>>>(C, ldc, A, lda, B, ldb, M, N, K);
  else if (lower) k_gemm_dmma<false, true><<<g, kThreads, kDmSmem, st>>>(C, ldc, A, lda, B, ldb, M, N, K);
  else k_gemm_dmma<false, false><<<g, kThreads, kDmSmem, st>>>(C, ldc, A, lda, B, ldb, M, N, K);
  return cudaGetLastError();
}

// Shared memory limits of the large-path kernels on the current device.
template <typename T>
cudaError_t set_large_attrs_dev() {
#define SA(x)                                  \
  do {                                         \
    const cudaError_t e_ = (x);                \
    if (e_ != cudaSuccess) return e_;          \
  } while (0)
  SA(cudaFuncSetAttribute(k_trsm_sub<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)trsm_smem<T>()));
  SA(cudaFuncSetAttribute(k_trsm_rhs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)trsm_smem<double>()));
  SA(cudaFuncSetAttribute(k_gemm_dmma<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDmSmem));
  SA(cudaFuncSetAttribute(k_gemm_dmma<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDmSmem));
  SA(cudaFuncSetAttribute(k_gemm_dmma<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDmSmem));
  SA(cudaFuncSetAttribute(k_gemm_dmma<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDmSmem));
  // the panel kernel also has a little static shared memory
  if constexpr (sizeof(T) == 4) {
    SA(cudaFuncSetAttribute(k_lu_panel_at<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 226 * 1024));
    SA(cudaFuncSetAttribute(k_diag_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDiagInvSmem));
  }
  else
    SA(cudaFuncSetAttribute(k_lu_panel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 226 * 1024));
    SA(cudaFuncSetAttribute(k_lu_panel_at<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 226 * 1024));
  SA(cudaFuncSetAttribute(k_trsv_wave<T, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)wave_smem<T, float>()));
  SA(cudaFuncSetAttribute(k_trsv_wave<T, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)wave_smem<T, double>()));
  SA(cudaFuncSetAttribute(k_chol_diag<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024));
  return cudaSuccess;
#undef SA
}

// once per device and precision, from any host thread
template <typename T>
int set_large_attrs() {
  static PerDeviceOnce once;
  return once.run(set_large_attrs_dev<T>) == cudaSuccess ? ASOLVE_OK : ASOLVE_E_CUDA;
}

// Blocked Cholesky of the working matrix; returns 0 or (failing column + 1).
template <typename T>
int chol_large(Fac<T>& f, int n, int num_sms, int* fail_out, cudaStream_t st) {
  LCK(cudaMemsetAsync(f.fail, 0, sizeof(int) * 2, st));
  const int nb = sizeof(T) == 4 ? 32 : 16;
  const size_t dsm = (size_t)kLB * nb * sizeof(T) + 64 * 32 * sizeof(T) * 2 + 256;
  for (int k0 = 0; k0 < n; k0 += kLB) {
    const int kb = std::min(kLB, n - k0);
    k_chol_diag<T><<<1, kThreads, dsm, st>>>(f.W, f.ldw, k0, kb, nb, f.fail);
    const int rest = n - k0 - kb;
    if (rest > 0) {
      k_trsm_sub<T><<<(rest + 63) / 64, kThreads, trsm_smem<T>(), st>>>(f.W, f.ldw, k0, kb, k0 + kb, n, 1, 0);
      T* L21 = f.W + (size_t)k0 * f.ldw + k0 + kb;
      LCK(gemm_update<T>(f.W + (size_t)(k0 + kb) * f.ldw + k0 + kb, f.ldw, L21, f.ldw, L21, f.ldw, rest, rest, kb,
                         true, true, f.fail + 1, f.gemm_mode, st, f.ozws));
    }
  }
  LCK(cudaGetLastError());
  int h[2];
  LCK(cudaMemcpyAsync(h, f.fail, sizeof(h), cudaMemcpyDeviceToHost, st));
  LCK(cudaStreamSynchronize(st));
  if (h[1]) return ASOLVE_E_TIMEOUT;
  *fail_out = h[0];
  return ASOLVE_OK;
}

template <typename T>
int lu_large(Fac<T>& f, int n, int num_sms, int* fail_out, cudaStream_t st) {
  LCK(cudaMemsetAsync(f.fail, 0, sizeof(int) * 2, st));
  for (int k0 = 0; k0 < n; k0 += kLB) {
    const int kb = std::min(kLB, n - k0), m = n - k0;
    const int G = num_sms;
    const int R = (m + G - 1) / G;
    const size_t psmem = sizeof(T) * ((size_t)R * (kLB + 1) + 2 * kLB) + 64;
    if (psmem > 226 * 1024) return ASOLVE_E_UNSUPPORTED;
    LCK(cudaMemsetAsync(f.pb.bar, 0, sizeof(unsigned) * 2, st));
    LCK(cudaMemsetAsync(f.pb.key, 0, sizeof(unsigned long long) * 3, st));
    T* W = f.W;
    int ldw = f.ldw;
    int* piv = f.piv;
    PanelBuf pb = f.pb;
    int* fail = f.fail;
    void* args[] = {&W, &ldw, &n, &k0, (void*)&kb, (void*)&R, &piv, &pb, &fail};
    const void* kern;
    if (sizeof(T) == 4 || m <= PivKey<double>::kMaxRows + 1) kern = (const void*)k_lu_panel_at<T>;
    else kern = (const void*)k_lu_panel<T>;
    LCK(cudaLaunchCooperativeKernel(kern, dim3(G), dim3(kThreads), args, psmem, st));
    k_swap_rows<T><<<(n + 255) / 256, 256, 0, st>>>(f.W, f.ldw, n, k0, kb, f.piv);
    const int rest = n - k0 - kb;
    if (rest > 0) {
      k_trsm_sub<T><<<(rest + 63) / 64, kThreads, trsm_smem<T>(), st>>>(f.W, f.ldw, k0, kb, k0 + kb, n, 0, 1);
      LCK(gemm_update<T>(f.W + (size_t)(k0 + kb) * f.ldw + k0 + kb, f.ldw, f.W + (size_t)k0 * f.ldw + k0 + kb,
                         f.ldw, f.W + (size_t)(k0 + kb) * f.ldw + k0, f.ldw, rest, rest, kb, false, false,
                         f.fail + 1, f.gemm_mode, st, f.ozws));
    }
  }
  LCK(cudaGetLastError());
  k_build_perm<<<1, 32, 0, st>>>(f.piv, n, f.perm);
  int h[2], perr = 0;
  LCK(cudaMemcpyAsync(h, f.fail, sizeof(h), cudaMemcpyDeviceToHost, st));
  LCK(cudaMemcpyAsync(&perr, f.pb.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  LCK(cudaStreamSynchronize(st));
  if (h[1] || perr) return ASOLVE_E_TIMEOUT;
  *fail_out = h[0];
  return ASOLVE_OK;
}

double rcond_of(double anorm, double est) {
  if (anorm == 0.0 || std::isinf(est) || est == 0.0) return 0.0;
  return (1.0 / est) / anorm;
}

}  // namespace

// Workspace of the Ozaki-split products: trailing and TRSM updates (K = kLB)
// and the residuals with more than 8 right-hand sides (K = kOzResK).
size_t oz_ws_bytes(int64_t n, int64_t nrhs) {
  const size_t upd = gemm_oz_ws_bytes((int)n, (int)(n > nrhs ? n : nrhs), kLB);
  const size_t res = nrhs > 8 ? gemm_oz_ws_bytes((int)n, (int)nrhs, (int)std::min<int64_t>(n, kOzResK)) : 0;
  return upd > res ? upd : res;
}

size_t large_ws_bytes(int64_t n, int64_t nrhs) {
  const size_t ldw = (size_t)((n + 3) & ~3);
  size_t b = 0;
  b += sizeof(double) * ldw * n + 256;                 // working matrix (FP64 worst case)
  b += 2 * sizeof(int) * n + 512;                      // piv, perm
  b += 2 * sizeof(float) * (size_t)((n + kInvBW - 1) / kInvBW) * kInvBW * kInvBW + 512;  // diagonal-block inverses
  b += sizeof(double) * kLB * kLB + 256;               // Dtmp
  b += 4 * sizeof(double) * (size_t)n * nrhs + 1024;   // R, Xs, tmp, (spare)
  b += sizeof(double) * kResMaxSeg * 8 * (size_t)n + 256;  // residual partials
  b += 4 * sizeof(double) * (size_t)n + 512;           // estimator vectors
  b += 2 * sizeof(double) * 1024 * (kLB + 4) + 2 * sizeof(double) * kLB + 1024;  // panel buffers (G <= 1024)
  b += scan_large_workspace(n) + 4096;
  b += sizeof(int) * (size_t)(((n + 63) / 64) * ((nrhs + kWaveNR - 1) / kWaveNR)) + 1024;  // wave flags
  if (n <= kSvdLargeMax) b += large_svd_ws_bytes(n, nrhs) + 4096;  // SVD fallback (V, sigma, coefficients)
  b += sizeof(double) * (size_t)n * (kGmresM + 4) + sizeof(double) * (kGmresM + 2) + 2048;  // GMRES-IR
  b += oz_ws_bytes(n, nrhs) + 256;  // Ozaki-split FP64 updates and residuals
  return b + (1 << 20);
}

// The adaptive solve of one large system.  ws: device workspace of at least
// large_ws_bytes(n, nrhs).  Fills *info; returns the status.
int large_solve(const LargeArgs& a, void* ws, size_t ws_bytes, asolve_info* info) {
  cudaStream_t st = a.st;
  const int n = (int)a.n, nrhs = (int)a.nrhs;
  Arena ar{static_cast<char*>(ws), 0, ws_bytes};
  memset(info, 0, sizeof(*info));
  info->rcond = NAN;
  info->berr = NAN;
  info->svd_rank = -1;
  // the factor block comes first, at offsets that depend on n only, so that a
  // kept factorisation is found again by a later call with another nrhs
  const int ldw = (n + 3) & ~3;
  void* Wv = ar.take(sizeof(double) * (size_t)ldw * n);
  int* piv = static_cast<int*>(ar.take(sizeof(int) * (size_t)n));
  int* perm = static_cast<int*>(ar.take(sizeof(int) * (size_t)n));
  const size_t inv_elems = (size_t)((n + kInvBW - 1) / kInvBW) * kInvBW * kInvBW;
  float* dinvL = static_cast<float*>(ar.take(sizeof(float) * inv_elems));
  float* dinvU = static_cast<float*>(ar.take(sizeof(float) * inv_elems));
  if (!Wv || !piv || !perm || !dinvL || !dinvU) return ASOLVE_E_NOMEM;
  // the symmetric-indefinite route exists on the batched path only
  // (n <= 1024, nrhs <= 8); here it would silently become LU
  if ((a.flags & ASOLVE_SYM_INDEF) && n <= kBatchNMax) return info->status = ASOLVE_E_UNSUPPORTED;
  LargeReuse* kept = a.reuse;
  constexpr uint32_t kRouteFlags = ASOLVE_FORCE_LU | ASOLVE_FORCE_SVD | ASOLVE_NO_RCOND | ASOLVE_NO_APPROX |
                                   ASOLVE_TRIDIAG | ASOLVE_SYM_INDEF;
  const bool reuse_hit = kept && kept->valid && kept->A == a.A && kept->n == a.n &&
                         kept->flags == (a.flags & kRouteFlags) && kept->precision >= 0;
  if (kept && !reuse_hit) kept->valid = 0;
  // ---- scan (Sec. 2.1, 2.2, Fig. 4)
  void* sws = ar.take(scan_large_workspace(n));
  ScanRes* dsr = static_cast<ScanRes*>(ar.take(sizeof(ScanRes)));
  double* dscal = static_cast<double*>(ar.take(sizeof(double) * 32));  // estimator scalars and partials
  int* dint = static_cast<int*>(ar.take(sizeof(int) * 8));
  const int wcap = ((n + 63) / 64) * ((nrhs + kWaveNR - 1) / kWaveNR);
  int* wflags = static_cast<int*>(ar.take(sizeof(int) * (size_t)wcap));
  int* werr = static_cast<int*>(ar.take(sizeof(int) * 4));
  if (!sws || !dsr || !dscal || !dint || !wflags || !werr) return ASOLVE_E_NOMEM;
  LCK(cudaMemsetAsync(werr, 0, sizeof(int) * 4, st));
  const WaveBuf wb{wflags, werr, wcap, a.num_sms};
  // a device-side wait of a triangular solve gave up: the result is not valid
  auto wave_failed = [&]() -> bool {
    int h = 0;
    if (cudaMemcpyAsync(&h, werr, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return true;
    if (cudaStreamSynchronize(st) != cudaSuccess) return true;
    return h != 0;
  };
  ScanRes sr{};
  if (reuse_hit) {  // A is unchanged: its scan results come with the kept factor
    sr.kl = (int)kept->kl;
    sr.ku = (int)kept->ku;
    sr.cls = ASOLVE_CLS_GENERAL;  // a dense route follows
    sr.norm1 = kept->norm1;
    sr.norminf = kept->norminf;
  } else {
    LCK(launch_scan_large(a.A, n, a.B, (int64_t)n * nrhs, a.band_frac, a.sympd_tol, sws, dsr, a.num_sms, st));
    LCK(cudaMemcpyAsync(&sr, dsr, sizeof(sr), cudaMemcpyDeviceToHost, st));
    LCK(cudaStreamSynchronize(st));
  }
  info->cls = sr.cls;
  info->kl = sr.kl;
  info->ku = sr.ku;
  if (sr.flags & (SF_NONFINITE | SF_B_NONFINITE)) return info->status = ASOLVE_E_NONFINITE;
  // the SVD fallback of Sec. 2.5 (dense, one-sided Jacobi) up to kSvdLargeMax
  const bool svd_allowed = !(a.flags & ASOLVE_NO_APPROX) && n <= kSvdLargeMax;
  const bool force_svd = (a.flags & ASOLVE_FORCE_SVD) != 0;
  if (force_svd && n > kSvdLargeMax) return info->status = ASOLVE_E_UNSUPPORTED;
  int cls = (a.flags & ASOLVE_FORCE_LU || reuse_hit) ? ASOLVE_CLS_GENERAL : sr.cls;
  bool band_as_dense = false;
  bool band_pending = false;  // the band route asks for the SVD fallback
  if (cls == ASOLVE_CLS_BANDED && !force_svd) {
    // Sec. 2.1 banded route.  Bandwidths beyond the band kernels' windows run
    // the dense LU below, which makes the same pivot choices (the entries
    // outside the band stay exactly zero), and report the banded route.
    if (band_window_fits(sr.kl, sr.ku)) {
      const size_t need = band_ws_bytes(n, sr.kl, sr.ku, nrhs);
      void* bws = ar.take(need);
      if (!bws) return info->status = ASOLVE_E_NOMEM;
      BandArgs ba{nullptr, 0, 0, 0, a.A, a.B, a.X, n, nrhs, a.flags, a.rcond_threshold, sr.kl, sr.ku,
                  sr.norm1, sr.norminf, st};
      const int brc = band_solve(ba, bws, need, info);
      if (brc != ASOLVE_PENDING) return info->status;
      band_pending = true;  // solver failed or rcond below the threshold: SVD below
    } else {
      band_as_dense = true;
      cls = ASOLVE_CLS_GENERAL;
    }
  }
  // dynamic shared memory limits of every kernel below (the triangular
  // route uses the FP64 kernels even in mixed precision)
  int arc = set_large_attrs<float>();
  if (!arc) arc = set_large_attrs<double>();
  if (arc) return info->status = arc;
  const bool no_rcond = (a.flags & ASOLVE_NO_RCOND) != 0;
  double* R = static_cast<double*>(ar.take(sizeof(double) * (size_t)n * nrhs));
  double* Pres = static_cast<double*>(ar.take(sizeof(double) * kResMaxSeg * 8 * (size_t)n));  // residual partials
  void* xs = ar.take(sizeof(double) * (size_t)n * nrhs);
  void* tmp = ar.take(sizeof(double) * (size_t)n * nrhs);
  void* ev = ar.take(sizeof(double) * (size_t)n);
  void* exi = ar.take(sizeof(double) * (size_t)n);
  unsigned long long* colmax = static_cast<unsigned long long*>(ar.take(sizeof(unsigned long long) * 3 * nrhs));
  if (!R || !Pres || !xs || !tmp || !ev || !exi || !colmax) return ASOLVE_E_NOMEM;
  // FP64 updates as Ozaki-split tensor products in every mode but the plain
  // FP64 one (which keeps the mma.sync f64 GEMM)
  void* ozws = a.precision != ASOLVE_PREC_FP64 ? ar.take(oz_ws_bytes(n, nrhs)) : nullptr;
  // FP64 normwise backward error of X, the maximum over the columns
  auto backward_error = [&](double& be) -> int {
    LCK(cudaMemsetAsync(colmax, 0, sizeof(unsigned long long) * 3 * nrhs, st));
    {
      const int rr_ = residual_large(a.A, n, a.B, a.X, nrhs, R, colmax, Pres, a.num_sms, st, ozws, werr);
      if (rr_) return rr_;
    }
    k_colmax_abs<double><<<dim3(64, nrhs), 256, 0, st>>>(a.X, n, nrhs, colmax + nrhs);
    k_colmax_abs<double><<<dim3(64, nrhs), 256, 0, st>>>(a.B, n, nrhs, colmax + 2 * nrhs);
    std::vector<unsigned long long> hm((size_t)3 * nrhs);
    LCK(cudaMemcpyAsync(hm.data(), colmax, sizeof(unsigned long long) * 3 * nrhs, cudaMemcpyDeviceToHost, st));
    LCK(cudaStreamSynchronize(st));
    be = 0.0;
    for (int c = 0; c < nrhs; ++c) {
      double rm, xm, bm;
      memcpy(&rm, &hm[c], 8);
      memcpy(&xm, &hm[nrhs + c], 8);
      memcpy(&bm, &hm[2 * nrhs + c], 8);
      const double den = sr.norminf * xm + bm;
      const double b1 = den > 0.0 ? rm / den : (rm > 0.0 ? INFINITY : 0.0);
      if (!(b1 <= be)) be = b1;
    }
    return ASOLVE_OK;
  };
  // Sec. 2.5: the routed solver failed, its rcond is below the threshold,
  // or FORCE_SVD: X is the minimum-norm solution through the SVD of A.  The
  // working matrix W (factors no longer needed) becomes the SVD's G; the
  // route and rcond already in info stay (the primary solver's).
  auto svd_fallback = [&]() -> int {
    if (kept) kept->valid = 0;
    void* vws = ar.take(large_svd_ws_bytes(n, nrhs));
    if (!vws) return info->status = ASOLVE_E_NOMEM;
    int64_t rank = 0;
    int sweeps = 0;
    const int r2 = large_svd(a.A, n, a.B, a.X, nrhs, a.svd_trunc_rel, static_cast<double*>(Wv), vws, &rank,
                             &sweeps, st);
    if (r2) return info->status = r2;
    info->svd_rank = rank;
    info->precision = ASOLVE_PREC_FP64;
    if (a.flags & ASOLVE_BERR) {
      double be;
      const int r3 = backward_error(be);
      if (r3) return info->status = r3;
      info->berr = be;
    }
    LCK(cudaStreamSynchronize(st));
    return info->status = ASOLVE_W_APPROX;
  };
  if (force_svd) {
    info->route = ASOLVE_ROUTE_SVD;
    info->precision = ASOLVE_PREC_FP64;
    return svd_fallback();
  }
  if (band_pending) return svd_fallback();
  // ---- triangular route (Sec. 2.2): FP64 substitution on A itself
  if (cls == ASOLVE_CLS_LOWER || cls == ASOLVE_CLS_UPPER) {
    const bool lower = cls == ASOLVE_CLS_LOWER;
    info->route = lower ? ASOLVE_ROUTE_TRI_LOWER : ASOLVE_ROUTE_TRI_UPPER;
    info->precision = ASOLVE_PREC_FP64;
    // singular iff some A_ii == 0 (the scan's diagonal is not kept: check here)
    LCK(cudaMemsetAsync(dint, 0, sizeof(int), st));
    {
      std::vector<double> diag((size_t)n);
      LCK(cudaMemcpy2DAsync(diag.data(), sizeof(double), a.A, sizeof(double) * (n + 1), sizeof(double), n,
                            cudaMemcpyDeviceToHost, st));
      LCK(cudaStreamSynchronize(st));
      for (int i = 0; i < n; ++i)
        if (diag[(size_t)i] == 0.0) {  // the substitution fails (Sec. 2.2)
          if (svd_allowed) return svd_fallback();
          LCK(cudaMemsetAsync(a.X, 0, sizeof(double) * (size_t)n * nrhs, st));
          LCK(cudaStreamSynchronize(st));
          return info->status = ASOLVE_E_SINGULAR;
        }
    }
    LCK(cudaMemcpyAsync(a.X, a.B, sizeof(double) * (size_t)n * nrhs, cudaMemcpyDeviceToDevice, st));
    int rc;
    if (nrhs >= kTrsmBlockedRhs) {
      // many right-hand sides: blocked TRSM, diagonal blocks by substitution,
      // the rest of the right-hand sides updated by the Ozaki-split product
      // (the mma.sync f64 GEMM in the plain FP64 mode)
      if (ozws) info->detail |= 64;
      const unsigned gr = (unsigned)((nrhs + 63) / 64);
      for (int q = 0; q < n; q += kLB) {
        const int k0 = lower ? q : ((n - 1 - q) / kLB) * kLB;
        const int kb = std::min(kLB, n - k0);
        k_trsm_rhs<<<gr, kThreads, trsm_smem<double>(), st>>>(a.A, n, k0, kb, a.X, n, nrhs, lower ? 0 : 1);
        if (lower && k0 + kb < n)
          LCK(gemm_update<double>(a.X + k0 + kb, n, a.A + (size_t)k0 * n + k0 + kb, n, a.X + k0, n, n - k0 - kb, nrhs,
                                  kb, false, false, werr, 0, st, ozws));
        if (!lower && k0 > 0)
          LCK(gemm_update<double>(a.X, n, a.A + (size_t)k0 * n, n, a.X + k0, n, k0, nrhs, kb, false, false, werr, 0,
                                  st, ozws));
      }
      LCK(cudaGetLastError());
    } else if ((rc = tri_solve_large<double>(a.A, n, n, lower, false, false, a.X, nrhs, false, wb, st))) {
      return rc;
    }
    double rc_val = NAN;
    if (!no_rcond) {
      double est;
      auto apply = [&](double* v, bool tr) { return tri_solve_large<double>(a.A, n, n, lower, tr, false, v, 1, false, wb, st); };
      rc = est_host<double>(n, (double*)ev, (double*)exi, dscal, dint, apply, st, &est);
      if (rc) return rc;
      rc_val = rcond_of(sr.norm1, est);
    }
    info->rcond = rc_val;
    if (a.flags & ASOLVE_BERR) {
      LCK(cudaMemsetAsync(colmax, 0, sizeof(unsigned long long) * 3 * nrhs, st));
      {
        const int rr_ = residual_large(a.A, n, a.B, a.X, nrhs, R, colmax, Pres, a.num_sms, st, ozws, werr);
        if (rr_) return rr_;
      }
      k_colmax_abs<double><<<dim3(64, nrhs), 256, 0, st>>>(a.X, n, nrhs, colmax + nrhs);
      k_colmax_abs<double><<<dim3(64, nrhs), 256, 0, st>>>(a.B, n, nrhs, colmax + 2 * nrhs);
      std::vector<unsigned long long> hm((size_t)3 * nrhs);
      LCK(cudaMemcpyAsync(hm.data(), colmax, sizeof(unsigned long long) * 3 * nrhs, cudaMemcpyDeviceToHost, st));
      LCK(cudaStreamSynchronize(st));
      double be = 0.0;
      for (int c = 0; c < nrhs; ++c) {
        double rm, xm, bm;
        memcpy(&rm, &hm[c], 8);
        memcpy(&xm, &hm[nrhs + c], 8);
        memcpy(&bm, &hm[2 * nrhs + c], 8);
        const double den = sr.norminf * xm + bm;
        const double b1 = den > 0.0 ? rm / den : (rm > 0.0 ? INFINITY : 0.0);
        if (!(b1 <= be)) be = b1;
      }
      info->berr = be;
    }
    if (wave_failed()) return info->status = ASOLVE_E_TIMEOUT;
    const bool poor = !no_rcond && !(rc_val >= a.rcond_threshold);
    if (poor && svd_allowed) return svd_fallback();
    info->status = poor ? ASOLVE_W_ILLCOND : ASOLVE_OK;
    return info->status;
  }
  // ---- dense routes: Cholesky (Sec. 2.3) or LU (Sec. 2.4)
  int* fail = static_cast<int*>(ar.take(sizeof(int) * 4));
  void* Dtmp = ar.take(sizeof(double) * kLB * kLB);
  void* pcand = ar.take(sizeof(double) * 2 * a.num_sms * 4);
  void* prows = ar.take(sizeof(double) * 2 * a.num_sms * kLB);
  void* pdiag = ar.take(sizeof(double) * 2 * kLB);
  unsigned* pbar = static_cast<unsigned*>(ar.take(sizeof(unsigned) * 4));
  int* perr = static_cast<int*>(ar.take(sizeof(int) * 4));
  unsigned long long* pkey = static_cast<unsigned long long*>(ar.take(sizeof(unsigned long long) * 4));
  if (!fail || !Dtmp || !pcand || !prows || !pdiag || !pbar || !perr || !pkey) return ASOLVE_E_NOMEM;
  LCK(cudaMemsetAsync(perr, 0, sizeof(int) * 4, st));
  PanelBuf pb{pcand, prows, pdiag, pbar, perr, pkey};
  bool chol = (cls == ASOLVE_CLS_SYMPD);
  info->route = chol ? ASOLVE_ROUTE_CHOL : ASOLVE_ROUTE_LU;
  int detail = 0;
  int rc;
  // refinement with FP32 factors: x0 = inv(A32) b; loop r = b - A x (FP64),
  // x += inv(A32) r.  Returns 1 converged, 0 stalled, < 0 error.
  auto mixed_ir = [&](Fac<float>& f, bool lu, int& iters, double& berr) -> int {
    std::vector<unsigned long long> hm((size_t)3 * nrhs);
    std::vector<double> scale((size_t)nrhs);
    double* dscale = static_cast<double*>(ev);  // reuse (n >= nrhs)
    LCK(cudaMemsetAsync(colmax, 0, sizeof(unsigned long long) * 3 * nrhs, st));
    k_colmax_abs<double><<<dim3(64, nrhs), 256, 0, st>>>(a.B, n, nrhs, colmax + 2 * nrhs);
    LCK(cudaMemcpyAsync(hm.data(), colmax, sizeof(unsigned long long) * 3 * nrhs, cudaMemcpyDeviceToHost, st));
    LCK(cudaStreamSynchronize(st));
    std::vector<double> bmax((size_t)nrhs);
    for (int c = 0; c < nrhs; ++c) {
      memcpy(&bmax[c], &hm[2 * nrhs + c], 8);
      if (!(bmax[c] <= DBL_MAX)) return ASOLVE_E_NONFINITE;
      scale[c] = bmax[c] > 0.0 ? bmax[c] : 1.0;
    }
    LCK(cudaMemcpyAsync(dscale, scale.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, st));
    k_scale_down<float><<<1024, 256, 0, st>>>(a.B, n, nrhs, dscale, (float*)xs);
    int r2 = apply_large<float, float>(f, lu, n, (float*)xs, nrhs, false, (float*)tmp, st);
    if (r2) return r2;
    k_scale_add<float><<<1024, 256, 0, st>>>(a.X, n, nrhs, dscale, (float*)xs, 1);
    double berr_prev = INFINITY;
    berr = INFINITY;
    iters = 0;
    int ok = 0;
    for (int it = 0;; ++it) {
      LCK(cudaMemsetAsync(colmax, 0, sizeof(unsigned long long) * 2 * nrhs, st));
      {
        const int rr_ = residual_large(a.A, n, a.B, a.X, nrhs, R, colmax, Pres, a.num_sms, st, ozws, werr);
        if (rr_) return rr_;
      }
      k_colmax_abs<double><<<dim3(64, nrhs), 256, 0, st>>>(a.X, n, nrhs, colmax + nrhs);
      LCK(cudaMemcpyAsync(hm.data(), colmax, sizeof(unsigned long long) * 2 * nrhs, cudaMemcpyDeviceToHost, st));
      LCK(cudaStreamSynchronize(st));
      berr = 0.0;
      for (int c = 0; c < nrhs; ++c) {
        double rm, xm;
        memcpy(&rm, &hm[c], 8);
        memcpy(&xm, &hm[nrhs + c], 8);
        const double den = sr.norminf * xm + bmax[c];
        const double b1 = den > 0.0 ? rm / den : (rm > 0.0 ? INFINITY : 0.0);
        if (!(b1 <= berr)) berr = b1;
        scale[c] = rm > 0.0 ? rm : 1.0;
      }
      const bool conv = berr <= a.ir_target_berr;
      if (!conv && (it >= a.ir_max_iter || !(berr < 0.5 * berr_prev))) break;
      berr_prev = berr;
      LCK(cudaMemcpyAsync(dscale, scale.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, st));
      k_scale_down<float><<<1024, 256, 0, st>>>(R, n, nrhs, dscale, (float*)xs);
      if ((r2 = apply_large<float, float>(f, lu, n, (float*)xs, nrhs, false, (float*)tmp, st))) return r2;
      k_scale_add<float><<<1024, 256, 0, st>>>(a.X, n, nrhs, dscale, (float*)xs, 0);
      ++iters;
      if (conv) { ok = 1; break; }
    }
    LCK(cudaStreamSynchronize(st));
    return ok;
  };
  // GMRES-IR (Carson & Higham): the correction solve A d = r of each
  // refinement step is GMRES in FP64 on inv(M) A d = inv(M) r, M the
  // low-precision factors applied in FP32 (left preconditioning), a Krylov
  // basis of at most kGmresM vectors, classical Gram-Schmidt done twice,
  // Givens rotations on the host's small Hessenberg matrix; one inner solve
  // per right-hand side and step.  Returns 1 converged, 0 stalled, < 0 error;
  // *inner: the inner iterations (products with A) over all steps.
  double* gV = static_cast<double*>(ar.take(sizeof(double) * (size_t)n * (kGmresM + 1)));
  double* gw = static_cast<double*>(ar.take(sizeof(double) * (size_t)n));
  double* gt = static_cast<double*>(ar.take(sizeof(double) * (size_t)n));
  double* gzero = static_cast<double*>(ar.take(sizeof(double) * (size_t)n));
  double* gh = static_cast<double*>(ar.take(sizeof(double) * (kGmresM + 2)));
  if (!gV || !gw || !gt || !gzero || !gh) return ASOLVE_E_NOMEM;
  auto gmres_ir = [&](Fac<float>& f, bool lu, int& iters, int& inner, double& berr) -> int {
    const unsigned gv = (unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
    float* xf = static_cast<float*>(xs);
    float* tf = static_cast<float*>(tmp);
    const double anrm = sr.norminf > 0.0 ? sr.norminf : 1.0;
    std::vector<double> H((size_t)(kGmresM + 1) * kGmresM), cs(kGmresM), sn(kGmresM), g(kGmresM + 1),
        hv(kGmresM + 1), y(kGmresM);
    LCK(cudaMemsetAsync(gzero, 0, sizeof(double) * (size_t)n, st));
    // out = s_out * inv(M) (v / s_in): v in FP64, brought into FP32 range by
    // s_in (a power-of-two-free scale; the product with s_out undoes it)
    auto precond = [&](const double* v, double s_in, double s_out, double* out) -> int {
      k_vec_to_f32<<<gv, 256, 0, st>>>(v, n, 1.0 / s_in, xf);
      const int r2 = apply_large<float, float>(f, lu, n, xf, 1, false, tf, st);
      if (r2) return r2;
      k_vec_from_f32<<<gv, 256, 0, st>>>(xf, n, s_out, out);
      return ASOLVE_OK;
    };
    auto dots = [&](const double* V, int m, const double* w, double* hh) -> int {
      k_krylov_dots<<<m, 256, 0, st>>>(V, n, n, m, w, gh);
      LCK(cudaMemcpyAsync(hh, gh, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
      LCK(cudaStreamSynchronize(st));
      return ASOLVE_OK;
    };
    // one inner GMRES solve for column c of R (max |r| = rm); d added to X
    auto solve_col = [&](int c, double rm) -> int {
      int r2;
      const double rs = rm > 0.0 ? rm : 1.0;
      if ((r2 = precond(R + (size_t)c * n, rs, rs, gw))) return r2;
      double nb;
      if ((r2 = dots(gw, 1, gw, &nb))) return r2;
      const double beta = sqrt(nb);
      if (!(beta > 0.0) || !(beta <= DBL_MAX)) return ASOLVE_OK;
      k_vec_scale<<<gv, 256, 0, st>>>(gV, gw, n, 1.0 / beta);
      std::fill(g.begin(), g.end(), 0.0);
      g[0] = beta;
      int k = 0;
      for (int j = 0; j < kGmresM; ++j) {
        double* vj = gV + (size_t)j * n;
        // w = inv(M) A v_j: the residual kernel gives t = 0 - A v_j
        LCK(cudaMemsetAsync(colmax, 0, sizeof(unsigned long long) * 2, st));
        if ((r2 = residual_large(a.A, n, gzero, vj, 1, gt, colmax, Pres, a.num_sms, st))) return r2;
        if ((r2 = precond(gt, anrm, -anrm, gw))) return r2;  // w = inv(M) A v_j
        // classical Gram-Schmidt, twice
        if ((r2 = dots(gV, j + 1, gw, hv.data()))) return r2;
        LCK(cudaMemcpyAsync(gh, hv.data(), sizeof(double) * (j + 1), cudaMemcpyHostToDevice, st));
        k_krylov_comb<<<gv, 256, 0, st>>>(gw, gV, n, n, j + 1, gh, -1.0);
        std::vector<double> h2((size_t)j + 1);
        if ((r2 = dots(gV, j + 1, gw, h2.data()))) return r2;
        LCK(cudaMemcpyAsync(gh, h2.data(), sizeof(double) * (j + 1), cudaMemcpyHostToDevice, st));
        k_krylov_comb<<<gv, 256, 0, st>>>(gw, gV, n, n, j + 1, gh, -1.0);
        for (int i = 0; i <= j; ++i) hv[i] += h2[i];
        double hn2;
        if ((r2 = dots(gw, 1, gw, &hn2))) return r2;
        const double hn = sqrt(hn2);
        if (!(hn <= DBL_MAX)) return ASOLVE_OK;  // NaN/Inf: give up this inner solve
        // Hessenberg column j, previous rotations, then a new one
        for (int i = 0; i <= j; ++i) H[(size_t)j * (kGmresM + 1) + i] = hv[i];
        H[(size_t)j * (kGmresM + 1) + j + 1] = hn;
        double* hc = &H[(size_t)j * (kGmresM + 1)];
        for (int i = 0; i < j; ++i) {
          const double t0 = cs[i] * hc[i] + sn[i] * hc[i + 1];
          hc[i + 1] = -sn[i] * hc[i] + cs[i] * hc[i + 1];
          hc[i] = t0;
        }
        const double rr = hypot(hc[j], hc[j + 1]);
        cs[j] = rr > 0.0 ? hc[j] / rr : 1.0;
        sn[j] = rr > 0.0 ? hc[j + 1] / rr : 0.0;
        hc[j] = rr;
        hc[j + 1] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        k = j + 1;
        ++inner;
        if (!(fabs(g[j + 1]) > kGmresTol * beta) || !(hn > 0.0)) break;
        k_vec_scale<<<gv, 256, 0, st>>>(gV + (size_t)(j + 1) * n, gw, n, 1.0 / hn);
      }
      // y = H(0:k, 0:k) \ g(0:k), then X(:, c) += V y
      for (int i = k - 1; i >= 0; --i) {
        double t0 = g[i];
        for (int q = i + 1; q < k; ++q) t0 -= H[(size_t)q * (kGmresM + 1) + i] * y[q];
        y[i] = H[(size_t)i * (kGmresM + 1) + i] != 0.0 ? t0 / H[(size_t)i * (kGmresM + 1) + i] : 0.0;
      }
      LCK(cudaMemcpyAsync(gh, y.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st));
      k_krylov_comb<<<gv, 256, 0, st>>>(a.X + (size_t)c * n, gV, n, n, k, gh, 1.0);
      LCK(cudaStreamSynchronize(st));
      return ASOLVE_OK;
    };
    std::vector<unsigned long long> hm((size_t)3 * nrhs);
    std::vector<double> bmax((size_t)nrhs);
    LCK(cudaMemsetAsync(colmax, 0, sizeof(unsigned long long) * 3 * nrhs, st));
    k_colmax_abs<double><<<dim3(64, nrhs), 256, 0, st>>>(a.B, n, nrhs, colmax + 2 * nrhs);
    LCK(cudaMemcpyAsync(hm.data(), colmax, sizeof(unsigned long long) * 3 * nrhs, cudaMemcpyDeviceToHost, st));
    LCK(cudaStreamSynchronize(st));
    for (int c = 0; c < nrhs; ++c) {
      memcpy(&bmax[c], &hm[2 * nrhs + c], 8);
      if (!(bmax[c] <= DBL_MAX)) return ASOLVE_E_NONFINITE;
    }
    // x0 = 0: the first step solves A d = b
    LCK(cudaMemsetAsync(a.X, 0, sizeof(double) * (size_t)n * nrhs, st));
    double berr_prev = INFINITY;
    berr = INFINITY;
    iters = 0;
    inner = 0;
    for (int it = 0;; ++it) {
      LCK(cudaMemsetAsync(colmax, 0, sizeof(unsigned long long) * 2 * nrhs, st));
      {
        const int rr_ = residual_large(a.A, n, a.B, a.X, nrhs, R, colmax, Pres, a.num_sms, st, ozws, werr);
        if (rr_) return rr_;
      }
      k_colmax_abs<double><<<dim3(64, nrhs), 256, 0, st>>>(a.X, n, nrhs, colmax + nrhs);
      LCK(cudaMemcpyAsync(hm.data(), colmax, sizeof(unsigned long long) * 2 * nrhs, cudaMemcpyDeviceToHost, st));
      LCK(cudaStreamSynchronize(st));
      berr = 0.0;
      std::vector<double> rmax((size_t)nrhs);
      for (int c = 0; c < nrhs; ++c) {
        double xm;
        memcpy(&rmax[c], &hm[c], 8);
        memcpy(&xm, &hm[nrhs + c], 8);
        const double den = sr.norminf * xm + bmax[c];
        const double b1 = den > 0.0 ? rmax[c] / den : (rmax[c] > 0.0 ? INFINITY : 0.0);
        if (!(b1 <= berr)) berr = b1;
      }
      if (berr <= a.ir_target_berr) return 1;
      if (it >= a.ir_max_iter || !(berr < 0.5 * berr_prev)) return 0;  // stalled
      berr_prev = berr;
      for (int c = 0; c < nrhs; ++c) {
        const int r2 = solve_col(c, rmax[c]);
        if (r2) return r2;
      }
      ++iters;
    }
  };
  // the kept factorisation fills the fields of a later call's info
  auto keep = [&](int precision, bool lu) {
    if (!kept) return;
    kept->valid = 1;
    kept->A = a.A;
    kept->n = a.n;
    kept->flags = a.flags & kRouteFlags;
    kept->cls = info->cls;
    kept->route = info->route;
    kept->precision = precision;
    kept->lu = lu ? 1 : 0;
    kept->detail = info->detail;
    kept->kl = info->kl;
    kept->ku = info->ku;
    kept->rcond = info->rcond;
    kept->norm1 = sr.norm1;
    kept->norminf = sr.norminf;
  };
  if (reuse_hit) {
    info->cls = kept->cls;
    info->route = kept->route;
    info->rcond = kept->rcond;
    info->precision = kept->precision;
    info->detail = kept->detail | 8;
    if (kept->precision != ASOLVE_PREC_FP64) {  // FP32-stored factors
      if ((rc = set_large_attrs<float>())) return rc;
      Fac<float> f{static_cast<float*>(Wv), ldw, piv, perm, static_cast<float*>(Dtmp), fail, pb, wb};
      f.dinvL = dinvL;  // kept with the factor (they follow it in the workspace)
      f.dinvU = kept->lu ? dinvU : nullptr;
      int iters = 0;
      double berr = NAN;
      const int ok = mixed_ir(f, kept->lu != 0, iters, berr);
      if (ok < 0) return info->status = ok;
      if (ok == 1) {
        info->berr = berr;
        info->ir_iters = iters;
        if (wave_failed()) return info->status = ASOLVE_E_TIMEOUT;
        return info->status = ASOLVE_OK;
      }
      kept->valid = 0;  // the kept factor does not refine this right-hand side: start over
      return large_solve(a, ws, ws_bytes, info);
    }
    Fac<double> f{static_cast<double*>(Wv), ldw, piv, perm, static_cast<double*>(Dtmp), fail, pb, wb};
    LCK(cudaMemsetAsync(colmax, 0, sizeof(unsigned long long) * 3 * nrhs, st));
    k_colmax_abs<double><<<dim3(64, nrhs), 256, 0, st>>>(a.B, n, nrhs, colmax + 2 * nrhs);
    std::vector<unsigned long long> hb((size_t)3 * nrhs);
    LCK(cudaMemcpyAsync(hb.data(), colmax, sizeof(unsigned long long) * 3 * nrhs, cudaMemcpyDeviceToHost, st));
    LCK(cudaStreamSynchronize(st));
    for (int c = 0; c < nrhs; ++c) {
      double bm;
      memcpy(&bm, &hb[2 * nrhs + c], 8);
      if (!(bm <= DBL_MAX)) return info->status = ASOLVE_E_NONFINITE;
    }
    LCK(cudaMemcpyAsync(a.X, a.B, sizeof(double) * (size_t)n * nrhs, cudaMemcpyDeviceToDevice, st));
    if ((rc = apply_large<double, double>(f, kept->lu != 0, n, a.X, nrhs, false, (double*)tmp, st))) return rc;
    if (a.flags & ASOLVE_BERR) {
      LCK(cudaMemsetAsync(colmax, 0, sizeof(unsigned long long) * 2 * nrhs, st));
      {
        const int rr_ = residual_large(a.A, n, a.B, a.X, nrhs, R, colmax, Pres, a.num_sms, st, ozws, werr);
        if (rr_) return rr_;
      }
      k_colmax_abs<double><<<dim3(64, nrhs), 256, 0, st>>>(a.X, n, nrhs, colmax + nrhs);
      LCK(cudaMemcpyAsync(hb.data(), colmax, sizeof(unsigned long long) * 3 * nrhs, cudaMemcpyDeviceToHost, st));
      LCK(cudaStreamSynchronize(st));
      double be = 0.0;
      for (int c = 0; c < nrhs; ++c) {
        double rm, xm, bm;
        memcpy(&rm, &hb[c], 8);
        memcpy(&xm, &hb[nrhs + c], 8);
        memcpy(&bm, &hb[2 * nrhs + c], 8);
        const double den = sr.norminf * xm + bm;
        const double b1 = den > 0.0 ? rm / den : (rm > 0.0 ? INFINITY : 0.0);
        if (!(b1 <= be)) be = b1;
      }
      info->berr = be;
    }
    LCK(cudaStreamSynchronize(st));
    if (wave_failed()) return info->status = ASOLVE_E_TIMEOUT;
    const bool poor = !no_rcond && !(kept->rcond >= a.rcond_threshold);
    if (poor && svd_allowed) return svd_fallback();
    return info->status = poor ? ASOLVE_W_ILLCOND : ASOLVE_OK;
  }
  // ---- mixed precision: FP32 factors (trailing updates as 3xTF32, BF16 or
  // FP16 tensor products), FP64 refinement
  if (a.precision != ASOLVE_PREC_FP64 && a.precision != ASOLVE_PREC_FP64_OZ && !(sr.flags & SF_NORM_FP64)) {
    if ((rc = set_large_attrs<float>())) return rc;
    Fac<float> f{static_cast<float*>(Wv), ldw, piv, perm, static_cast<float*>(Dtmp), fail, pb, wb};
    f.gemm_mode = a.precision == ASOLVE_PREC_BF16   ? kGemmBf16
                  : a.precision == ASOLVE_PREC_FP16 ? kGemmFp16
                  : a.precision == ASOLVE_PREC_FP8  ? kGemmFp8
                                                    : 3;
    // the refinement converges while kappa times the factors' relative
    // error stays below one: the 16-bit updates lower the kappa limit
    const double klim = a.precision == ASOLVE_PREC_BF16   ? fmin(a.ir_kappa_limit, kKappaLimitBf16)
                        : a.precision == ASOLVE_PREC_FP16 ? fmin(a.ir_kappa_limit, kKappaLimitFp16)
                        : a.precision == ASOLVE_PREC_FP8  ? fmin(a.ir_kappa_limit, kKappaLimitFp8)
                                                          : a.ir_kappa_limit;
    for (int attempt = 0; attempt < 2; ++attempt) {
      const bool try_chol = chol && attempt == 0;
      if (!chol && attempt == 1) break;
      k_to_work<float><<<a.num_sms * 4, 256, 0, st>>>(a.A, n, f.W, ldw);
      int fcol = 0;
      rc = try_chol ? chol_large<float>(f, n, a.num_sms, &fcol, st) : lu_large<float>(f, n, a.num_sms, &fcol, st);
      if (rc) return rc;
      if (fcol) {
        if (try_chol) detail |= 4;
        break;  // FP32 factorisation failed: FP64 path decides
      }
      const bool lu = !try_chol;
      // inverses of the diagonal blocks for the wavefront solves
      k_diag_inv<<<(n + kInvBW - 1) / kInvBW, kThreads, kDiagInvSmem, st>>>(f.W, ldw, n, lu ? 1 : 0, dinvL,
                                                                            lu ? dinvU : nullptr);
      LCK(cudaGetLastError());
      f.dinvL = dinvL;
      f.dinvU = lu ? dinvU : nullptr;
      double rcv = NAN;
      bool gate_ok = true;
      // the 16-bit modes also have GMRES-IR, which reaches much larger kappa
      const bool sixteen =
          a.precision == ASOLVE_PREC_BF16 || a.precision == ASOLVE_PREC_FP16 || a.precision == ASOLVE_PREC_FP8;
      const double klim_gm = a.precision == ASOLVE_PREC_BF16   ? kKappaLimitGmresBf16
                             : a.precision == ASOLVE_PREC_FP16 ? kKappaLimitGmresFp16
                                                               : kKappaLimitGmresFp8;
      bool gm_ok = sixteen;
      if (!no_rcond) {
        double est;
        auto apply = [&](float* v, bool tr) { return apply_large<float, float>(f, lu, n, v, 1, tr, (float*)tmp, st); };
        rc = est_host<float>(n, (float*)ev, (float*)exi, dscal, dint, apply, st, &est);
        if (rc) return rc;
        rcv = rcond_of(sr.norm1, est);
        gate_ok = rcv >= 1.0 / klim;
        gm_ok = sixteen && rcv >= 1.0 / fmin(a.ir_kappa_limit, klim_gm);
      }
      if (!gate_ok && !gm_ok) { detail |= 1; break; }
      int iters = 0;
      double berr = NAN;
      int okc = 0;
      if (gate_ok) {  // classical refinement first
        okc = mixed_ir(f, lu, iters, berr);
        if (okc < 0) return info->status = okc;
      }
      if (okc == 0 && gm_ok) {  // beyond its kappa limit, or stalled: GMRES-IR
        int it2 = 0, inner = 0;
        okc = gmres_ir(f, lu, it2, inner, berr);
        if (okc < 0) return info->status = okc;
        iters += it2;
        if (okc == 1) detail |= 32;
      }
      const bool ok = okc == 1;
      if (ok) {
        info->route = try_chol ? ASOLVE_ROUTE_CHOL : (chol ? ASOLVE_ROUTE_CHOL_FAIL_LU : ASOLVE_ROUTE_LU);
        if (band_as_dense) info->route = ASOLVE_ROUTE_BAND_LU;
        info->rcond = rcv;
        info->berr = berr;
        info->ir_iters = iters;
        info->precision = a.precision;
        info->detail = detail;
        if (wave_failed()) return info->status = ASOLVE_E_TIMEOUT;
        keep(a.precision, lu);
        return info->status = ASOLVE_OK;
      }
      detail |= 2;
      break;
    }
  }
  // ---- FP64 path
  if ((rc = set_large_attrs<double>())) return rc;
  Fac<double> f{static_cast<double*>(Wv), ldw, piv, perm, static_cast<double*>(Dtmp), fail, pb, wb};
  f.ozws = ozws;
  if (ozws) detail |= 64;
  info->precision = ASOLVE_PREC_FP64;
  info->detail = detail;
  bool lu = !chol;
  int fcol = 0;
  if (chol) {
    k_to_work<double><<<a.num_sms * 4, 256, 0, st>>>(a.A, n, f.W, ldw);
    if ((rc = chol_large<double>(f, n, a.num_sms, &fcol, st))) return rc;
    if (fcol) {  // not sympd after all (Sec. 2.3): the general solver
      lu = true;
      info->route = ASOLVE_ROUTE_CHOL_FAIL_LU;
    }
  }
  if (lu) {
    k_to_work<double><<<a.num_sms * 4, 256, 0, st>>>(a.A, n, f.W, ldw);
    fcol = 0;
    if ((rc = lu_large<double>(f, n, a.num_sms, &fcol, st))) return rc;
  }
  if (band_as_dense) info->route = ASOLVE_ROUTE_BAND_LU;
  if (fcol) {  // the factorisation failed (an exact zero pivot)
    if (svd_allowed) return svd_fallback();
    LCK(cudaMemsetAsync(a.X, 0, sizeof(double) * (size_t)n * nrhs, st));
    LCK(cudaStreamSynchronize(st));
    return info->status = ASOLVE_E_SINGULAR;
  }
  LCK(cudaMemcpyAsync(a.X, a.B, sizeof(double) * (size_t)n * nrhs, cudaMemcpyDeviceToDevice, st));
  if ((rc = apply_large<double, double>(f, lu, n, a.X, nrhs, false, (double*)tmp, st))) return rc;
  double rcv = NAN;
  if (!no_rcond) {
    double est;
    auto apply = [&](double* v, bool tr) { return apply_large<double, double>(f, lu, n, v, 1, tr, (double*)tmp, st); };
    if ((rc = est_host<double>(n, (double*)ev, (double*)exi, dscal, dint, apply, st, &est))) return rc;
    rcv = rcond_of(sr.norm1, est);
  }
  info->rcond = rcv;
  if (a.flags & ASOLVE_BERR) {
    LCK(cudaMemsetAsync(colmax, 0, sizeof(unsigned long long) * 3 * nrhs, st));
    {
        const int rr_ = residual_large(a.A, n, a.B, a.X, nrhs, R, colmax, Pres, a.num_sms, st, ozws, werr);
        if (rr_) return rr_;
      }
    k_colmax_abs<double><<<dim3(64, nrhs), 256, 0, st>>>(a.X, n, nrhs, colmax + nrhs);
    k_colmax_abs<double><<<dim3(64, nrhs), 256, 0, st>>>(a.B, n, nrhs, colmax + 2 * nrhs);
    std::vector<unsigned long long> hm((size_t)3 * nrhs);
    LCK(cudaMemcpyAsync(hm.data(), colmax, sizeof(unsigned long long) * 3 * nrhs, cudaMemcpyDeviceToHost, st));
    LCK(cudaStreamSynchronize(st));
    double be = 0.0;
    for (int c = 0; c < nrhs; ++c) {
      double rm, xm, bm;
      memcpy(&rm, &hm[c], 8);
      memcpy(&xm, &hm[nrhs + c], 8);
      memcpy(&bm, &hm[2 * nrhs + c], 8);
      const double den = sr.norminf * xm + bm;
      const double b1 = den > 0.0 ? rm / den : (rm > 0.0 ? INFINITY : 0.0);
      if (!(b1 <= be)) be = b1;
    }
    info->berr = be;
  }
  LCK(cudaStreamSynchronize(st));
  if (wave_failed()) return info->status = ASOLVE_E_TIMEOUT;
  const bool poor = !no_rcond && !(rcv >= a.rcond_threshold);
  if (poor && svd_allowed) return svd_fallback();
  keep(ASOLVE_PREC_FP64, lu);
  return info->status = poor ? ASOLVE_W_ILLCOND : ASOLVE_OK;
}

}  // namespace asv
