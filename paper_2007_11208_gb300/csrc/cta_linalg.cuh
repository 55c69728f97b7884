// cta_linalg.cuh -- dense linear algebra performed by ONE thread block on one
// system (n <= 1024): the building blocks of the class-routed batched path.
//
//   cta_lu_factor     Sec. 2.4 / Eq. 4: blocked right-looking LU with partial
//                     pivoting (first index of the largest |a|), panel in
//                     shared memory, trailing update on FP32 FMA (T = float)
//                     or on the FP64 tensor path, mma.sync m8n8k4 (T = double)
//   cta_chol_factor   Sec. 2.3: blocked right-looking Cholesky, lower
//   cta_tri_solve     Eq. 3 forward substitution / back substitution with a
//                     triangular factor, optionally transposed
//   cta_residual      R = B - A X in FP64, with per-column max norms
//   cta_rcond_est     1-norm estimate of inv(A) (Hager 1984, Higham 1988)
//
// All reductions use a fixed order, so results do not depend on scheduling.
#pragma once
#include "asolve_internal.cuh"

namespace asv {
// internal linkage: every translation unit that includes this header gets
// its own copy of these device functions
namespace {

constexpr int kThreads = kCtaThreads;
constexpr int kWarps = kThreads / kWarp;

// ---------------------------------------------------------------- reductions
struct CtaRed {
  double d[kWarps];
  int i[kWarps];
  int flag;
};

__device__ __forceinline__ double cta_sum(double v, CtaRed& r) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) r.d[w] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kWarps; ++k) s += r.d[k];
  return s;
}

__device__ __forceinline__ double cta_max(double v, CtaRed& r) {
  v = warp_max(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) r.d[w] = v;
  __syncthreads();
  double s = r.d[0];
#pragma unroll
  for (int k = 1; k < kWarps; ++k) s = r.d[k] > s ? r.d[k] : s;
  return s;
}

// first index of max |value| (value given as non-negative magnitude)
template <typename M>
__device__ __forceinline__ int cta_argmax_first(M v, int idx, CtaRed& r) {
  warp_argmax_first(v, idx);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  M* rv = reinterpret_cast<M*>(r.d);
  __syncthreads();
  if (lane == 0) { rv[w] = v; r.i[w] = idx; }
  __syncthreads();
  M bv = rv[0];
  int bi = r.i[0];
#pragma unroll
  for (int k = 1; k < kWarps; ++k)
    if (rv[k] > bv || (rv[k] == bv && r.i[k] < bi)) { bv = rv[k]; bi = r.i[k]; }
  return bi;
}

// ----------------------------------------------------------- DMMA fragment
// mma.sync.aligned.m8n8k4.row.col.f64: A 8x4, B 4x8, C 8x8.
// lane = 4*g + t: A[g][t], B[t][g], C[g][2t], C[g][2t+1].
__device__ __forceinline__ void dmma_8x8x4(double& c0, double& c1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(c0), "+d"(c1)
               : "d"(a), "d"(b));
}

// ------------------------------------------------------------ GEMM update
// Trailing update of a blocked factorisation:  C(m x nc) -= As(m x kb) * Bt,
// with As in shared memory (column-major, ld lda) and the kb x 64 tile Bt in
// shared memory (row-major, Bt[k * 64 + c]).  C is global (column-major,
// ld ldc).  With lower_only, row tiles entirely above the diagonal of C
// (rows < cols, counting rows from row_off) are skipped.
//
// FP32: CTA tile 128 x 64; lane -> rows lane + 32 i (i < 4), warp -> 8
// columns, so every global access of C is one 128-byte line per warp.
// FP64: the 8x8x4 tensor instruction (mma.sync f64); warp tile 16 x 32.
template <typename T>
__device__ void tile_gemm_sub(T* C, int ldc, const T* As, int lda, const T* Bt, int m, int nc, int kb,
                              int col_off, bool lower_only);

template <>
__device__ __noinline__ void tile_gemm_sub<float>(float* C, int ldc, const float* As, int lda,
                                                  const float* Bt, int m, int nc, int kb, int col_off,
                                                  bool lower_only) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int istart = lower_only ? (col_off / 128) * 128 : 0;
  for (int i0 = istart; i0 < m; i0 += 128) {
    // C tile loaded first, so its latency overlaps the k loop
    float acc[4][8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = w * 8 + j;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = i0 + lane + 32 * i;
        acc[i][j] = (c < nc && r < m) ? C[(size_t)c * ldc + r] : 0.f;
      }
    }
#pragma unroll 2
    for (int k = 0; k < kb; ++k) {
      float a[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = i0 + lane + 32 * i;
        a[i] = (r < m) ? As[(size_t)k * lda + r] : 0.f;
      }
      const float4 b0 = *reinterpret_cast<const float4*>(Bt + k * 64 + w * 8);
      const float4 b1 = *reinterpret_cast<const float4*>(Bt + k * 64 + w * 8 + 4);
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(-a[i], b[j], acc[i][j]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = w * 8 + j;
      if (c >= nc) continue;
      float* col = C + (size_t)c * ldc;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = i0 + lane + 32 * i;
        if (r < m) col[r] = acc[i][j];
      }
    }
  }
}

template <>
__device__ __noinline__ void tile_gemm_sub<double>(double* C, int ldc, const double* As, int lda,
                                                   const double* Bt, int m, int nc, int kb, int col_off,
                                                   bool lower_only) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int wr = (w & 3) * 16, wc = (w >> 2) * 32;
  const int kb4 = (kb + 3) & ~3;
  const int istart = lower_only ? (col_off / 64) * 64 : 0;
  for (int i0 = istart; i0 < m; i0 += 64) {
    // the C tile is the accumulator's initial value: its 16 loads go out
    // together, and the products are accumulated negated
    double acc[2][4][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int r = i0 + wr + a * 8 + g, c = wc + b * 8 + 2 * t + q;
          acc[a][b][q] = (r < m && c < nc) ? C[(size_t)c * ldc + r] : 0.0;
        }
#pragma unroll 2
    for (int k = 0; k < kb4; k += 4) {
      double af[2], bf[4];
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const int r = i0 + wr + a * 8 + g;
        af[a] = (r < m && k + t < kb) ? -As[(size_t)(k + t) * lda + r] : 0.0;
      }
#pragma unroll
      for (int b = 0; b < 4; ++b) bf[b] = (k + t < kb) ? Bt[(k + t) * 64 + wc + b * 8 + g] : 0.0;
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) dmma_8x8x4(acc[a][b][0], acc[a][b][1], af[a], bf[b]);
    }
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const int r = i0 + wr + a * 8 + g;
      if (r >= m) continue;
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int c = wc + b * 8 + 2 * t + q;
          if (c < nc) C[(size_t)c * ldc + r] = acc[a][b][q];
        }
    }
  }
}

// Inverse of the unit lower triangular kb x kb block L11 (panel rows 0..kb-1,
// ld m) into Li (32 x 32, column-major, ld 33), by warp 0: lane j forms
// column j.  Padded with the identity past kb.
template <typename T>
__device__ void unit_lower_inverse(const T* Pn, int m, int kb, T* Li) {
  if (threadIdx.x < 32) {
    const int j = threadIdx.x;
    T x[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      T s = (i == j) ? T(1) : T(0);
#pragma unroll
      for (int k = 0; k < i; ++k)
        if (i < kb) s -= Pn[(size_t)k * m + i] * x[k];
      x[i] = s;
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) Li[j * 33 + i] = x[i];
  }
}

// LU panel epilogue: U12 = inv(L11) A12 and A22 -= L21 U12, column block by
// column block of 64.  Ta, Tu: smem tiles of 32 x 64.
template <typename T>
__device__ __noinline__ void cta_lu_update(T* W, int ldw, int n, int k0, int kb, const T* Pn, int m,
                                           T* Li, T* Ta, T* Tu) {
  unit_lower_inverse<T>(Pn, m, kb, Li);
  const int j_lo = k0 + kb;
  for (int j0 = j_lo; j0 < n; j0 += 64) {
    const int nc = min(64, n - j0);
    __syncthreads();
    // stage A12 columns j0.. (rows k0..k0+kb-1): lanes over rows ->
    // coalesced loads; row stride 65 keeps the stores conflict-free
    for (int e = threadIdx.x; e < 32 * 64; e += kThreads) {
      const int k = e & 31, c = e >> 5;
      Ta[k * 65 + c] = (k < kb && c < nc) ? W[(size_t)(j0 + c) * ldw + k0 + k] : T(0);
    }
    __syncthreads();
    // U tile = inv(L11) A12 tile
    if constexpr (sizeof(T) == 8) {
      // FP64: 32 x 64 x 32 on mma.sync f64; warp w owns row tile (w & 3)
      // and column tiles 4 (w >> 2) .. 4 (w >> 2) + 3
      const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
      const int g = lane >> 2, t = lane & 3;
      const int ri = (w & 3) * 8;
      double acc[4][2];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q][0] = acc[q][1] = 0.0;
#pragma unroll
      for (int k = 0; k < 32; k += 4) {
        const double a = Li[(k + t) * 33 + ri + g];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int cj = ((w >> 2) * 4 + q) * 8;
          dmma_8x8x4(acc[q][0], acc[q][1], a, Ta[(k + t) * 65 + cj + g]);
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int cj = ((w >> 2) * 4 + q) * 8;
        Tu[(ri + g) * 64 + cj + 2 * t] = acc[q][0];
        Tu[(ri + g) * 64 + cj + 2 * t + 1] = acc[q][1];
      }
    } else {
      for (int e = threadIdx.x; e < 32 * 64; e += kThreads) {
        const int c = e & 63, i = e >> 6;
        T acc = T(0);
#pragma unroll 8
        for (int k = 0; k < 32; ++k) acc += Li[k * 33 + i] * Ta[k * 65 + c];
        Tu[i * 64 + c] = acc;
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * 64; e += kThreads) {
      const int k = e & 31, c = e >> 5;
      if (k < kb && c < nc) W[(size_t)(j0 + c) * ldw + k0 + k] = Tu[k * 64 + c];
    }
    const int mr = m - kb;
    if (mr > 0)
      tile_gemm_sub<T>(W + (size_t)j0 * ldw + k0 + kb, ldw, Pn + kb, m, Tu, mr, nc, kb, 0, false);
  }
  __syncthreads();
}

// Cholesky panel epilogue: A22 -= L21 L21^T on the lower triangle, column
// block by column block; the B tile (L21^T) is staged from the panel.
template <typename T>
__device__ __noinline__ void cta_chol_update(T* W, int ldw, int n, int k0, int kb, const T* Pn, int m, T* Tu) {
  const int mr = m - kb;
  for (int jc = 0; jc < mr; jc += 64) {
    const int nc = min(64, mr - jc);
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * 64; e += kThreads) {
      const int c = e & 63, k = e >> 6;
      Tu[k * 64 + c] = (k < kb && c < nc) ? Pn[(size_t)k * m + kb + jc + c] : T(0);
    }
    __syncthreads();
    // rows jc.. of the trailing block (the diagonal tile and below)
    tile_gemm_sub<T>(W + (size_t)(k0 + kb + jc) * ldw + k0 + kb + jc, ldw, Pn + kb + jc, m, Tu, mr - jc, nc, kb,
                     0, false);
  }
  __syncthreads();
}

// 2-D copy of an m x nc column-major block.  The block is cut into 32-row
// pieces of columns; warp w takes pieces w, w + 8, ... and has eight of
// them (eight loads per lane) in flight before it stores any.  The piece's
// (column, row) position advances incrementally: no integer division.
template <typename D, typename S>
__device__ __forceinline__ void cta_copy_block(D* dst, int ldd, const S* src, int lds, int m, int nc) {
  constexpr int U = 8;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int chunks = (m + 31) >> 5;
  int c = 0, k = w;  // piece w: column c, 32-row chunk k
  while (k >= chunks && c < nc) {
    k -= chunks;
    ++c;
  }
  while (c < nc) {
    S v[U];
    int cc[U], rr[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      cc[q] = c;
      rr[q] = 32 * k + lane;
      v[q] = (c < nc && rr[q] < m) ? src[(size_t)c * lds + rr[q]] : S(0);
      k += kWarps;
      while (k >= chunks) {
        k -= chunks;
        ++c;
      }
    }
#pragma unroll
    for (int q = 0; q < U; ++q)
      if (cc[q] < nc && rr[q] < m) dst[(size_t)cc[q] * ldd + rr[q]] = (D)v[q];
  }
}

// Reduction record of the panel pivot search: magnitude, row, signed value.
template <typename T>
struct PivRed {
  T mag[kWarps];
  T val[kWarps];
  int idx[kWarps];
};

// --------------------------------------------------------------- LU factor
// W: n x n (ld ldw), overwritten by L\U; piv[k] = row swapped with k.
// smem: panel (m x nb of T, ld m), then the L11 inverse and two 32 x 64
// tiles (see cta_lu_update).  Returns 0, or
// k+1 at an exact zero (or NaN-only) pivot, where it stops: the solver has
// then failed.  Two barriers per panel column.
template <typename T>
__device__ __noinline__ int cta_lu_factor(T* W, int ldw, int n, int* piv, T* smem, int nb) {
  __shared__ PivRed<T> pr;
  __shared__ T prow[32];
  __shared__ int spiv[32];  // this panel's pivot rows, for the swaps outside it
  T* Pn = smem;
  // after the panel: L11 inverse (32 x 33) and two 32 x 64 tiles
  T* Li = smem + (size_t)n * nb;
  T* Ta = Li + 32 * 33 + 3;
  Ta = reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(Ta) + 15) & ~(uintptr_t)15);
  T* Tu = Ta + 32 * 65 + 4;
  Tu = reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(Tu) + 15) & ~(uintptr_t)15);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k0 = 0; k0 < n; k0 += nb) {
    const int kb = min(nb, n - k0), m = n - k0;
    __syncthreads();
    cta_copy_block<T, T>(Pn, m, W + (size_t)k0 * ldw + k0, ldw, m, kb);
    __syncthreads();
    for (int c = 0; c < kb; ++c) {
      // pivot search over this thread's rows (written by this thread only)
      T best = T(-1), bval = T(0);
      int bi = 0x7fffffff;
      for (int r = c + threadIdx.x; r < m; r += kThreads) {
        const T v = Pn[(size_t)c * m + r];
        const T a = fabs(v);
        if (a > best) { best = a; bi = r; bval = v; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        const T ov = __shfl_xor_sync(0xffffffffu, bval, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; bval = ov; }
      }
      if (lane == 0) { pr.mag[w] = best; pr.idx[w] = bi; pr.val[w] = bval; }
      __syncthreads();  // S1
      // the 8 warps' candidates: lane l reads candidate l & 7, then a
      // butterfly over groups of 8 lanes (the same order: largest |v|,
      // then the smallest row)
      static_assert(kWarps == 8, "pivot candidates: one per warp, 8 warps");
      T bm = pr.mag[lane & 7], pv = pr.val[lane & 7];
      int p = pr.idx[lane & 7];
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) {
        const T ob = __shfl_xor_sync(0xffffffffu, bm, o);
        const int oi = __shfl_xor_sync(0xffffffffu, p, o);
        const T ov = __shfl_xor_sync(0xffffffffu, pv, o);
        if (ob > bm || (ob == bm && oi < p)) { bm = ob; p = oi; pv = ov; }
      }
      if (p < c || p >= m || pv == T(0) || pv != pv) {
        __syncthreads();
        return k0 + c + 1;
      }
      // swap rows c and p inside the panel, one thread per column; the new
      // pivot row is also kept in prow
      if (threadIdx.x < kb) {  // the whole panel row, multipliers included
        const int cc = threadIdx.x;
        const T a = Pn[(size_t)cc * m + c], b = Pn[(size_t)cc * m + p];
        Pn[(size_t)cc * m + c] = b;
        Pn[(size_t)cc * m + p] = a;
        prow[cc] = b;
      }
      if (threadIdx.x == 0) {
        piv[k0 + c] = k0 + p;
        spiv[c] = k0 + p;
      }
      __syncthreads();  // S2
      const T inv = T(1) / pv;
      for (int r = c + 1 + threadIdx.x; r < m; r += kThreads) {
        const T l = Pn[(size_t)c * m + r] * inv;
        Pn[(size_t)c * m + r] = l;
#pragma unroll 4
        for (int cc = c + 1; cc < kb; ++cc) Pn[(size_t)cc * m + r] -= l * prow[cc];
      }
    }
    __syncthreads();
    cta_copy_block<T, T>(W + (size_t)k0 * ldw + k0, ldw, Pn, m, m, kb);
    // apply this panel's row swaps to the columns left and right of it
    for (int col = threadIdx.x; col < n; col += kThreads) {
      if (col >= k0 && col < k0 + kb) continue;
      T* cp = W + (size_t)col * ldw;
      for (int c = 0; c < kb; ++c) {
        const int p = spiv[c];
        if (p != k0 + c) {
          const T a = cp[k0 + c];
          cp[k0 + c] = cp[p];
          cp[p] = a;
        }
      }
    }
    __syncthreads();
    if (n - k0 - kb > 0) cta_lu_update<T>(W, ldw, n, k0, kb, Pn, m, Li, Ta, Tu);
  }
  __syncthreads();
  return 0;
}

// --------------------------------------------------------- Cholesky factor
// Lower Cholesky of W (only the lower triangle is read and written).
// Returns 0, or k+1 where the pivot is not > 0 (incl. NaN).  One barrier
// per panel column: the step for column c reads the unscaled column c and
// forms the multipliers on the fly; each thread scales its own rows of
// column c during the next step, when nobody reads that column any more.
template <typename T>
__device__ __noinline__ int cta_chol_factor(T* W, int ldw, int n, T* smem, int nb) {
  T* Pn = smem;
  T* Tu = smem + (size_t)n * nb;
  Tu = reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(Tu) + 15) & ~(uintptr_t)15);
  for (int k0 = 0; k0 < n; k0 += nb) {
    const int kb = min(nb, n - k0), m = n - k0;
    __syncthreads();
    cta_copy_block<T, T>(Pn, m, W + (size_t)k0 * ldw + k0, ldw, m, kb);
    T prev_inv = T(0), prev_ljj = T(0);
    for (int c = 0; c < kb; ++c) {
      __syncthreads();
      const T d = Pn[(size_t)c * m + c];
      if (!(d > T(0))) {
        __syncthreads();
        return k0 + c + 1;
      }
      const T ljj = sqrt(d);
      const T inv = T(1) / ljj;
      for (int r = c + threadIdx.x; r < m; r += kThreads) {
        if (c > 0) Pn[(size_t)(c - 1) * m + r] *= prev_inv;  // deferred scaling of column c-1
        if (r == c) continue;
        const T l = Pn[(size_t)c * m + r] * inv;
        const int cmax = min(kb - 1, r);
        for (int cc = c + 1; cc <= cmax; ++cc) Pn[(size_t)cc * m + r] -= l * (Pn[(size_t)c * m + cc] * inv);
      }
      // rows < c of column c-1 are above the diagonal (unused); row c-1 of
      // column c-1 is the diagonal entry, stored below
      if (threadIdx.x == 0 && c > 0) Pn[(size_t)(c - 1) * m + (c - 1)] = prev_ljj;
      prev_inv = inv;
      prev_ljj = ljj;
    }
    __syncthreads();
    {  // scale the last column and store the diagonal
      const int c = kb - 1;
      for (int r = c + threadIdx.x; r < m; r += kThreads)
        Pn[(size_t)c * m + r] = (r == c) ? prev_ljj : Pn[(size_t)c * m + r] * prev_inv;
    }
    __syncthreads();
    for (int c = (threadIdx.x >> 5); c < kb; c += kWarps)
      for (int r = c + (threadIdx.x & 31); r < m; r += 32)
        W[(size_t)(k0 + c) * ldw + k0 + r] = Pn[(size_t)c * m + r];
    __syncthreads();
    if (n - k0 - kb > 0) cta_chol_update<T>(W, ldw, n, k0, kb, Pn, m, Tu);
  }
  __syncthreads();
  return 0;
}

// ------------------------------------------------------- triangular solves
// Inverses of the 32 x 32 diagonal blocks of a triangular M (lower/upper,
// unit or not), padded with the identity past n.  Block b is stored
// column-major at Dinv + 1024 b.  One warp per block: lane j forms column
// j of the inverse by substitution against e_j.
template <typename T>
__device__ __noinline__ void cta_block_inverses(const T* __restrict__ M, int ldm, int n, bool lower,
                                                bool unit, T* Dinv) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nblk = (n + 31) / 32;
  for (int b = w; b < nblk; b += kWarps) {
    const int b0 = b * 32, bs = min(32, n - b0);
    T x[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) x[i] = (i == lane) ? T(1) : T(0);
    if (lower) {
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        if (i < bs) {
          T s = x[i];
#pragma unroll
          for (int k = 0; k < i; ++k) s -= M[(size_t)(b0 + k) * ldm + b0 + i] * x[k];
          x[i] = unit ? s : s / M[(size_t)(b0 + i) * ldm + b0 + i];
        }
      }
    } else {
#pragma unroll
      for (int ii = 0; ii < 32; ++ii) {
        const int i = 31 - ii;
        if (i < bs) {
          T s = x[i];
#pragma unroll
          for (int k = i + 1; k < 32; ++k)
            if (k < bs) s -= M[(size_t)(b0 + k) * ldm + b0 + i] * x[k];
          x[i] = unit ? s : s / M[(size_t)(b0 + i) * ldm + b0 + i];
        }
      }
    }
    T* out = Dinv + (size_t)b * 1024 + (size_t)lane * 32;
#pragma unroll
    for (int i = 0; i < 32; ++i) out[i] = x[i];
  }
  __syncthreads();
}

// Compile-time right-hand-side count: with_nr(nrhs, f) calls f with an
// IntC<nrhs> (1 <= nrhs <= 8), so that per-column loops unroll to exactly
// nrhs operations.  A loop over 8 columns predicated on c < nrhs still
// issues all 8 instructions per warp, and on GB300's FP64 pipe (2 lanes
// per clock per SM) every issued FP64 warp instruction costs 16 SM cycles
// whether its lanes are on or off.
template <int N>
struct IntC {
  static constexpr int value = N;
};
template <typename F>
__device__ __forceinline__ void with_nr(int nrhs, F&& f) {
  switch (nrhs) {
    case 0: break;
    case 1: f(IntC<1>{}); break;
    case 2: f(IntC<2>{}); break;
    case 3: f(IntC<3>{}); break;
    case 4: f(IntC<4>{}); break;
    case 5: f(IntC<5>{}); break;
    case 6: f(IntC<6>{}); break;
    case 7: f(IntC<7>{}); break;
    default: f(IntC<8>{}); break;
  }
}

// Row update of a blocked triangular solve, E = M:  x(r, :) -= M(r, b0 +
// j) x(b0 + j, :) for rows r_lo <= r < r_hi, j < bs; thread per row,
// coalesced over r, the block's loads of M unrolled so that they are in
// flight together.
template <int NR, typename T, typename V>
__device__ __forceinline__ void tri_update_direct(const T* __restrict__ M, int ldm, V* x, int ldx, int b0, int bs,
                                                  int r_lo, int r_hi) {
  for (int r = r_lo + (int)threadIdx.x; r < r_hi; r += kThreads) {
    V acc[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) acc[c] = V(0);
#pragma unroll 16
    for (int j = 0; j < bs; ++j) {
      const V m = (V)M[(size_t)(b0 + j) * ldm + r];
#pragma unroll
      for (int c = 0; c < NR; ++c) acc[c] += m * x[(size_t)c * ldx + b0 + j];
    }
#pragma unroll
    for (int c = 0; c < NR; ++c) x[(size_t)c * ldx + r] -= acc[c];
  }
}

// The same with E = M^T:  x(r, :) -= M(b0 + j, r) x(b0 + j, :).  Each warp
// stages the 32 x 32 tile M(b0.., r0..) in `tile` (32 x 33) with coalesced
// column loads, then lane i finishes row r0 + i.
template <int NR, typename T, typename V>
__device__ __forceinline__ void tri_update_staged(const T* __restrict__ M, int ldm, V* x, int ldx, int b0, int bs,
                                                  int r_lo, int r_hi, T* tile) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int r0 = r_lo + 32 * w; r0 < r_hi; r0 += 32 * kWarps) {
#pragma unroll 8
    for (int i = 0; i < 32; ++i) {
      const int r = r0 + i;
      tile[i * 33 + lane] = (r < r_hi && lane < bs) ? M[(size_t)r * ldm + b0 + lane] : T(0);
    }
    __syncwarp();
    const int r = r0 + lane;
    if (r < r_hi) {
      V acc[NR];
#pragma unroll
      for (int c = 0; c < NR; ++c) acc[c] = V(0);
      for (int j = 0; j < bs; ++j) {
        const V m = (V)tile[lane * 33 + j];
#pragma unroll
        for (int c = 0; c < NR; ++c) acc[c] += m * x[(size_t)c * ldx + b0 + j];
      }
#pragma unroll
      for (int c = 0; c < NR; ++c) x[(size_t)c * ldx + r] -= acc[c];
    }
    __syncwarp();
  }
}

// x (smem, n x nrhs, ld ldx) <- inv(E) x with E = trans ? M^T : M, M lower
// or upper (ld ldm), unit diagonal if `unit`.  Blocked by 32 rows.  With
// Dinv (the diagonal-block inverses of M) the block step is a product with
// the inverse; without it the block is loaded into registers (lane i holds
// row i) and solved by substitution, one warp per right-hand side.  The
// rows after the block are then updated by all threads.  MT (optional,
// with E = M^T): M's transpose, ld ldm; the updates then read E's rows
// as coalesced columns of MT instead of strided rows of M.
template <typename T, typename V, bool ELOWER>
__device__ __noinline__ void cta_tri_solve_dir(const T* __restrict__ M, int ldm, int n, bool trans, bool unit,
                                               V* x, int ldx, int nrhs, const T* __restrict__ Dinv,
                                               T* stage, const T* __restrict__ MT) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nblk = (n + 31) / 32;
  for (int bi = 0; bi < nblk; ++bi) {
    const int blk = ELOWER ? bi : nblk - 1 - bi;
    const int b0 = blk * 32, bs = min(32, n - b0);
    __syncthreads();
    if (w < nrhs) {
      if (Dinv) {
        const T* D = Dinv + (size_t)blk * 1024;
        for (int c = w; c < nrhs; c += kWarps) {
          V xin = (lane < bs) ? x[(size_t)c * ldx + b0 + lane] : V(0);
          V acc = V(0);
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const V xj = __shfl_sync(0xffffffffu, xin, j);
            // inv(E)(lane, j): E = M^T -> inv(D)(j, lane)
            const V dij = (V)(trans ? D[(size_t)lane * 32 + j] : D[(size_t)j * 32 + lane]);
            acc += dij * xj;
          }
          if (lane < bs) x[(size_t)c * ldx + b0 + lane] = acc;
        }
      } else {
        V e[32];
        const int r = b0 + lane;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          V v = (lane == j) ? V(1) : V(0);
          if (lane < bs && j < bs) {
            const bool inside = ELOWER ? (j <= lane) : (j >= lane);
            if (inside && !(unit && j == lane))
              v = (V)(trans ? M[(size_t)r * ldm + b0 + j] : M[(size_t)(b0 + j) * ldm + r]);
          }
          e[j] = v;
        }
        V dinv = V(1);
        if (!unit) {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (j == lane) dinv = V(1) / e[j];
        }
        for (int c = w; c < nrhs; c += kWarps) {
          V xi = (lane < bs) ? x[(size_t)c * ldx + b0 + lane] : V(0);
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) {
            const int j = ELOWER ? jj : 31 - jj;
            if (lane == j) xi = unit ? xi : xi * dinv;
            const V xj = __shfl_sync(0xffffffffu, xi, j);
            if (ELOWER ? (lane > j) : (lane < j)) xi -= e[j] * xj;
          }
          if (lane < bs) x[(size_t)c * ldx + b0 + lane] = xi;
        }
      }
    }
    __syncthreads();
    const int r_lo = ELOWER ? b0 + bs : 0, r_hi = ELOWER ? n : b0;
    if (!trans || MT) {
      const T* E = trans ? MT : M;
      with_nr(nrhs, [&](auto nr) { tri_update_direct<decltype(nr)::value, T, V>(E, ldm, x, ldx, b0, bs, r_lo, r_hi); });
    } else if (stage) {
      with_nr(nrhs, [&](auto nr) {
        tri_update_staged<decltype(nr)::value, T, V>(M, ldm, x, ldx, b0, bs, r_lo, r_hi, stage + (size_t)w * 32 * 33);
      });
    } else {
      // E(r, j) = M(j, r): warp per row, lanes over j (coalesced), shuffle sums
      for (int r = r_lo + w; r < r_hi; r += kWarps) {
        const V m = (lane < bs) ? (V)M[(size_t)r * ldm + b0 + lane] : V(0);
        for (int c = 0; c < nrhs; ++c) {
          const V sum = warp_sum(m * ((lane < bs) ? x[(size_t)c * ldx + b0 + lane] : V(0)));
          if (lane == 0) x[(size_t)c * ldx + r] -= sum;
        }
      }
    }
  }
  __syncthreads();
}

// stage: optional shared-memory scratch of 8 x 32 x 33 elements of T for
// the transposed update (without it, warp-per-row shuffle sums are used);
// MT: optional transpose of M, which the transposed update reads instead.
template <typename T, typename V>
__device__ void cta_tri_solve(const T* M, int ldm, int n, bool lower, bool trans, bool unit, V* x, int ldx,
                              int nrhs, const T* Dinv = nullptr, T* stage = nullptr, const T* MT = nullptr) {
  if (lower != trans) cta_tri_solve_dir<T, V, true>(M, ldm, n, trans, unit, x, ldx, nrhs, Dinv, stage, MT);
  else cta_tri_solve_dir<T, V, false>(M, ldm, n, trans, unit, x, ldx, nrhs, Dinv, stage, MT);
}

// Row permutation of LU with partial pivoting as one gather: after the
// swaps k <-> piv[k] (k = 0..n-1), position k holds original row perm[k].
// The swaps form one sequential chain, so they run in shared memory
// (s_tmp: 2n ints); a chain of dependent global-memory round trips cost
// ~0.4 ms at n = 512.
__device__ void cta_build_perm(const int* piv, int n, int* perm, int* s_tmp) {
  int* sp = s_tmp;
  int* sq = s_tmp + n;
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += kThreads) {
    sp[k] = piv[k];
    sq[k] = k;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < n; ++k) {
      const int p = sp[k];
      const int t = sq[k];
      sq[k] = sq[p];
      sq[p] = t;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += kThreads) perm[k] = sq[k];
  __syncthreads();
}

// x <- P x (forward) or x <- P^T x (inverse), x in smem, n x nrhs, through
// the scratch buffer tmp (n x nrhs).
template <typename V>
__device__ __noinline__ void cta_permute(V* x, int ldx, int n, int nrhs, const int* perm, bool inverse,
                                         V* tmp) {
  __syncthreads();  // x may have just been written by other threads
  for (int c = 0; c < nrhs; ++c)
    for (int k = threadIdx.x; k < n; k += kThreads) {
      const int src = inverse ? k : perm[k];
      const int dst = inverse ? perm[k] : k;
      tmp[(size_t)c * n + dst] = x[(size_t)c * ldx + src];
    }
  __syncthreads();
  for (int c = 0; c < nrhs; ++c)
    for (int k = threadIdx.x; k < n; k += kThreads) x[(size_t)c * ldx + k] = tmp[(size_t)c * n + k];
  __syncthreads();
}

// LU application: x <- inv(A) x (trans: inv(A)^T x) with A = P L U, where
// perm is the gather form of the pivots (cta_build_perm).  Linv/Uinv: the
// diagonal-block inverses of L and U, or null for substitution.  WT: the
// factor's transpose (cta_transpose), or null.
template <typename T, typename V>
__device__ void cta_lu_apply(const T* W, int ldw, int n, const int* perm, V* x, int ldx, int nrhs,
                             bool trans, V* tmp, const T* Linv = nullptr, const T* Uinv = nullptr,
                             T* stage = nullptr, const T* WT = nullptr) {
  if (!trans) {
    cta_permute<V>(x, ldx, n, nrhs, perm, false, tmp);
    cta_tri_solve<T, V>(W, ldw, n, true, false, true, x, ldx, nrhs, Linv, stage);
    cta_tri_solve<T, V>(W, ldw, n, false, false, false, x, ldx, nrhs, Uinv, stage);
  } else {
    cta_tri_solve<T, V>(W, ldw, n, false, true, false, x, ldx, nrhs, Uinv, stage, WT);
    cta_tri_solve<T, V>(W, ldw, n, true, true, true, x, ldx, nrhs, Linv, stage, WT);
    cta_permute<V>(x, ldx, n, nrhs, perm, true, tmp);
  }
}

template <typename T, typename V>
__device__ void cta_chol_apply(const T* W, int ldw, int n, V* x, int ldx, int nrhs,
                               const T* Linv = nullptr, T* stage = nullptr, const T* WT = nullptr) {
  cta_tri_solve<T, V>(W, ldw, n, true, false, false, x, ldx, nrhs, Linv, stage);
  cta_tri_solve<T, V>(W, ldw, n, true, true, false, x, ldx, nrhs, Linv, stage, WT);
}

// WT = W^T (n x n, both ld ldw; W and WT do not overlap), through one
// 32 x 33 shared-memory tile per warp (stage: 8 x 32 x 33 elements of T):
// coalesced column loads of W and column stores of WT.
template <typename T>
__device__ __noinline__ void cta_transpose(const T* __restrict__ W, int ldw, int n, T* __restrict__ WT, T* stage) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T* tile = stage + (size_t)w * 32 * 33;
  const int nt = (n + 31) / 32;
  __syncthreads();
  for (int t = w; t < nt * nt; t += kWarps) {
    const int i0 = (t % nt) * 32, j0 = (t / nt) * 32;
    const int i = i0 + lane;
#pragma unroll 8
    for (int c = 0; c < 32; ++c) {  // tile[c][lane] = W(i0 + lane, j0 + c)
      const int j = j0 + c;
      tile[c * 33 + lane] = (i < n && j < n) ? W[(size_t)j * ldw + i] : T(0);
    }
    __syncwarp();
    const int j = j0 + lane;
#pragma unroll 8
    for (int c = 0; c < 32; ++c) {  // WT(j0 + lane, i0 + c) = W(i0 + c, j0 + lane)
      const int ic = i0 + c;
      if (ic < n && j < n) WT[(size_t)ic * ldw + j] = tile[lane * 33 + c];
    }
    __syncwarp();
  }
  __syncthreads();
}

// -------------------------------------------------------------- residual
// R = B - A X in FP64 (A: n x n ld lda; X: n x nrhs ld n), writes R (ld n)
// and the per-column max |r| to rmax_s[c] (NaN when a column has one).
// DFMA, one thread per row (coalesced over the rows of column-major A) and
// exactly nrhs accumulators: the work is n^2 nrhs FP64 FMAs, which bound
// it on GB300's narrow FP64 pipe (the 8-column mma.sync f64 form would
// spend n^2 8 whatever nrhs is, at a lower rate than DFMA).
template <int NR>
__device__ __forceinline__ void residual_rows(const double* __restrict__ A, int lda, int n,
                                              const double* __restrict__ B, const double* Xs, double* R,
                                              unsigned long long* s_mx) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  constexpr int U = NR == 1 ? 16 : (NR == 2 ? 8 : (NR <= 4 ? 4 : 2));
  unsigned long long mx[NR];
#pragma unroll
  for (int c = 0; c < NR; ++c) mx[c] = 0ull;
  for (int i0 = 32 * w; i0 < n; i0 += kThreads) {  // warp-uniform: idle warps skip
    const int i = i0 + lane;
    const bool ok = i < n;
    double acc[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) acc[c] = 0.0;
#pragma unroll U
    for (int j = 0; j < n; ++j) {
      const double a = ok ? __ldg(A + (size_t)j * lda + i) : 0.0;
#pragma unroll
      for (int c = 0; c < NR; ++c) acc[c] = fma(a, Xs[(size_t)c * n + j], acc[c]);
    }
    if (ok) {
#pragma unroll
      for (int c = 0; c < NR; ++c) {
        const double r = B[(size_t)c * n + i] - acc[c];
        R[(size_t)c * n + i] = r;
        // |r| as bits: ordered like the values, NaN above every number
        const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(r));
        mx[c] = b > mx[c] ? b : mx[c];
      }
    }
  }
#pragma unroll
  for (int c = 0; c < NR; ++c) {
    unsigned long long v = mx[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
      v = u > v ? u : v;
    }
    if (lane == 0) atomicMax(s_mx + c, v);
  }
}

__device__ __noinline__ void cta_residual(const double* __restrict__ A, int lda, int n, const double* __restrict__ B,
                                          const double* Xs, int nrhs, double* R, double* rmax_s) {
  __shared__ unsigned long long s_mx[8];
  if (threadIdx.x < 8) s_mx[threadIdx.x] = 0ull;
  __syncthreads();
  with_nr(nrhs, [&](auto nr) { residual_rows<decltype(nr)::value>(A, lda, n, B, Xs, R, s_mx); });
  __syncthreads();
  if (threadIdx.x < nrhs) rmax_s[threadIdx.x] = __longlong_as_double((long long)s_mx[threadIdx.x]);
  __syncthreads();
}

// ------------------------------------------------------------ estimator
// 1-norm estimate of inv(A) (Hager 1984; Higham 1988): apply(v, trans, k)
// overwrites the k <= 2 smem columns v, v + n with inv(A) v or inv(A)^T v.
// v: room for 2n values; xi: smem scratch of length n after them.  The
// closing test vector of alternating signs (Higham 1988) does not depend on
// the iteration, so it is the second column of the first product: the same
// values as a product of its own, one dependent solve fewer.
template <typename V, typename Apply>
__device__ double cta_est_inv_norm1(int n, V* v, V* xi, Apply apply, CtaRed& red) {
  __syncthreads();
  if (n == 1) {
    if (threadIdx.x == 0) v[0] = V(1);
    apply(v, false, 1);
    __syncthreads();
    double e = fabs((double)v[0]);
    __syncthreads();
    return e;
  }
  for (int i = threadIdx.x; i < n; i += kThreads) {
    v[i] = V(1) / V(n);
    const V sgn = (i & 1) ? V(-1) : V(1);
    v[n + i] = sgn * (V(1) + V(i) / V(n - 1));
  }
  apply(v, false, 2);
  auto sum_abs_of = [&](const V* p) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += kThreads) s += fabs((double)p[i]);
    return cta_sum(s, red);
  };
  auto sum_abs = [&]() { return sum_abs_of(v); };
  const double temp = 2.0 * sum_abs_of(v + n) / (double)(3 * n);
  double est = sum_abs();
  for (int i = threadIdx.x; i < n; i += kThreads) {
    V sg = v[i] >= V(0) ? V(1) : V(-1);
    xi[i] = sg;
    v[i] = sg;
  }
  apply(v, true, 1);
  int k = 2;
  for (;;) {
    double best = -1.0;
    int bi = 0x7fffffff;
    for (int i = threadIdx.x; i < n; i += kThreads) {
      double a = fabs((double)v[i]);
      if (a > best) { best = a; bi = i; }
    }
    const int j = cta_argmax_first<double>(best, bi, red);
    __syncthreads();
    if (j < 0 || j >= n) {  // only NaN entries: no estimate
      est = __longlong_as_double(0x7ff8000000000000ll);
      break;
    }
    for (int i = threadIdx.x; i < n; i += kThreads) v[i] = (i == j) ? V(1) : V(0);
    apply(v, false, 1);
    const double estold = est;
    est = sum_abs();
    bool same = true;
    for (int i = threadIdx.x; i < n; i += kThreads) {
      V sg = v[i] >= V(0) ? V(1) : V(-1);
      if (sg != xi[i]) same = false;
    }
    same = __syncthreads_and(same) != 0;
    if (same || est <= estold) break;
    for (int i = threadIdx.x; i < n; i += kThreads) {
      V sg = v[i] >= V(0) ? V(1) : V(-1);
      xi[i] = sg;
      v[i] = sg;
    }
    apply(v, true, 1);
    double best2 = -1.0;
    int bi2 = 0x7fffffff;
    for (int i = threadIdx.x; i < n; i += kThreads) {
      double a = fabs((double)v[i]);
      if (a > best2) { best2 = a; bi2 = i; }
    }
    const int jn = cta_argmax_first<double>(best2, bi2, red);
    ++k;
    if (jn < 0 || jn >= n) {
      est = __longlong_as_double(0x7ff8000000000000ll);
      break;
    }
    const double vj = (double)v[j], vjn = fabs((double)v[jn]);
    __syncthreads();
    if (vj == vjn || k > 5) break;
  }
  if (temp > est) est = temp;
  __syncthreads();
  return est;
}

__device__ __forceinline__ double rcond_from(double anorm, double ainvnm) {
  if (anorm == 0.0 || isinf(ainvnm) || ainvnm == 0.0) return 0.0;
  return (1.0 / ainvnm) / anorm;
}

}  // namespace
}  // namespace asv
