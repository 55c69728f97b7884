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
// C(m x nc) -= As(m x kb, smem, ld lda) * B(kb x nc, global, ld ldb); C global.
// Only tiles with (row tile) >= (col tile) when lower_only (Cholesky SYRK).
// Bs: smem staging of kb x 64 entries of B.
template <typename T>
__device__ void cta_gemm_sub(T* C, int ldc, const T* As, int lda, const T* B, int ldb, int m, int nc,
                             int kb, T* Bs, int row_off_for_lower, bool lower_only);

// FP32 SIMT: CTA tile 128 x 64, thread micro-tile 8 x 4.
template <>
__device__ void cta_gemm_sub<float>(float* C, int ldc, const float* As, int lda, const float* B,
                                    int ldb, int m, int nc, int kb, float* Bs, int row_off,
                                    bool lower_only) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int j0 = 0; j0 < nc; j0 += 64) {
    __syncthreads();
    for (int e = threadIdx.x; e < kb * 64; e += kThreads) {
      int k = e >> 6, c = e & 63;
      Bs[e] = (j0 + c < nc) ? B[(size_t)(j0 + c) * ldb + k] : 0.f;
    }
    __syncthreads();
    int istart = 0;
    if (lower_only) istart = max(0, ((j0 + row_off) / 128) * 128 - row_off);
    for (int i0 = istart; i0 < m; i0 += 128) {
      const int r0 = i0 + ty * 8, c0 = j0 + tx * 4;
      float acc[8][4];
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
#pragma unroll 4
      for (int k = 0; k < kb; ++k) {
        float a[8], b[4];
#pragma unroll
        for (int r = 0; r < 8; ++r) a[r] = (r0 + r < m) ? As[(size_t)k * lda + r0 + r] : 0.f;
#pragma unroll
        for (int c = 0; c < 4; ++c) b[c] = Bs[k * 64 + tx * 4 + c];
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (c0 + c >= nc) continue;
        float* col = C + (size_t)(c0 + c) * ldc;
#pragma unroll
        for (int r = 0; r < 8; ++r)
          if (r0 + r < m) col[r0 + r] -= acc[r][c];
      }
    }
  }
  __syncthreads();
}

// FP64 on the tensor path: CTA tile 64 x 64, warp tile 16 x 32 (2 x 4 mma tiles).
template <>
__device__ void cta_gemm_sub<double>(double* C, int ldc, const double* As, int lda, const double* B,
                                     int ldb, int m, int nc, int kb, double* Bs, int row_off,
                                     bool lower_only) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int wr = (w & 3) * 16, wc = (w >> 2) * 32;
  const int kb4 = (kb + 3) & ~3;
  for (int j0 = 0; j0 < nc; j0 += 64) {
    __syncthreads();
    for (int e = threadIdx.x; e < kb4 * 64; e += kThreads) {
      int k = e >> 6, c = e & 63;
      Bs[e] = (k < kb && j0 + c < nc) ? B[(size_t)(j0 + c) * ldb + k] : 0.0;
    }
    __syncthreads();
    int istart = 0;
    if (lower_only) istart = max(0, ((j0 + row_off) / 64) * 64 - row_off);
    for (int i0 = istart; i0 < m; i0 += 64) {
      double acc[2][4][2];
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b][0] = acc[a][b][1] = 0.0;
      for (int k = 0; k < kb4; k += 4) {
        double af[2], bf[4];
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          int r = i0 + wr + a * 8 + g;
          af[a] = (r < m && k + t < kb) ? As[(size_t)(k + t) * lda + r] : 0.0;
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) bf[b] = Bs[(k + t) * 64 + wc + b * 8 + g];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) dmma_8x8x4(acc[a][b][0], acc[a][b][1], af[a], bf[b]);
      }
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        int r = i0 + wr + a * 8 + g;
        if (r >= m) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            int c = j0 + wc + b * 8 + 2 * t + q;
            if (c < nc) C[(size_t)c * ldc + r] -= acc[a][b][q];
          }
        }
      }
    }
  }
  __syncthreads();
}

// --------------------------------------------------------------- LU factor
// W: n x n (ld ldw), overwritten by L\U; piv[k] = row swapped with k.
// smem: panel (m x nb of T) then Bs (nb x 64 of T).  Returns 0 or k+1 at an
// exact zero pivot (stops there, as the solver then counts as failed).
template <typename T>
__device__ int cta_lu_factor(T* W, int ldw, int n, int* piv, T* smem, int nb, CtaRed& red) {
  T* Pn = smem;  // panel: column-major, ld = m
  for (int k0 = 0; k0 < n; k0 += nb) {
    const int kb = min(nb, n - k0), m = n - k0;
    T* Bs = smem + (size_t)m * nb;
    __syncthreads();
    for (int e = threadIdx.x; e < m * kb; e += kThreads) {
      int r = e % m, c = e / m;
      Pn[(size_t)c * m + r] = W[(size_t)(k0 + c) * ldw + k0 + r];
    }
    __syncthreads();
    // unblocked LU of the m x kb panel; thread t owns rows t, t+256, ...
    for (int c = 0; c < kb; ++c) {
      T best = T(-1);
      int bi = 0x7fffffff;
      for (int r = c + threadIdx.x; r < m; r += kThreads) {
        T v = fabs(Pn[(size_t)c * m + r]);
        if (v > best) { best = v; bi = r; }
      }
      const int p = cta_argmax_first<T>(best, bi, red);  // contains __syncthreads
      const T pv = Pn[(size_t)c * m + p];
      if (pv == T(0)) {
        __syncthreads();
        return k0 + c + 1;
      }
      if (threadIdx.x == 0) piv[k0 + c] = k0 + p;
      const T inv = T(1) / pv;
      __syncthreads();
      if (p != c && threadIdx.x < kb) {
        const int cc = threadIdx.x;
        T a = Pn[(size_t)cc * m + c], b = Pn[(size_t)cc * m + p];
        Pn[(size_t)cc * m + c] = b;
        Pn[(size_t)cc * m + p] = a;
      }
      __syncthreads();
      for (int r = c + 1 + threadIdx.x; r < m; r += kThreads) {
        T l = Pn[(size_t)c * m + r] * inv;
        Pn[(size_t)c * m + r] = l;
        for (int cc = c + 1; cc < kb; ++cc) Pn[(size_t)cc * m + r] -= l * Pn[(size_t)cc * m + c];
      }
      __syncthreads();
    }
    // write the panel back
    for (int e = threadIdx.x; e < m * kb; e += kThreads) {
      int r = e % m, c = e / m;
      W[(size_t)(k0 + c) * ldw + k0 + r] = Pn[(size_t)c * m + r];
    }
    // apply this panel's row swaps to the columns left and right of it
    for (int col = threadIdx.x; col < n; col += kThreads) {
      if (col >= k0 && col < k0 + kb) continue;
      T* cp = W + (size_t)col * ldw;
      for (int c = 0; c < kb; ++c) {
        int p = piv[k0 + c];
        if (p != k0 + c) {
          T a = cp[k0 + c];
          cp[k0 + c] = cp[p];
          cp[p] = a;
        }
      }
    }
    __syncthreads();
    const int nr = n - k0 - kb;
    if (nr > 0) {
      // U12 = inv(L11) A12: unit lower substitution, one thread per column
      for (int col = k0 + kb + threadIdx.x; col < n; col += kThreads) {
        T* cp = W + (size_t)col * ldw + k0;
        T x[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) x[i] = (i < kb) ? cp[i] : T(0);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          if (j >= kb) break;
#pragma unroll
          for (int i = j + 1; i < 32; ++i)
            if (i < kb) x[i] -= Pn[(size_t)j * m + i] * x[j];
        }
#pragma unroll
        for (int i = 0; i < 32; ++i)
          if (i < kb) cp[i] = x[i];
      }
      __syncthreads();
      // A22 -= L21 U12
      cta_gemm_sub<T>(W + (size_t)(k0 + kb) * ldw + k0 + kb, ldw, Pn + kb, m,
                      W + (size_t)(k0 + kb) * ldw + k0, ldw, nr, nr, kb, Bs, 0, false);
    }
  }
  __syncthreads();
  return 0;
}

// --------------------------------------------------------- Cholesky factor
// Lower Cholesky of W (only the lower triangle is read and written).
// Returns 0 or k+1 where the pivot is not > 0 (incl. NaN).
template <typename T>
__device__ int cta_chol_factor(T* W, int ldw, int n, T* smem, int nb, CtaRed& red) {
  T* Pn = smem;
  for (int k0 = 0; k0 < n; k0 += nb) {
    const int kb = min(nb, n - k0), m = n - k0;
    T* Bs = smem + (size_t)m * nb;
    __syncthreads();
    for (int e = threadIdx.x; e < m * kb; e += kThreads) {
      int r = e % m, c = e / m;
      Pn[(size_t)c * m + r] = (r >= c) ? W[(size_t)(k0 + c) * ldw + k0 + r] : T(0);
    }
    __syncthreads();
    for (int c = 0; c < kb; ++c) {
      const T d = Pn[(size_t)c * m + c];
      if (!(d > T(0))) {
        __syncthreads();
        return k0 + c + 1;
      }
      const T ljj = sqrt(d);
      const T inv = T(1) / ljj;
      __syncthreads();
      for (int r = c + threadIdx.x; r < m; r += kThreads)
        Pn[(size_t)c * m + r] = (r == c) ? ljj : Pn[(size_t)c * m + r] * inv;
      __syncthreads();
      for (int r = c + 1 + threadIdx.x; r < m; r += kThreads) {
        const T l = Pn[(size_t)c * m + r];
        for (int cc = c + 1; cc < kb && cc <= r; ++cc)
          Pn[(size_t)cc * m + r] -= l * Pn[(size_t)c * m + cc];
      }
      __syncthreads();
    }
    for (int e = threadIdx.x; e < m * kb; e += kThreads) {
      int r = e % m, c = e / m;
      if (r >= c) W[(size_t)(k0 + c) * ldw + k0 + r] = Pn[(size_t)c * m + r];
    }
    __syncthreads();
    const int nr = n - k0 - kb;
    if (nr > 0) {
      // A22 -= L21 L21^T on the lower triangle.  B = L21^T is read from
      // the panel rows kb..m-1 written back to W: B(k, j) = L21(j, k).
      // Stage it transposed into a column-major kb x nr view through W's
      // upper triangle (unused by Cholesky): U(k0+k, k0+kb+j) = L21(j, k).
      for (int e = threadIdx.x; e < nr * kb; e += kThreads) {
        int j = e % nr, k = e / nr;
        W[(size_t)(k0 + kb + j) * ldw + k0 + k] = Pn[(size_t)k * m + kb + j];
      }
      __syncthreads();
      cta_gemm_sub<T>(W + (size_t)(k0 + kb) * ldw + k0 + kb, ldw, Pn + kb, m,
                      W + (size_t)(k0 + kb) * ldw + k0, ldw, nr, nr, kb, Bs, 0, true);
    }
  }
  __syncthreads();
  return 0;
}

// ------------------------------------------------------- triangular solves
// x (smem, n x nrhs, ld ldx) <- inv(E) x with E = trans ? M^T : M, M lower
// or upper (ld ldm), unit diagonal if `unit`.  Blocked by 32.
template <typename T, typename V>
__device__ void cta_tri_solve(const T* M, int ldm, int n, bool lower, bool trans, bool unit, V* x,
                              int ldx, int nrhs) {
  const bool elower = (lower != trans);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nblk = (n + 31) / 32;
  auto E = [&](int r, int c) -> V { return (V)(trans ? M[(size_t)r * ldm + c] : M[(size_t)c * ldm + r]); };
  for (int bi = 0; bi < nblk; ++bi) {
    const int blk = elower ? bi : nblk - 1 - bi;
    const int b0 = blk * 32, bs = min(32, n - b0);
    __syncthreads();
    if (w == 0) {  // diagonal block
      const int i = lane;
      for (int c = 0; c < nrhs; ++c) {
        V xi = (i < bs) ? x[(size_t)c * ldx + b0 + i] : V(0);
        for (int jj = 0; jj < bs; ++jj) {
          const int j = elower ? jj : bs - 1 - jj;
          if (i == j && !unit) xi = xi / E(b0 + i, b0 + i);
          V xj = __shfl_sync(0xffffffffu, xi, j);
          bool after = elower ? (i > j) : (i < j);
          if (after && i < bs) xi -= E(b0 + i, b0 + j) * xj;
        }
        if (i < bs) x[(size_t)c * ldx + b0 + i] = xi;
      }
    }
    __syncthreads();
    // rows not yet solved: x_r -= sum_{j in block} E(r, j) x_j
    const int r_lo = elower ? b0 + bs : 0, r_hi = elower ? n : b0;
    if (r_hi > r_lo) {
      if (!trans) {  // E(r, j) = M(r, j): coalesced over r
        for (int r = r_lo + threadIdx.x; r < r_hi; r += kThreads) {
          for (int c = 0; c < nrhs; ++c) {
            V s = V(0);
            for (int j = 0; j < bs; ++j) s += (V)M[(size_t)(b0 + j) * ldm + r] * x[(size_t)c * ldx + b0 + j];
            x[(size_t)c * ldx + r] -= s;
          }
        }
      } else {  // E(r, j) = M(j, r): warp per row, lanes over j
        for (int r = r_lo + w; r < r_hi; r += kWarps) {
          V m = (lane < bs) ? (V)M[(size_t)r * ldm + b0 + lane] : V(0);
          for (int c = 0; c < nrhs; ++c) {
            V s = warp_sum(m * ((lane < bs) ? x[(size_t)c * ldx + b0 + lane] : V(0)));
            if (lane == 0) x[(size_t)c * ldx + r] -= s;
          }
        }
      }
    }
  }
  __syncthreads();
}

// LU application: x <- inv(A) x (trans: inv(A)^T x) with A = P L U.
template <typename T, typename V>
__device__ void cta_lu_apply(const T* W, int ldw, int n, const int* piv, V* x, int ldx, int nrhs,
                             bool trans) {
  if (!trans) {
    __syncthreads();
    for (int c = threadIdx.x; c < nrhs; c += kThreads)
      for (int k = 0; k < n; ++k) {
        int p = piv[k];
        if (p != k) { V t = x[(size_t)c * ldx + k]; x[(size_t)c * ldx + k] = x[(size_t)c * ldx + p]; x[(size_t)c * ldx + p] = t; }
      }
    cta_tri_solve<T, V>(W, ldw, n, true, false, true, x, ldx, nrhs);
    cta_tri_solve<T, V>(W, ldw, n, false, false, false, x, ldx, nrhs);
  } else {
    cta_tri_solve<T, V>(W, ldw, n, false, true, false, x, ldx, nrhs);
    cta_tri_solve<T, V>(W, ldw, n, true, true, true, x, ldx, nrhs);
    __syncthreads();
    for (int c = threadIdx.x; c < nrhs; c += kThreads)
      for (int k = n - 1; k >= 0; --k) {
        int p = piv[k];
        if (p != k) { V t = x[(size_t)c * ldx + k]; x[(size_t)c * ldx + k] = x[(size_t)c * ldx + p]; x[(size_t)c * ldx + p] = t; }
      }
    __syncthreads();
  }
}

template <typename T, typename V>
__device__ void cta_chol_apply(const T* W, int ldw, int n, V* x, int ldx, int nrhs) {
  cta_tri_solve<T, V>(W, ldw, n, true, false, false, x, ldx, nrhs);
  cta_tri_solve<T, V>(W, ldw, n, true, true, false, x, ldx, nrhs);
}

// -------------------------------------------------------------- residual
// R = B - A X in FP64 (A: n x n ld lda, Xs: smem n x nrhs ld n), writes R to
// global (ld n) and returns per-column max |r| in rmax[c].
__device__ void cta_residual(const double* __restrict__ A, int lda, int n, const double* __restrict__ B,
                             const double* Xs, int nrhs, double* R, double* rmax_s, CtaRed& red) {
  constexpr int kRows = 4;
  double acc[kRows][8];
  const int t = threadIdx.x;
#pragma unroll
  for (int q = 0; q < kRows; ++q)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[q][c] = 0.0;
  for (int j = 0; j < n; ++j) {
    double xv[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) xv[c] = (c < nrhs) ? Xs[(size_t)c * n + j] : 0.0;
#pragma unroll
    for (int q = 0; q < kRows; ++q) {
      const int i = t + q * kThreads;
      if (i < n) {
        const double a = __ldg(A + (size_t)j * lda + i);
#pragma unroll
        for (int c = 0; c < 8; ++c)
          if (c < nrhs) acc[q][c] = fma(a, xv[c], acc[q][c]);
      }
    }
  }
  double mx[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) mx[c] = 0.0;
#pragma unroll
  for (int q = 0; q < kRows; ++q) {
    const int i = t + q * kThreads;
    if (i < n) {
#pragma unroll
      for (int c = 0; c < 8; ++c)
        if (c < nrhs) {
          double r = B[(size_t)c * n + i] - acc[q][c];
          R[(size_t)c * n + i] = r;
          mx[c] = fmax(mx[c], fabs(r));
        }
    }
  }
  for (int c = 0; c < nrhs; ++c) {
    double m = cta_max(mx[c], red);
    if (threadIdx.x == 0) rmax_s[c] = m;
  }
  __syncthreads();
}

// ------------------------------------------------------------ estimator
// 1-norm estimate of inv(A) (Hager 1984; Higham 1988): apply(v, trans)
// overwrites the smem vector v (length n) with inv(A) v or inv(A)^T v.
// xi: smem scratch of length n.
template <typename V, typename Apply>
__device__ double cta_est_inv_norm1(int n, V* v, V* xi, Apply apply, CtaRed& red) {
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += kThreads) v[i] = V(1) / V(n);
  apply(v, false);
  if (n == 1) {
    __syncthreads();
    double e = fabs((double)v[0]);
    __syncthreads();
    return e;
  }
  auto sum_abs = [&]() {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += kThreads) s += fabs((double)v[i]);
    return cta_sum(s, red);
  };
  double est = sum_abs();
  for (int i = threadIdx.x; i < n; i += kThreads) {
    V sg = v[i] >= V(0) ? V(1) : V(-1);
    xi[i] = sg;
    v[i] = sg;
  }
  apply(v, true);
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
    for (int i = threadIdx.x; i < n; i += kThreads) v[i] = (i == j) ? V(1) : V(0);
    apply(v, false);
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
    apply(v, true);
    double best2 = -1.0;
    int bi2 = 0x7fffffff;
    for (int i = threadIdx.x; i < n; i += kThreads) {
      double a = fabs((double)v[i]);
      if (a > best2) { best2 = a; bi2 = i; }
    }
    const int jn = cta_argmax_first<double>(best2, bi2, red);
    ++k;
    const double vj = (double)v[j], vjn = fabs((double)v[jn]);
    __syncthreads();
    if (vj == vjn || k > 5) break;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += kThreads) {
    V sgn = (i & 1) ? V(-1) : V(1);
    v[i] = sgn * (V(1) + V(i) / V(n - 1));
  }
  apply(v, false);
  const double temp = 2.0 * sum_abs() / (double)(3 * n);
  if (temp > est) est = temp;
  __syncthreads();
  return est;
}

__device__ __forceinline__ double rcond_from(double anorm, double ainvnm) {
  if (anorm == 0.0 || isinf(ainvnm) || ainvnm == 0.0) return 0.0;
  return (1.0 / ainvnm) / anorm;
}

}  // namespace asv
