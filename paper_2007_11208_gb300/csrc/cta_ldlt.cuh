// cta_ldlt.cuh -- symmetric-indefinite LDL^T with Bunch-Kaufman pivoting,
// performed by ONE thread block on one system (n <= 1024): the batched
// path's route for plain symmetric systems (the paper's closing remarks
// name them for specialised handling; opt-in flag ASOLVE_SYM_INDEF).
//
// The factorisation works on the lower triangle of the FP64 working copy,
// column by column: the pivot search (largest off-diagonal modulus of the
// column, then of the candidate's row and column) is a block reduction,
// the symmetric interchange and the rank-1 or rank-2 update of the trailing
// lower triangle are spread over the block (a warp per column, lanes over
// rows, so every access is coalesced).  Every product and sum is explicitly
// rounded (no fused multiply-add), in the order of the definition, so the
// pivot decisions and the factors are those of the plain CPU restatement of
// the same algorithm.  FP64 throughout: Bunch-Kaufman's 2 x 2 pivots are
// chosen for matrices far from definite, where low-precision factors would
// not serve refinement.
#pragma once
#include "cta_linalg.cuh"

namespace asv {
namespace {

// Fig. 4's symmetry test on its own: every pair within tol, absolute or
// relative.  A: n x n, ld n.
__device__ bool cta_is_symmetric(const double* __restrict__ A, int n, double tol) {
  bool ok = true;
  const int64_t tot = (int64_t)n * n;
  for (int64_t e = threadIdx.x; e < tot && ok; e += kThreads) {
    const int j = (int)(e / n), i = (int)(e - (int64_t)j * n);
    if (i > j) {
      const double aij = A[(size_t)j * n + i], aji = A[(size_t)i * n + j];
      const double delta = fabs(__dadd_rn(aij, -aji));
      const double mx = fabs(aij) > fabs(aji) ? fabs(aij) : fabs(aji);
      if (delta > tol && delta > __dmul_rn(tol, mx)) ok = false;
    }
  }
  return __syncthreads_and(ok) != 0;
}

__device__ __forceinline__ void dswap(double& a, double& b) {
  const double t = a;
  a = b;
  b = t;
}

// P A P^T = L D L^T of W (n x n, ld ldw; the lower triangle is read and
// overwritten).  piv[k] = kp >= 0: a 1 x 1 pivot with k and kp
// interchanged; piv[k] = piv[k+1] = -(kp+1): a 2 x 2 pivot at (k, k+1) with
// k+1 and kp interchanged.  wbuf: 2 x 1024 doubles of shared memory.
// Returns 0, or k+1 at the first exactly zero column (a zero 1 x 1 pivot).
__device__ __noinline__ int cta_ldlt_factor(double* W, int ldw, int n, int* piv, double* wbuf, CtaRed& red) {
  __shared__ int s_info;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double alpha = (1.0 + sqrt(17.0)) / 8.0;
  if (tid == 0) s_info = 0;
  __syncthreads();
  int k = 0;
  while (k < n) {
    double* ck = W + (size_t)k * ldw;
    // column k below the diagonal: first index of the largest modulus
    double best = -1.0;
    int bi = 0x7fffffff;
    for (int i = k + 1 + tid; i < n; i += kThreads) {
      const double a = fabs(ck[i]);
      if (a > best) { best = a; bi = i; }
    }
    const int im = cta_argmax_first<double>(best, bi, red);
    const bool has = im >= k + 1 && im < n;
    const int imax = has ? im : k;
    const double colmax = has ? fabs(ck[imax]) : 0.0;
    const double absakk = fabs(ck[k]);
    __syncthreads();
    if (absakk == 0.0 && colmax == 0.0) {  // a zero column: D(k) = 0
      if (tid == 0) {
        if (!s_info) s_info = k + 1;
        piv[k] = k;
      }
      __syncthreads();
      k += 1;
      continue;
    }
    int kp = k, kstep = 1;
    if (absakk < __dmul_rn(alpha, colmax)) {
      double rm = 0.0;
      for (int j = k + tid; j < imax; j += kThreads) rm = fmax(rm, fabs(W[(size_t)j * ldw + imax]));
      for (int i = imax + 1 + tid; i < n; i += kThreads) rm = fmax(rm, fabs(W[(size_t)imax * ldw + i]));
      const double rowmax = cta_max(rm, red);
      __syncthreads();
      if (absakk >= __dmul_rn(__dmul_rn(alpha, colmax), __ddiv_rn(colmax, rowmax))) kp = k;
      else if (fabs(W[(size_t)imax * ldw + imax]) >= __dmul_rn(alpha, rowmax)) kp = imax;
      else { kp = imax; kstep = 2; }
    }
    const int kk = k + kstep - 1;
    if (kp != kk) {  // symmetric interchange of kk and kp in the trailing lower triangle
      double* ckk = W + (size_t)kk * ldw;
      double* ckp = W + (size_t)kp * ldw;
      for (int i = kp + 1 + tid; i < n; i += kThreads) dswap(ckk[i], ckp[i]);
      for (int j = kk + 1 + tid; j < kp; j += kThreads) dswap(ckk[j], W[(size_t)j * ldw + kp]);
      if (tid == 0) {
        dswap(ckk[kk], ckp[kp]);
        if (kstep == 2) dswap(ck[k + 1], ck[kp]);
      }
      __syncthreads();
    }
    if (kstep == 1) {
      const double dk = ck[k];
      for (int j = k + 1 + tid; j < n; j += kThreads) wbuf[j] = __ddiv_rn(ck[j], dk);  // multipliers
      __syncthreads();
      for (int j = k + 1 + warp; j < n; j += kWarps) {  // A22 -= c l^T (lower)
        const double lj = wbuf[j];
        double* cj = W + (size_t)j * ldw;
        for (int i = j + lane; i < n; i += 32) cj[i] = __dadd_rn(cj[i], -__dmul_rn(ck[i], lj));
      }
      __syncthreads();
      for (int i = k + 1 + tid; i < n; i += kThreads) ck[i] = wbuf[i];
      if (tid == 0) piv[k] = kp;
    } else {
      // E = [a b; b c], E^-1 = [c -b; -b a] / (a c - b^2)
      const double* ck1 = W + (size_t)(k + 1) * ldw;
      const double a = ck[k], b = ck[k + 1], c = ck1[k + 1];
      const double det = __dadd_rn(__dmul_rn(a, c), -__dmul_rn(b, b));
      for (int j = k + 2 + tid; j < n; j += kThreads) {
        const double x = ck[j], y = ck1[j];
        wbuf[j] = __ddiv_rn(__dadd_rn(__dmul_rn(c, x), -__dmul_rn(b, y)), det);
        wbuf[1024 + j] = __ddiv_rn(__dadd_rn(__dmul_rn(a, y), -__dmul_rn(b, x)), det);
      }
      __syncthreads();
      for (int j = k + 2 + warp; j < n; j += kWarps) {  // A22 -= C E^-1 C^T (lower)
        const double w0 = wbuf[j], w1 = wbuf[1024 + j];
        double* cj = W + (size_t)j * ldw;
        for (int i = j + lane; i < n; i += 32)
          cj[i] = __dadd_rn(__dadd_rn(cj[i], -__dmul_rn(ck[i], w0)), -__dmul_rn(ck1[i], w1));
      }
      __syncthreads();
      for (int j = k + 2 + tid; j < n; j += kThreads) {
        ck[j] = wbuf[j];
        W[(size_t)(k + 1) * ldw + j] = wbuf[1024 + j];
      }
      if (tid == 0) piv[k] = piv[k + 1] = -(kp + 1);
    }
    __syncthreads();
    k += kstep;
  }
  const int info = s_info;
  __syncthreads();
  return info;
}

// x (n x nrhs, ld ldx, shared memory) <- inv(A) x with the LDL^T factors:
// L D y = P b by columns, then L^T, then the interchanges undone in reverse.
// One warp works (the steps form one chain); the block waits.
__device__ __noinline__ void cta_ldlt_solve(const double* __restrict__ W, int ldw, int n,
                                            const int* __restrict__ piv, double* x, int ldx, int nrhs) {
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int c = 0; c < nrhs; ++c) {
      double* b = x + (size_t)c * ldx;
      int k = 0;
      while (k < n) {
        const double* ck = W + (size_t)k * ldw;
        if (piv[k] >= 0) {
          const int kp = piv[k];
          if (kp != k && lane == 0) dswap(b[k], b[kp]);
          __syncwarp();
          const double bk = b[k];
          for (int i = k + 1 + lane; i < n; i += 32) b[i] = __dadd_rn(b[i], -__dmul_rn(ck[i], bk));
          __syncwarp();
          if (lane == 0) b[k] = __ddiv_rn(bk, ck[k]);
          __syncwarp();
          k += 1;
        } else {
          const int kp = -piv[k] - 1;
          const double* ck1 = W + (size_t)(k + 1) * ldw;
          if (kp != k + 1 && lane == 0) dswap(b[k + 1], b[kp]);
          __syncwarp();
          const double y0 = b[k], y1 = b[k + 1];
          for (int i = k + 2 + lane; i < n; i += 32)
            b[i] = __dadd_rn(__dadd_rn(b[i], -__dmul_rn(ck[i], y0)), -__dmul_rn(ck1[i], y1));
          __syncwarp();
          if (lane == 0) {
            const double a = ck[k], bb = ck[k + 1], cc = ck1[k + 1];
            const double det = __dadd_rn(__dmul_rn(a, cc), -__dmul_rn(bb, bb));
            b[k] = __ddiv_rn(__dadd_rn(__dmul_rn(cc, y0), -__dmul_rn(bb, y1)), det);
            b[k + 1] = __ddiv_rn(__dadd_rn(__dmul_rn(a, y1), -__dmul_rn(bb, y0)), det);
          }
          __syncwarp();
          k += 2;
        }
      }
      k = n - 1;
      while (k >= 0) {
        if (piv[k] >= 0) {
          const double* ck = W + (size_t)k * ldw;
          double s = 0.0;
          for (int i = k + 1 + lane; i < n; i += 32) s += ck[i] * b[i];
          s = warp_sum(s);
          if (lane == 0) {
            b[k] -= s;
            const int kp = piv[k];
            if (kp != k) dswap(b[k], b[kp]);
          }
          __syncwarp();
          k -= 1;
        } else {  // the 2 x 2 block (k-1, k)
          const double* ck = W + (size_t)k * ldw;
          const double* cm = W + (size_t)(k - 1) * ldw;
          double s1 = 0.0, s0 = 0.0;
          for (int i = k + 1 + lane; i < n; i += 32) {
            s1 += ck[i] * b[i];
            s0 += cm[i] * b[i];
          }
          s1 = warp_sum(s1);
          s0 = warp_sum(s0);
          if (lane == 0) {
            b[k] -= s1;
            b[k - 1] -= s0;
            const int kp = -piv[k] - 1;
            if (kp != k) dswap(b[k], b[kp]);
          }
          __syncwarp();
          k -= 2;
        }
      }
    }
  }
  __syncthreads();
}

}  // namespace
}  // namespace asv
