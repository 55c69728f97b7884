// band_large.cu -- the banded route (Sec. 2.1) for one system of any order:
// a matrix given in band storage (asolve_solve_band), or a dense matrix the
// scan classified as banded with n > 1024.  xGBTRF / xGBTRS / xGBCON
// semantics: LU with partial pivoting inside the band (U fills out to kl+ku
// super-diagonals), the solve with those factors, and the Hager/Higham
// 1-norm estimate of inv(A) through them.
//
// The elimination is a chain of n dependent column steps, so one warp runs
// it and the kernels are built around the latency of one step:
//   k_band_lu_win  the active window of the factor (columns j .. j+kl+ku)
//                  lives in shared memory; columns stream in with cp.async
//                  a few steps ahead and go back to global memory once final;
//   k_band_solve   one warp per right-hand side: the window of the vector
//                  being eliminated sits in registers across the lanes (one
//                  element per lane and register), the factor columns
//                  stream through a cp.async ring;
//   k_band_est     the estimate, driven on the device by one warp with the
//                  same sweeps.
// From n = 2048 on (windows of up to 72 elements) the solve and the estimate
// instead run the partitioned sweeps (k_sw_*): each sweep is a linear
// recurrence, evaluated block-parallel through per-block transfer maps and
// one chained scan, with the estimate's iteration driven from the host
// (est_host.cuh).  Bandwidths beyond the windows fall back to the warp
// routines that work on global memory directly (band_warp.cuh).  Scan,
// packing and the FP64 backward error are ordinary data-parallel kernels.
//
// Long systems (n >= 4096) that are diagonally dominant by rows or by
// columns take a partitioned route instead (unless ASOLVE_BAND_SPIKE=0 is
// set in the environment) (band_spike.cuh, k_spk_*): blocks factored in parallel
// without pivoting, one small system per block boundary, and solves with A
// and A^T in three block-parallel steps; a zero pivot, a singular boundary
// system or spikes that have not decayed across a block send the system
// back to the path above.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <stdlib.h>

#include "band_spike.cuh"
#include "band_warp.cuh"
#include "est_host.cuh"

namespace asv {

namespace {

constexpr size_t kWinSmemMax = 200 * 1024;
constexpr size_t kTailBytes = 16384;  // scan record, scalars and per-column maxima (nrhs <= 256)

#define BCK(x)                                        \
  do {                                                \
    cudaError_t _e = (x);                             \
    if (_e != cudaSuccess) {                          \
      cudaGetLastError();                             \
      return _e == cudaErrorMemoryAllocation ? ASOLVE_E_NOMEM : ASOLVE_E_CUDA; \
    }                                                 \
  } while (0)

// ------------------------------------------------------------ scan / pack
struct BandScan {
  int kl, ku, nonfinite, b_nonfinite;
  unsigned long long norm1, norminf;  // bit patterns of non-negative doubles
};

// True bandwidths inside the declared band, non-finite flags, and the 1- and
// inf-norms (Sec. 2.1 finds kl, ku by the last non-zero diagonal).
__global__ void k_bscan(const double* __restrict__ AB, int64_t ldab, int kld, int kud, int64_t n,
                        const double* __restrict__ B, int64_t nb, BandScan* out) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int kl = 0, ku = 0, bad = 0;
  double n1 = 0.0, ninf = 0.0;
  for (int64_t j = tid; j < n; j += stride) {
    const int64_t lo = j - kud > 0 ? j - kud : 0, hi = j + kld < n - 1 ? j + kld : n - 1;
    double cs = 0.0;
    for (int64_t i = lo; i <= hi; ++i) {
      const double v = AB[(size_t)(kud + i - j) + (size_t)j * ldab];
      if (is_nonfinite_bits(dbits(v))) bad = 1;
      if (is_nonzero_bits(dbits(v))) {
        if (i > j && (int)(i - j) > kl) kl = (int)(i - j);
        if (j > i && (int)(j - i) > ku) ku = (int)(j - i);
      }
      cs += fabs(v);
    }
    n1 = fmax(n1, cs);
  }
  for (int64_t i = tid; i < n; i += stride) {
    const int64_t lo = i - kld > 0 ? i - kld : 0, hi = i + kud < n - 1 ? i + kud : n - 1;
    double rs = 0.0;
    for (int64_t j = lo; j <= hi; ++j) rs += fabs(AB[(size_t)(kud + i - j) + (size_t)j * ldab]);
    ninf = fmax(ninf, rs);
  }
  int bbad = 0;
  for (int64_t e = tid; e < nb; e += stride)
    if (is_nonfinite_bits(dbits(B[e]))) bbad = 1;
  kl = warp_max(kl);
  ku = warp_max(ku);
  bad = warp_max(bad);
  bbad = warp_max(bbad);
  n1 = warp_max(n1);
  ninf = warp_max(ninf);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&out->kl, kl);
    atomicMax(&out->ku, ku);
    atomicMax(&out->nonfinite, bad);
    atomicMax(&out->b_nonfinite, bbad);
    atomicMax(&out->norm1, (unsigned long long)dbits(n1));
    atomicMax(&out->norminf, (unsigned long long)dbits(ninf));
  }
}

// Band factor storage F (ldf = 2kl+ku+1, kv = kl+ku): A(i,j) at
// F[(kv+i-j) + j*ldf]; rows 0..kl-1 (the fill of U) start at zero.
__global__ void k_bpack(const double* __restrict__ AB, int64_t ldab, int kud, const double* __restrict__ A,
                        int64_t n, int kl, int ku, double* __restrict__ F) {
  const int ldf = 2 * kl + ku + 1, kv = kl + ku;
  const int64_t total = (int64_t)ldf * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % ldf);
    const int64_t j = e / ldf, i = r - kv + j;
    double v = 0.0;
    if (r >= kl && i >= 0 && i < n) v = A ? A[(size_t)j * n + i] : AB[(size_t)(kud + i - j) + (size_t)j * ldab];
    F[e] = v;
  }
}

__global__ void k_band_to_dense(const double* __restrict__ AB, int64_t ldab, int kld, int kud, int64_t n,
                                double* __restrict__ A) {
  const int64_t total = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / n, i = e % n;
    A[e] = (i - j <= kld && j - i <= kud) ? AB[(size_t)(kud + i - j) + (size_t)j * ldab] : 0.0;
  }
}

// ------------------------------------------------------------ factor
constexpr int kFlatNP = 8;  // update pairs per lane of the narrow-band factorisation

// GBTRF on F with the active window in shared memory: S = kv+1+kD column
// slots of ldf doubles; column c lives in slot c % S while it is active.
__global__ void __launch_bounds__(32) k_band_lu_win(double* __restrict__ F, int ldf, int n, int kl, int ku,
                                                    int* __restrict__ piv, int* __restrict__ fail) {
  extern __shared__ double win[];
  const int lane = threadIdx.x;
  const int kv = kl + ku, S = kv + 1 + kD;
  auto slot = [&](int c) { return win + (size_t)(c % S) * ldf; };
  // columns 0 .. S-1 in flight, one commit group each
  for (int c = 0; c < S; ++c) {
    if (c < n)
      for (int r = lane; r < ldf; r += 32) cp_async8(slot(c) + r, F + (size_t)c * ldf + r);
    cp_commit();
  }
  // narrow bands: the kl x kv update pairs spread over the lanes, at most
  // kFlatNP per lane (pair e: row 1 + e % kl, column e / kl after j)
  const bool flat = kl >= 1 && kl * kv <= 32 * kFlatNP;
  int ft[kFlatNP], fc[kFlatNP];
#pragma unroll
  for (int i = 0; i < kFlatNP; ++i) {
    const int e = lane + 32 * i;
    const bool on = flat && e < kl * kv;
    ft[i] = on ? 1 + e % kl : 0;
    fc[i] = on ? e / kl : 0;
  }
  int ju = 0;
  for (int j = 0; j < n; ++j) {
    // column j + kv is the last one step j touches: kD newer groups may pend
    cp_wait<kD>();
    __syncwarp();
    double* cj = slot(j);
    const int km = min(kl, n - 1 - j);
    // the first largest |a(j+t, j)|, t = 0..km, in passes of 32 candidates
    int bi = -1;
    unsigned long long kbest = 0ull;
    for (int t0 = 0; t0 <= km; t0 += 32) {
      const int t = t0 + lane;
      unsigned long long kp;
      const int l = warp_first_max_key(t <= km ? abs_key(cj[kv + t]) : 0ull, kp);
      if (l >= 0 && kp > kbest) { kbest = kp; bi = t0 + l; }
    }
    if (bi < 0 || bi > km || !(cj[kv + bi] != 0.0)) {  // exact zero (or invalid) pivot
      if (lane == 0) *fail = j + 1;
      cp_wait_all();
      __syncwarp();
      // leave the columns already final in F; the factor is not used
      return;
    }
    if (lane == 0) piv[j] = j + bi;
    ju = max(ju, min(j + ku + bi, n - 1));
    if (bi != 0)
      for (int c = j + lane; c <= ju; c += 32) {
        double* cc = slot(c);
        const double t0 = cc[kv + j - c];
        cc[kv + j - c] = cc[kv + j + bi - c];
        cc[kv + j + bi - c] = t0;
      }
    __syncwarp();
    const double inv = 1.0 / cj[kv];
    for (int t = 1 + lane; t <= km; t += 32) cj[kv + t] *= inv;
    __syncwarp();
    // rank-1 update of rows j+1..j+km, columns j+1..ju
    if (flat) {  // lane <-> fixed (row, column) pairs of the window
      const int sj = j % S;
#pragma unroll
      for (int i = 0; i < kFlatNP; ++i) {
        const int t = ft[i], cc = fc[i];
        int sl = sj + 1 + cc;
        if (sl >= S) sl -= S;
        if (t > 0 && t <= km && j + 1 + cc <= ju) {
          double* col = win + (size_t)sl * ldf + kv - 1 - cc;  // col[0]: row j of column j+1+cc
          col[t] = fma(-cj[kv + t], col[0], col[t]);
        }
      }
    } else {  // lane <-> row
      for (int t0 = 1; t0 <= km; t0 += 32) {
        const int t = t0 + lane;
        const bool on = t <= km;
        const double l = on ? cj[kv + t] : 0.0;
        int sc = (j + 1) % S;
#pragma unroll 4
        for (int c = j + 1; c <= ju; ++c) {
          double* cc = win + (size_t)sc * ldf;
          const double u = cc[kv + j - c];
          if (on) cc[kv + j + t - c] = fma(-l, u, cc[kv + j + t - c]);
          sc = (sc + 1 == S) ? 0 : sc + 1;
        }
      }
    }
    __syncwarp();
    // column j is final
    for (int r = lane; r < ldf; r += 32) F[(size_t)j * ldf + r] = cj[r];
    __syncwarp();
    const int cn = j + S;
    if (cn < n)
      for (int r = lane; r < ldf; r += 32) cp_async8(cj + r, F + (size_t)cn * ldf + r);
    cp_commit();
  }
  cp_wait_all();
  // columns still resident are final too (they were written above as j passed)
}

// The general-bandwidth fallback: the warp routine on global memory.
__global__ void __launch_bounds__(32) k_band_lu_glob(double* F, int ldf, int n, int kl, int ku, int* piv,
                                                     int* fail) {
  WarpBand b;
  b.F = F;
  b.piv = piv;
  b.n = n;
  b.kl = kl;
  b.ku = ku;
  b.kv = kl + ku;
  b.ldf = ldf;
  const int f = warp_band_lu(b);
  if ((threadIdx.x & 31) == 0 && f) *fail = f;
}

template <int R>
__global__ void __launch_bounds__(32) k_band_solve(const double* F, int ldf, int n, int kl, int ku, const int* piv,
                                                   double* X) {
  __shared__ double ring[kD * (32 * kMaxR + 2)];
  __shared__ int pring[kD];
  band_apply<R>(F, ldf, n, kl, ku, piv, X + (size_t)blockIdx.x * n, ring, pring);
}

// General-bandwidth fallback of the solve (global-memory warp routine).
__global__ void __launch_bounds__(32) k_band_solve_glob(double* F, int ldf, int n, int kl, int ku, int* piv,
                                                        double* X) {
  WarpBand b;
  b.F = F;
  b.piv = piv;
  b.n = n;
  b.kl = kl;
  b.ku = ku;
  b.kv = kl + ku;
  b.ldf = ldf;
  warp_band_apply(b, X + (size_t)blockIdx.x * n, false);
}

// ------------------------------------------------------------ estimate
// 1-norm estimate of inv(A) (Hager 1984, Higham 1988) with the band factors,
// driven by one warp: the same iteration as the other routes' estimators.
template <int R, bool GLOB>
__global__ void __launch_bounds__(32) k_band_est(double* F, int ldf, int n, int kl, int ku, int* piv, double* v,
                                                 double* xi, double* out) {
  __shared__ double ring[kD * (32 * kMaxR + 2)];
  __shared__ int pring[kD];
  const int lane = threadIdx.x & 31;
  WarpBand b;
  b.F = F;
  b.piv = piv;
  b.n = n;
  b.kl = kl;
  b.ku = ku;
  b.kv = kl + ku;
  b.ldf = ldf;
  auto apply = [&](bool trans) {
    __syncwarp();
    __threadfence();
    if (GLOB) warp_band_apply(b, v, trans);
    else if (trans) band_apply_t<R>(F, ldf, n, kl, ku, piv, v, ring, pring);
    else band_apply<R>(F, ldf, n, kl, ku, piv, v, ring, pring);
    __syncwarp();
    __threadfence();
  };
  auto sum_abs = [&]() {
    double s = 0.0;
    for (int i = lane; i < n; i += 32) s += fabs(v[i]);
    return warp_sum_d(s);
  };
  auto argmax = [&]() {
    double best = -1.0;
    int bi = 0x7fffffff;
    for (int i = lane; i < n; i += 32) {
      const double a = fabs(v[i]);
      if (a > best) { best = a; bi = i; }
    }
    warp_argmax_first(best, bi);
    return bi;
  };
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  for (int i = lane; i < n; i += 32) v[i] = 1.0 / (double)n;
  apply(false);
  if (n == 1) {
    if (lane == 0) *out = fabs(v[0]);
    return;
  }
  double est = sum_abs();
  for (int i = lane; i < n; i += 32) {
    const double sg = v[i] >= 0.0 ? 1.0 : -1.0;
    xi[i] = sg;
    v[i] = sg;
  }
  apply(true);
  int k = 2;
  for (;;) {
    const int j = argmax();
    if (j < 0 || j >= n) {
      est = nan;
      break;
    }
    __syncwarp();
    for (int i = lane; i < n; i += 32) v[i] = (i == j) ? 1.0 : 0.0;
    apply(false);
    const double estold = est;
    est = sum_abs();
    bool same = true;
    for (int i = lane; i < n; i += 32)
      if ((v[i] >= 0.0 ? 1.0 : -1.0) != xi[i]) same = false;
    same = __all_sync(0xffffffffu, same);
    if (same || est <= estold) break;
    for (int i = lane; i < n; i += 32) {
      const double sg = v[i] >= 0.0 ? 1.0 : -1.0;
      xi[i] = sg;
      v[i] = sg;
    }
    apply(true);
    const int jn = argmax();
    ++k;
    if (jn < 0 || jn >= n) {
      est = nan;
      break;
    }
    const double vj = v[j], vjn = fabs(v[jn]);
    __syncwarp();
    if (vj == vjn || k > 5) break;
  }
  if (est == est) {
    __syncwarp();
    for (int i = lane; i < n; i += 32) v[i] = ((i & 1) ? -1.0 : 1.0) * (1.0 + (double)i / (double)(n - 1));
    apply(false);
    const double temp = 2.0 * sum_abs() / (double)(3 * n);
    if (temp > est) est = temp;
  }
  if (lane == 0) *out = est;
}

// ------------------------------------------------------------ berr
// Per column: max |b - A x|, max |x|, max |b| (FP64; A read in its input form).
// r = b - A x for one right-hand side (A in band storage or dense), and
// x += d, the refinement steps of the partitioned sweeps.
__global__ void k_band_resid(const double* __restrict__ AB, int64_t ldab, int kud, const double* __restrict__ A,
                             int64_t n, int kl, int ku, const double* __restrict__ b, const double* __restrict__ x,
                             double* __restrict__ r) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t lo = i - kl > 0 ? i - kl : 0, hi = i + ku < n - 1 ? i + ku : n - 1;
    double acc = 0.0;
    for (int64_t j = lo; j <= hi; ++j) {
      const double a = A ? A[(size_t)j * n + i] : AB[(size_t)(kud + i - j) + (size_t)j * ldab];
      acc = fma(a, x[j], acc);
    }
    r[i] = b[i] - acc;
  }
}
__global__ void k_band_xadd(double* __restrict__ x, const double* __restrict__ d, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += d[i];
}

__global__ void k_band_berr(const double* __restrict__ AB, int64_t ldab, int kud, const double* __restrict__ A,
                            int64_t n, int kl, int ku, const double* __restrict__ B, const double* __restrict__ X,
                            int nrhs, unsigned long long* colmax) {
  const int c = blockIdx.y;
  const double* b = B + (size_t)c * n;
  const double* x = X + (size_t)c * n;
  double rm = 0.0, xm = 0.0, bm = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t lo = i - kl > 0 ? i - kl : 0, hi = i + ku < n - 1 ? i + ku : n - 1;
    double acc = 0.0;
    for (int64_t j = lo; j <= hi; ++j) {
      const double a = A ? A[(size_t)j * n + i] : AB[(size_t)(kud + i - j) + (size_t)j * ldab];
      acc = fma(a, x[j], acc);
    }
    rm = fmax(rm, fabs(b[i] - acc));
    xm = fmax(xm, fabs(x[i]));
    bm = fmax(bm, fabs(b[i]));
  }
  rm = warp_max(rm);
  xm = warp_max(xm);
  bm = warp_max(bm);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(colmax + c, (unsigned long long)dbits(rm));
    atomicMax(colmax + nrhs + c, (unsigned long long)dbits(xm));
    atomicMax(colmax + 2 * nrhs + c, (unsigned long long)dbits(bm));
  }
}

// ------------------------------------------------ partitioned sweeps
// The solve with the band factors is four linear recurrences (sweeps) that
// carry a window of the vector from step to step:
//   SW_L  forward, step j = 0..n-1: window x[j..j+kl]; interchange with row
//         piv[j], eliminate rows j+1.. with column j of L; out x[j]; in x[j+kl+1]
//   SW_U  backward, i = n-1..0: element q = y[i-q], q <= kv; x_i = w0 / u_ii,
//         w_q -= u(i-q, i) x_i; out x[i]; in y[i-kv-1]
//   SW_UT forward, i = 0..n-1: w0 = b_i, w_q = z_{i-q}; z_i = (w0 - sum_q
//         u(i-q, i) w_q) / u_ii; out z_i; in b_{i+1}
//   SW_LT backward, j = n-1..0: window x[j..j+kl]; w0 -= sum_t l(j+t, j) w_t,
//         interchange with row piv[j]; out x[j+kl]; in x[j-1] (the last step
//         flushes x[0..kl])
// Each step is affine in the window, so the n steps are cut into P blocks:
//   maps: for every block, the window after it from each unit starting
//         window with no inputs (one lane each) -- the block's matrix T_b;
//         it depends on the factors only and is kept for every solve;
//   part: from a zero window with the block's inputs -- the vector t_b;
//   scan: one CTA chains W_{b+1} = T_b W_b + t_b from the true first window;
//   out:  every block reruns its steps from W_b and writes its outputs.
// The steps are those of the sequential sweeps; only the order in which
// the contributions of earlier blocks are summed changes.
enum : int { SW_L = 0, SW_U = 1, SW_UT = 2, SW_LT = 3 };

struct SweepCtx {
  const double* F;
  int ldf, n, kl, ku;
  const int* piv;
  int L, P;  // steps per block, blocks
};

__host__ __device__ __forceinline__ int sw_ws(int kind, int kl, int ku) {
  return (kind == SW_L || kind == SW_LT) ? kl + 1 : kl + ku + 1;
}

// one step of sweep KIND on the window w (element e in w[e], WM >= window
// size); xin: inputs (null: none), out: outputs (null: not written)
template <int KIND, int WM>
__device__ __forceinline__ void sw_step(const SweepCtx& c, double (&w)[WM], int s, const double* __restrict__ xin,
                                        double* __restrict__ out) {
  const int n = c.n, kl = c.kl, kv = c.kl + c.ku;
  if (KIND == SW_L) {
    const int j = s;
    const double* col = c.F + (size_t)j * c.ldf + kv;  // col[t] = l(j+t, j)
    const int km = min(kl, n - 1 - j);
    const int d = __ldg(c.piv + j) - j;
    const double e0 = w[0];
    double ed = e0;
#pragma unroll
    for (int t = 1; t < WM; ++t) ed = (t == d) ? w[t] : ed;
#pragma unroll
    for (int t = 1; t < WM; ++t) w[t] = (t == d) ? e0 : w[t];
    w[0] = ed;
#pragma unroll
    for (int t = 1; t < WM; ++t)
      if (t <= km) w[t] = fma(-__ldg(col + t), ed, w[t]);
    if (out) out[j] = ed;
#pragma unroll
    for (int t = 0; t + 1 < WM; ++t) w[t] = w[t + 1];
    w[WM - 1] = 0.0;
    const double in = (xin && j + kl + 1 < n) ? xin[j + kl + 1] : 0.0;
#pragma unroll
    for (int t = 0; t < WM; ++t) w[t] = (t == kl) ? in : w[t];
  } else if (KIND == SW_U) {
    const int i = n - 1 - s;
    const double* col = c.F + (size_t)i * c.ldf + kv;  // col[-q] = u(i-q, i)
    const int lim = min(kv, i);
    const double xi = w[0] / __ldg(col);
#pragma unroll
    for (int q = 1; q < WM; ++q)
      if (q <= lim) w[q] = fma(-__ldg(col - q), xi, w[q]);
    if (out) out[i] = xi;
#pragma unroll
    for (int q = 0; q + 1 < WM; ++q) w[q] = w[q + 1];
    w[WM - 1] = 0.0;
    const double in = (xin && i - kv - 1 >= 0) ? xin[i - kv - 1] : 0.0;
#pragma unroll
    for (int q = 0; q < WM; ++q) w[q] = (q == kv) ? in : w[q];
  } else if (KIND == SW_UT) {
    const int i = s;
    const double* col = c.F + (size_t)i * c.ldf + kv;
    const int lim = min(kv, i);
    double acc = 0.0;
#pragma unroll
    for (int q = 1; q < WM; ++q)
      if (q <= lim) acc = fma(__ldg(col - q), w[q], acc);
    const double zi = (w[0] - acc) / __ldg(col);
    if (out) out[i] = zi;
    w[0] = zi;
#pragma unroll
    for (int q = WM - 1; q >= 1; --q) w[q] = (q <= kv) ? w[q - 1] : 0.0;
    w[0] = (xin && i + 1 < n) ? xin[i + 1] : 0.0;
  } else {  // SW_LT
    const int j = n - 1 - s;
    const double* col = c.F + (size_t)j * c.ldf + kv;
    const int km = min(kl, n - 1 - j);
    double acc = 0.0;
#pragma unroll
    for (int t = 1; t < WM; ++t)
      if (t <= km) acc = fma(__ldg(col + t), w[t], acc);
    const double v = w[0] - acc;
    const int d = __ldg(c.piv + j) - j;
    double ed = v;
#pragma unroll
    for (int t = 1; t < WM; ++t) ed = (t == d) ? w[t] : ed;
#pragma unroll
    for (int t = 1; t < WM; ++t) w[t] = (t == d) ? v : w[t];
    w[0] = ed;
    if (j == 0) {
      if (out)
#pragma unroll
        for (int t = 0; t < WM; ++t)
          if (t <= kl && t < n) out[t] = w[t];
      return;
    }
    if (out && j + kl < n) {
      double ek = 0.0;
#pragma unroll
      for (int t = 0; t < WM; ++t) ek = (t == kl) ? w[t] : ek;
      out[j + kl] = ek;
    }
#pragma unroll
    for (int t = WM - 1; t >= 1; --t) w[t] = (t <= kl) ? w[t - 1] : 0.0;
    w[0] = xin ? xin[j - 1] : 0.0;
  }
}

// maps: T[b][col][r] = element r of the window after block b from unit
// window e_col (no inputs); grid (P, ceil(ws / 32)), 32 threads
template <int KIND, int WM>
__global__ void __launch_bounds__(32) k_sw_maps(SweepCtx c, int ws, double* __restrict__ T) {
  const int b = blockIdx.x, col = blockIdx.y * 32 + threadIdx.x;
  if (col >= ws) return;
  double w[WM];
#pragma unroll
  for (int e = 0; e < WM; ++e) w[e] = (e == col) ? 1.0 : 0.0;
  const int s0 = b * c.L, s1 = min(c.n, s0 + c.L);
  for (int s = s0; s < s1; ++s) sw_step<KIND, WM>(c, w, s, nullptr, nullptr);
  double* o = T + ((size_t)b * ws + col) * ws;
#pragma unroll
  for (int e = 0; e < WM; ++e)
    if (e < ws) o[e] = w[e];
}

// part: tv[b][r] = element r of the window after block b from a zero window
// with the block's inputs; one thread per block
template <int KIND, int WM>
__global__ void __launch_bounds__(128) k_sw_part(SweepCtx c, int ws, const double* __restrict__ xin,
                                                 double* __restrict__ tv) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= c.P) return;
  double w[WM];
#pragma unroll
  for (int e = 0; e < WM; ++e) w[e] = 0.0;
  const int s0 = b * c.L, s1 = min(c.n, s0 + c.L);
  for (int s = s0; s < s1; ++s) sw_step<KIND, WM>(c, w, s, xin, nullptr);
#pragma unroll
  for (int e = 0; e < WM; ++e)
    if (e < ws) tv[(size_t)b * ws + e] = w[e];
}

// scan: one CTA; Ws[b] = the true window before block b.  T_b and t_b
// stream through a three-stage cp.async ring.
constexpr int kSwScanThreads = 128;
__host__ __device__ constexpr size_t sw_scan_smem(int ws) { return sizeof(double) * 3 * ((size_t)ws * ws + ws) + 2 * sizeof(double) * 128; }
template <int KIND>
__global__ void __launch_bounds__(kSwScanThreads) k_sw_scan(SweepCtx c, int ws, const double* __restrict__ xin,
                                                           const double* __restrict__ T,
                                                           const double* __restrict__ tv, double* __restrict__ Ws) {
  extern __shared__ __align__(16) double sm[];
  const int stage = ws * ws + ws;
  double* W = sm + 3 * (size_t)stage;  // current window (128 slots)
  const int tid = threadIdx.x, n = c.n, kl = c.kl, kv = c.kl + c.ku;
  auto issue = [&](int b) {
    if (b < c.P) {
      double* dst = sm + (size_t)(b % 3) * stage;
      const double* srcT = T + (size_t)b * ws * ws;
      for (int e = tid; e < ws * ws; e += kSwScanThreads) cp_async8(dst + e, srcT + e);
      for (int e = tid; e < ws; e += kSwScanThreads) cp_async8(dst + ws * ws + e, tv + (size_t)b * ws + e);
    }
    cp_commit();
  };
  issue(0);
  issue(1);
  if (tid < ws) {
    double v = 0.0;
    if (KIND == SW_L) v = (tid <= kl && tid < n) ? xin[tid] : 0.0;
    else if (KIND == SW_U) v = (tid <= kv && n - 1 - tid >= 0) ? xin[n - 1 - tid] : 0.0;
    else if (KIND == SW_UT) v = (tid == 0) ? xin[0] : 0.0;
    else v = (tid == 0) ? xin[n - 1] : 0.0;
    W[tid] = v;
  }
  for (int b = 0; b < c.P; ++b) {
    issue(b + 2);
    cp_wait<2>();
    __syncthreads();
    const double* st = sm + (size_t)(b % 3) * stage;
    double nw = 0.0;
    if (tid < ws) {
      Ws[(size_t)b * ws + tid] = W[tid];
      nw = st[ws * ws + tid];
      for (int col = 0; col < ws; ++col) nw = fma(st[col * ws + tid], W[col], nw);
    }
    __syncthreads();
    if (tid < ws) W[tid] = nw;
  }
  cp_wait_all();
}

// out: block b reruns its steps from Ws[b] with its inputs and writes its
// outputs; one thread per block
template <int KIND, int WM>
__global__ void __launch_bounds__(128) k_sw_out(SweepCtx c, int ws, const double* __restrict__ xin,
                                                const double* __restrict__ Ws, double* __restrict__ xout) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= c.P) return;
  double w[WM];
#pragma unroll
  for (int e = 0; e < WM; ++e) w[e] = (e < ws) ? Ws[(size_t)b * ws + e] : 0.0;
  const int s0 = b * c.L, s1 = min(c.n, s0 + c.L);
  for (int s = s0; s < s1; ++s) sw_step<KIND, WM>(c, w, s, xin, xout);
}

constexpr int kSwMaxWs = 72;     // widest window of the partitioned sweeps
constexpr int64_t kSwMinN = 2048;  // shorter systems keep the one-warp sweeps
constexpr int kSwRefineSteps = 3;  // refinement steps after the sweeps before the sequential solve

struct SweepPlan {
  SweepCtx c;
  double* T[4];   // maps of the four sweeps
  double* tv;     // P x ws_max
  double* Ws;     // P x ws_max
  double* tmp;    // n
};

int sw_blocks(int64_t n) {
  int P = (int)sqrt(1.5 * (double)n);
  return P < 1 ? 1 : (P > 4096 ? 4096 : P);
}

size_t sw_bytes(int64_t n, int kl, int ku) {
  const int P0 = sw_blocks(n);
  const int L = (int)((n + P0 - 1) / P0);
  const int P = (int)((n + L - 1) / L);
  size_t b = 0;
  for (int k = 0; k < 4; ++k) {
    const size_t ws = (size_t)sw_ws(k, kl, ku);
    b += (sizeof(double) * (size_t)P * ws * ws + 255) & ~(size_t)255;
  }
  b += 2 * ((sizeof(double) * (size_t)P * (kl + ku + 1) + 255) & ~(size_t)255);
  b += (sizeof(double) * (size_t)n + 255) & ~(size_t)255;
  return b;
}

template <int KIND, int WM>
int sw_run_wm(const SweepPlan& pl, int ws, const double* xin, double* xout, bool maps, cudaStream_t st) {
  const SweepCtx& c = pl.c;
  if (maps) {
    k_sw_maps<KIND, WM><<<dim3((unsigned)c.P, (unsigned)((ws + 31) / 32)), 32, 0, st>>>(c, ws, pl.T[KIND]);
    BCK(cudaGetLastError());
    return ASOLVE_OK;
  }
  const unsigned g = (unsigned)((c.P + 127) / 128);
  k_sw_part<KIND, WM><<<g, 128, 0, st>>>(c, ws, xin, pl.tv);
  const size_t sm = sw_scan_smem(ws);
  BCK(ASV_SMEM_LIMIT_ONCE(k_sw_scan<KIND>, sw_scan_smem(kSwMaxWs)));
  k_sw_scan<KIND><<<1, kSwScanThreads, sm, st>>>(c, ws, xin, pl.T[KIND], pl.tv, pl.Ws);
  k_sw_out<KIND, WM><<<g, 128, 0, st>>>(c, ws, xin, pl.Ws, xout);
  BCK(cudaGetLastError());
  return ASOLVE_OK;
}

// one sweep (maps: precompute T of this sweep instead)
template <int KIND>
int sw_run(const SweepPlan& pl, const double* xin, double* xout, bool maps, cudaStream_t st) {
  const int ws = sw_ws(KIND, pl.c.kl, pl.c.ku);
  if (ws <= 8) return sw_run_wm<KIND, 8>(pl, ws, xin, xout, maps, st);
  if (ws <= 24) return sw_run_wm<KIND, 24>(pl, ws, xin, xout, maps, st);
  return sw_run_wm<KIND, kSwMaxWs>(pl, ws, xin, xout, maps, st);
}

// x <- inv(A) x (trans: inv(A)^T x) in place, through pl.tmp
int sw_apply(const SweepPlan& pl, double* x, bool trans, cudaStream_t st) {
  int rc;
  if (!trans) {
    if ((rc = sw_run<SW_L>(pl, x, pl.tmp, false, st))) return rc;
    return sw_run<SW_U>(pl, pl.tmp, x, false, st);
  }
  if ((rc = sw_run<SW_UT>(pl, x, pl.tmp, false, st))) return rc;
  return sw_run<SW_LT>(pl, pl.tmp, x, false, st);
}

int window_r(int kv) {
  const int need = (kv + 1 + 31) / 32;
  if (need <= 1) return 1;
  if (need <= 2) return 2;
  if (need <= 4) return 4;
  if (need <= 8) return 8;
  return 0;  // beyond the register window: global fallback
}

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

double rcond_from_est(double anorm, double est) {
  if (anorm == 0.0 || isinf(est) || est == 0.0) return 0.0;
  return (1.0 / est) / anorm;
}

// ------------------------------------------- partitioned route (dominant)
// Long band systems that are diagonally dominant by rows or by columns can
// be solved block-parallel without pivoting (band_spike.cuh).  The route is
// on by default; the environment variable ASOLVE_BAND_SPIKE=0 turns it off,
// and every band system then keeps the GBTRF-order path below.
constexpr int64_t kSpkMinN = 4096;      // shorter systems: the one-warp path
constexpr int64_t kSpkBlocks = 19456;   // target number of blocks (128 per SM: the block steps run a
                                        // thread, or a warp, per block)
constexpr double kSpkFarTol = 8.67e-19; // 2^-60: far spike tips dropped below this
constexpr int kSpkThreads = 128;

bool spike_enabled() {
  static int on = -1;
  if (on < 0) {
    const char* e = getenv("ASOLVE_BAND_SPIKE");
    on = (e && e[0] == '0' && e[1] == 0) ? 0 : 1;
  }
  return on == 1;
}

// Block length and count at attempt `level`: at least 16 (kl+ku) and 128
// rows per block (on the band workload's matrices the far tips fell below
// 2^-60 from about 16 (kl+ku) rows, but not within 64 rows at kl = ku = 2),
// doubled at each further attempt.
bool spike_shape(int64_t n, int kl, int ku, int level, int64_t* m, int64_t* P) {
  int64_t mm = n / kSpkBlocks;
  if (mm < 16 * (int64_t)(kl + ku)) mm = 16 * (int64_t)(kl + ku);
  if (mm < 128) mm = 128;
  mm <<= level;
  *m = mm;
  *P = n / mm;
  return *P >= 2;
}

// Sized for the first attempt, which has the most blocks.
size_t spike_bytes(int64_t n, int kl, int ku) {
  int64_t m, P;
  if (!spike_shape(n, kl, ku, 0, &m, &P)) return 0;
  const size_t q = (size_t)(kl + ku), qq = q > 0 ? q : 1;
  return round256(sizeof(double) * (size_t)n * qq) +             // spike columns
         2 * round256(sizeof(double) * (size_t)P * qq * qq) +     // boundary systems, A and A^T
         2 * round256(sizeof(int) * (size_t)P * qq) +             // their pivots
         round256(sizeof(double) * (size_t)n) +                   // G
         round256(sizeof(double) * (size_t)P * qq) +              // Y
         round256(sizeof(double) * (size_t)n) +                   // reciprocals of U's diagonal
         256;                                                     // far tips, flags
}

struct SpikePlan {
  spk::Ctx c;
  double* scr;
  double* M[2];
  int* piv[2];
  double* G;
  double* Y;
  double* rd;               // 1 / U_ii (the window solves)
  unsigned long long* far;  // [2]
  int* flags;               // [0] rows, [1] columns dominant, [2] failure
};

SpikePlan spike_layout(double* F, int64_t ldf, int64_t n, int kl, int ku, int level, char* q) {
  SpikePlan pl{};
  int64_t m = 0, P = 0;
  spike_shape(n, kl, ku, level, &m, &P);
  pl.c = spk::Ctx{F, ldf, n, kl, ku, m, P};
  const size_t qn = (size_t)(kl + ku), qq = qn > 0 ? qn : 1;
  pl.scr = reinterpret_cast<double*>(q);
  q += round256(sizeof(double) * (size_t)n * qq);
  for (int k = 0; k < 2; ++k) {
    pl.M[k] = reinterpret_cast<double*>(q);
    q += round256(sizeof(double) * (size_t)P * qq * qq);
  }
  for (int k = 0; k < 2; ++k) {
    pl.piv[k] = reinterpret_cast<int*>(q);
    q += round256(sizeof(int) * (size_t)P * qq);
  }
  pl.G = reinterpret_cast<double*>(q);
  q += round256(sizeof(double) * (size_t)n);
  pl.Y = reinterpret_cast<double*>(q);
  q += round256(sizeof(double) * (size_t)P * qq);
  pl.rd = reinterpret_cast<double*>(q);
  q += round256(sizeof(double) * (size_t)n);
  pl.far = reinterpret_cast<unsigned long long*>(q);
  pl.flags = reinterpret_cast<int*>(q + 64);
  return pl;
}

unsigned spk_grid(int64_t count) { return (unsigned)((count + kSpkThreads - 1) / kSpkThreads); }

__global__ void k_spk_dominance(spk::Ctx c, int* flags) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c.n; i += (int64_t)gridDim.x * blockDim.x) {
    int r, cc;
    spk::dominance(c, i, &r, &cc);
    if (!r) flags[0] = 0;
    if (!cc) flags[1] = 0;
  }
}

__global__ void k_spk_factor(spk::Ctx c, int* flags) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b < c.P && spk::factor_block(c, b)) atomicExch(&flags[2], 1);
}

__global__ void k_spk_spikes(spk::Ctx c, bool tr, double* scr, double* M, unsigned long long* far) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < c.P * spk::q_of(c)) spk::spike_column(c, tr, t, scr, M, far);
}

__global__ void k_spk_boundary(spk::Ctx c, double* M, int* piv, int* flags) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b + 1 < c.P && spk::factor_boundary(c, b, M, piv)) atomicExch(&flags[2], 1);
}

__global__ void k_spk_step1(spk::Ctx c, bool tr, const double* x, double* G) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b < c.P) spk::solve_step1(c, tr, b, x, G);
}

__global__ void k_spk_step2(spk::Ctx c, bool tr, const double* G, const double* M, const int* piv, double* Y) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b + 1 < c.P) spk::solve_step2(c, tr, b, G, M, piv, Y);
}

__global__ void k_spk_step3(spk::Ctx c, bool tr, const double* Y, double* x) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b < c.P) spk::solve_step3(c, tr, b, Y, x);
}

// Wide bands (kl + ku >= kSpkWarpQ): one warp per block for the block
// factorisation and the block solves, lanes over the rows of each step.
constexpr int64_t kSpkWarpQ = 16;
bool spk_warp(const spk::Ctx& c) { return spk::q_of(c) >= kSpkWarpQ; }

__global__ void __launch_bounds__(kSpkThreads) k_spk_factor_w(spk::Ctx c, int* flags) {
  const int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (b >= c.P) return;  // the whole warp
  auto run = [&](auto&& f) {
    f(lane);
    __syncwarp();
  };
  if (spk::wfactor_block(c, b, run) && lane == 0) atomicExch(&flags[2], 1);
}

__global__ void __launch_bounds__(kSpkThreads) k_spk_step1_w(spk::Ctx c, bool tr, const double* x, double* G) {
  __shared__ double red[kSpkThreads];
  const int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (b >= c.P) return;
  auto run = [&](auto&& f) {
    f(lane);
    __syncwarp();
  };
  spk::wsolve_step1(c, tr, b, x, G, red + (threadIdx.x & ~31u), run);
}

__global__ void __launch_bounds__(kSpkThreads) k_spk_step3_w(spk::Ctx c, bool tr, const double* Y, double* x) {
  __shared__ double red[kSpkThreads];
  const int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (b >= c.P) return;
  auto run = [&](auto&& f) {
    f(lane);
    __syncwarp();
  };
  spk::wsolve_step3(c, tr, b, Y, x, red + (threadIdx.x & ~31u), run);
}

// ------------------------------------------------ bands up to 32 wide
// For kl, ku <= 32 the spike columns run by sliding windows
// (spike_column_win, one thread each, coalesced).  From kl + ku >= 16 on
// (spk_warp) the other steps take forms whose chains do not wait on global
// memory: the block factorisation one phase per column (wlu_step), the
// boundary systems and their solves one warp each, and the block solves
// below.  Narrower bands keep the per-thread steps, which use every lane.
bool spk_win(const spk::Ctx& c) { return c.kl <= spk::kWinMaxBand && c.ku <= spk::kWinMaxBand; }
bool spk_wide_win(const spk::Ctx& c) { return spk_win(c) && spk::q_of(c) >= kSpkWarpQ; }

__global__ void __launch_bounds__(kSpkThreads) k_spk_factor_s(spk::Ctx c, int* flags, double* rd) {
  const int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (b >= c.P) return;  // the whole warp
  auto run = [&](auto&& f) {
    f(lane);
    __syncwarp();
  };
  if (spk::wfactor_block_step(c, b, rd, run) && lane == 0) atomicExch(&flags[2], 1);
}

// rd[i] = 1 / U_ii after the per-thread or phase factorisations.
__global__ void k_spk_rdiag(spk::Ctx c, double* rd) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c.n; i += (int64_t)gridDim.x * blockDim.x)
    rd[i] = 1.0 / spk::fa(c, i, i);
}

__global__ void __launch_bounds__(kSpkThreads) k_spk_spikes_win(spk::Ctx c, bool tr, double* scr, double* M,
                                                                 unsigned long long* far, const double* rd) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < c.P * spk::q_of(c)) spk::spike_column_win(c, tr, t, scr, M, far, rd);
}

__global__ void __launch_bounds__(kSpkThreads) k_spk_boundary_w(spk::Ctx c, double* M, int* piv, int* flags) {
  __shared__ double rv[kSpkThreads / 32][33];
  __shared__ int ri[kSpkThreads / 32][33];
  const int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (b + 1 >= c.P) return;  // the whole warp
  auto run = [&](auto&& f) {
    f(lane);
    __syncwarp();
  };
  if (spk::wfactor_boundary(c, b, M, piv, rv[w], ri[w], run) && lane == 0) atomicExch(&flags[2], 1);
}

__global__ void __launch_bounds__(kSpkThreads) k_spk_step2_w(spk::Ctx c, bool tr, const double* G, const double* M,
                                                              const int* piv, double* Y) {
  const int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (b + 1 >= c.P) return;
  auto run = [&](auto&& f) {
    f(lane);
    __syncwarp();
  };
  spk::wsolve_step2(c, tr, b, G, M, piv, Y, run);
}

// out[s..e) := A_bb^-1 in[s..e) (tr: A_bb^-T) by one warp, kl, ku <= 32.
// The lanes hold a window of 32 partial sums in registers, lane l the row
// l + 1 ahead of the current one (behind it, going backwards); each step
// finishes the current row in lane 0, broadcasts it, updates the rows
// within the bandwidth (one coalesced column of the factor for A, a gather
// of one factor row for A^T), shifts the window by a shuffle and takes the
// row 32 ahead into lane 31.  Row i receives its terms in the same order as
// solve_block; the diagonal enters as the reciprocal rd (one multiply in
// place of a division per row).  The loads of kGroup steps are issued
// together ahead of their chain.  in and out may alias.  (A variant with
// rotating row ownership, one shuffle fewer per step, measured slower.)
constexpr int kGroup = 8;

__device__ __forceinline__ void wsolve_win(const spk::Ctx& c, int64_t b, bool tr, const double* in, double* out,
                                           const double* __restrict__ rd, int lane) {
  const int64_t s = spk::blk_s(c, b), e = spk::blk_e(c, b);
  const int bl = spk::sys_kl(c, tr), bu = spk::sys_ku(c, tr);
  constexpr unsigned kAll = 0xffffffffu;
  // forward: the lower factor (A: unit L; A^T: U^T, diagonal U_jj)
  double acc = s + lane < e ? in[s + lane] : 0.0;
  for (int64_t j0 = s; j0 < e; j0 += kGroup) {
    double f[kGroup], nx[kGroup], rj[kGroup];
#pragma unroll
    for (int u = 0; u < kGroup; ++u) {
      const int64_t j = j0 + u, i = j + 1 + lane;
      f[u] = (j < e && lane < bl && i < e) ? spk::blkf(c, tr, i, j) : 0.0;
      nx[u] = (lane == 31 && j + 32 < e) ? in[j + 32] : 0.0;
      rj[u] = (tr && j < e) ? rd[j] : 1.0;
    }
#pragma unroll
    for (int u = 0; u < kGroup; ++u) {
      const int64_t j = j0 + u;
      if (j >= e) break;
      const double yj = __shfl_sync(kAll, (tr && lane == 0) ? acc * rj[u] : acc, 0);
      if (lane == 0) out[j] = yj;
      acc = __shfl_down_sync(kAll, acc, 1);
      if (lane == 31) acc = nx[u];
      if (lane < bl && j + 1 + lane < e) acc -= f[u] * yj;
    }
  }
  __syncwarp();
  // backward: the upper factor (A: U, diagonal U_jj; A^T: unit L^T)
  acc = e - 1 - lane >= s ? out[e - 1 - lane] : 0.0;
  for (int64_t j0 = e - 1; j0 >= s; j0 -= kGroup) {
    double f[kGroup], nx[kGroup], rj[kGroup];
#pragma unroll
    for (int u = 0; u < kGroup; ++u) {
      const int64_t j = j0 - u, i = j - 1 - lane;
      f[u] = (j >= s && lane < bu && i >= s) ? spk::blkf(c, tr, i, j) : 0.0;
      nx[u] = (lane == 31 && j - 32 >= s) ? out[j - 32] : 0.0;
      rj[u] = (!tr && j >= s) ? rd[j] : 1.0;
    }
#pragma unroll
    for (int u = 0; u < kGroup; ++u) {
      const int64_t j = j0 - u;
      if (j < s) break;
      const double xj = __shfl_sync(kAll, (!tr && lane == 0) ? acc * rj[u] : acc, 0);
      if (lane == 0) out[j] = xj;
      acc = __shfl_down_sync(kAll, acc, 1);
      if (lane == 31) acc = nx[u];
      if (lane < bu && j - 1 - lane >= s) acc -= f[u] * xj;
    }
  }
  __syncwarp();
}

__global__ void __launch_bounds__(kSpkThreads) k_spk_step1_r(spk::Ctx c, bool tr, const double* x, double* G,
                                                              const double* rd) {
  const int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (b >= c.P) return;
  wsolve_win(c, b, tr, x, G, rd, lane);
}

__global__ void __launch_bounds__(kSpkThreads) k_spk_step3_r(spk::Ctx c, bool tr, const double* Y, double* x,
                                                              const double* rd) {
  const int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (b >= c.P) return;
  spk::step3_couplings(c, tr, b, Y, x, lane);
  __syncwarp();
  wsolve_win(c, b, tr, x, x, rd, lane);
}

// x := A^-1 x (tr: A^-T x) in place with the partitioned factors.
int spike_apply(const SpikePlan& pl, double* x, bool tr, cudaStream_t st) {
  const spk::Ctx& c = pl.c;
  const int k = tr ? 1 : 0;
  if (spk_wide_win(c)) {
    k_spk_step1_r<<<spk_grid(32 * c.P), kSpkThreads, 0, st>>>(c, tr, x, pl.G, pl.rd);
    BCK(cudaGetLastError());
    if (spk::q_of(c) > 0) {
      k_spk_step2_w<<<spk_grid(32 * c.P), kSpkThreads, 0, st>>>(c, tr, pl.G, pl.M[k], pl.piv[k], pl.Y);
      BCK(cudaGetLastError());
    }
    k_spk_step3_r<<<spk_grid(32 * c.P), kSpkThreads, 0, st>>>(c, tr, pl.Y, x, pl.rd);
    BCK(cudaGetLastError());
    return ASOLVE_OK;
  }
  const bool w = spk_warp(c);
  if (w) k_spk_step1_w<<<spk_grid(32 * c.P), kSpkThreads, 0, st>>>(c, tr, x, pl.G);
  else k_spk_step1<<<spk_grid(c.P), kSpkThreads, 0, st>>>(c, tr, x, pl.G);
  BCK(cudaGetLastError());
  if (spk::q_of(c) > 0) {
    k_spk_step2<<<spk_grid(c.P), kSpkThreads, 0, st>>>(c, tr, pl.G, pl.M[k], pl.piv[k], pl.Y);
    BCK(cudaGetLastError());
  }
  if (w) k_spk_step3_w<<<spk_grid(32 * c.P), kSpkThreads, 0, st>>>(c, tr, pl.Y, x);
  else k_spk_step3<<<spk_grid(c.P), kSpkThreads, 0, st>>>(c, tr, pl.Y, x);
  BCK(cudaGetLastError());
  return ASOLVE_OK;
}

// FP64 normwise backward error of X, the maximum over the right-hand sides
// (||b - Ax||inf / (||A||inf ||x||inf + ||b||inf)), into *out.
int band_berr(const BandArgs& a, int kl, int ku, double norminf, unsigned long long* colmax, double* out,
              cudaStream_t st) {
  const int64_t n = a.n, nrhs = a.nrhs;
  BCK(cudaMemsetAsync(colmax, 0, sizeof(unsigned long long) * 3 * nrhs, st));
  dim3 g((unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), (unsigned)nrhs);
  k_band_berr<<<g, 256, 0, st>>>(a.AB, a.ldab, (int)a.kud, a.A, n, kl, ku, a.B, a.X, (int)nrhs, colmax);
  BCK(cudaGetLastError());
  unsigned long long hm[3 * 256];
  BCK(cudaMemcpyAsync(hm, colmax, sizeof(unsigned long long) * 3 * nrhs, cudaMemcpyDeviceToHost, st));
  BCK(cudaStreamSynchronize(st));
  double be = 0.0;
  for (int64_t c = 0; c < nrhs; ++c) {
    double rm, xm, bm;
    memcpy(&rm, &hm[c], 8);
    memcpy(&xm, &hm[nrhs + c], 8);
    memcpy(&bm, &hm[2 * nrhs + c], 8);
    const double den = norminf * xm + bm;
    const double b1 = den > 0.0 ? rm / den : (rm > 0.0 ? INFINITY : 0.0);
    if (!(b1 <= be)) be = b1;
  }
  *out = be;
  return ASOLVE_OK;
}

// The partitioned route's answer is kept only with a backward error this
// far below the 1e-13 bar (2^-46); otherwise the GBTRF-order path solves.
constexpr double kSpkBerrMax = 1.4210854715202004e-14;

// Outcome of one attempt of the partitioned route.
enum SpikeOutcome { SPK_OK = 0, SPK_NOT_DOMINANT, SPK_NUMERIC, SPK_FAR_TIPS };

// Dominance test, block factors, spikes and boundary systems (both systems
// unless no_rcond).  *out: SPK_OK (dominant, no zero pivot, no singular
// boundary system, far tips below kSpkFarTol) or why not; *touched: F was
// modified (re-packed before another attempt or the GBTRF-order path).
int spike_prepare(const SpikePlan& pl, bool no_rcond, int* out, bool* touched, cudaStream_t st) {
  const spk::Ctx& c = pl.c;
  *out = SPK_NOT_DOMINANT;
  *touched = false;
  BCK(cudaMemsetAsync(pl.flags, 0x01, 2 * sizeof(int), st));  // non-zero: dominant until a row says no
  BCK(cudaMemsetAsync(pl.flags + 2, 0, sizeof(int), st));
  BCK(cudaMemsetAsync(pl.far, 0, 2 * sizeof(unsigned long long), st));
  k_spk_dominance<<<4 * 152, 256, 0, st>>>(c, pl.flags);
  BCK(cudaGetLastError());
  int h[3];
  BCK(cudaMemcpyAsync(h, pl.flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  BCK(cudaStreamSynchronize(st));
  if (!h[0] && !h[1]) return ASOLVE_OK;
  *touched = true;
  *out = SPK_NUMERIC;
  const bool win = spk_wide_win(c);
  if (win) k_spk_factor_s<<<spk_grid(32 * c.P), kSpkThreads, 0, st>>>(c, pl.flags, pl.rd);
  else if (spk_warp(c)) k_spk_factor_w<<<spk_grid(32 * c.P), kSpkThreads, 0, st>>>(c, pl.flags);
  else k_spk_factor<<<spk_grid(c.P), kSpkThreads, 0, st>>>(c, pl.flags);
  BCK(cudaGetLastError());
  if (!win && spk_win(c)) {  // the window spikes take the diagonal's reciprocals
    k_spk_rdiag<<<4 * 152, 256, 0, st>>>(c, pl.rd);
    BCK(cudaGetLastError());
  }
  const int64_t q = spk::q_of(c);
  for (int k = 0; k < (no_rcond ? 1 : 2) && q > 0; ++k) {
    BCK(cudaMemsetAsync(pl.M[k], 0, sizeof(double) * (size_t)(c.P * q * q), st));
    if (spk_win(c))
      k_spk_spikes_win<<<spk_grid(c.P * q), kSpkThreads, 0, st>>>(c, k == 1, pl.scr, pl.M[k], pl.far + k, pl.rd);
    else
      k_spk_spikes<<<spk_grid(c.P * q), kSpkThreads, 0, st>>>(c, k == 1, pl.scr, pl.M[k], pl.far + k);
    BCK(cudaGetLastError());
    if (win) k_spk_boundary_w<<<spk_grid(32 * c.P), kSpkThreads, 0, st>>>(c, pl.M[k], pl.piv[k], pl.flags);
    else k_spk_boundary<<<spk_grid(c.P), kSpkThreads, 0, st>>>(c, pl.M[k], pl.piv[k], pl.flags);
    BCK(cudaGetLastError());
  }
  unsigned long long fb[2];
  BCK(cudaMemcpyAsync(&h[2], pl.flags + 2, sizeof(int), cudaMemcpyDeviceToHost, st));
  BCK(cudaMemcpyAsync(fb, pl.far, sizeof(fb), cudaMemcpyDeviceToHost, st));
  BCK(cudaStreamSynchronize(st));
  double far0, far1;
  memcpy(&far0, &fb[0], 8);
  memcpy(&far1, &fb[1], 8);
  if (h[2] == 0) *out = (far0 <= kSpkFarTol && far1 <= kSpkFarTol) ? SPK_OK : SPK_FAR_TIPS;
  return ASOLVE_OK;
}

}  // namespace

// Whether the fast kernels (shared-memory window, register window) cover
// these bandwidths.
bool band_window_fits(int64_t kl, int64_t ku) {
  const int64_t kv = kl + ku, ldf = 2 * kl + ku + 1;
  return kv + 1 <= 32 * kMaxR && (size_t)(kv + 1 + kD) * (size_t)ldf * sizeof(double) <= kWinSmemMax;
}

size_t band_ws_bytes(int64_t n, int64_t kl, int64_t ku, int64_t nrhs) {
  (void)nrhs;
  const size_t ldf = (size_t)(2 * kl + ku + 1);
  size_t sw = 0;  // partitioned sweeps: sized for the widest window they take
  if (n >= kSwMinN) sw = (kl + ku + 1 <= kSwMaxWs) ? sw_bytes(n, (int)kl, (int)ku) : sw_bytes(n, kSwMaxWs - 1, 0);
  if (spike_enabled() && n >= kSpkMinN) {  // the partitioned route uses the same area
    const size_t sp = spike_bytes(n, (int)kl, (int)ku);
    if (sp > sw) sw = sp;
  }
  return round256(sizeof(double) * ldf * (size_t)n) + round256(sizeof(int) * (size_t)n) +
         2 * round256(sizeof(double) * (size_t)n) + sw + kTailBytes;
}

// Device memory needed before the true bandwidths are known (declared band).
size_t band_ws_bytes_declared(int64_t n, int64_t kld, int64_t kud, int64_t nrhs) {
  return band_ws_bytes(n, kld, kud, nrhs);
}

// The banded route for one system.  Returns the status (also in info).
// status ASOLVE_PENDING means: the factor failed or rcond is below the
// threshold, the SVD fallback is allowed and n <= kSvdLargeMax -- the
// caller runs it on a dense copy.
int band_solve(const BandArgs& a, void* ws, size_t ws_bytes, asolve_info* info) {
  cudaStream_t st = a.st;
  const int64_t n = a.n, nrhs = a.nrhs;
  memset(info, 0, sizeof(*info));
  info->rcond = NAN;
  info->berr = NAN;
  info->svd_rank = -1;
  info->cls = ASOLVE_CLS_BANDED;
  info->route = ASOLVE_ROUTE_BAND_LU;
  info->precision = ASOLVE_PREC_FP64;
  if (n > INT32_MAX / 2) return info->status = ASOLVE_E_UNSUPPORTED;
  if (nrhs > 256) return info->status = ASOLVE_E_UNSUPPORTED;
  if (ws_bytes < kTailBytes) return info->status = ASOLVE_E_NOMEM;
  char* base = static_cast<char*>(ws);
  char* tail = base + ((ws_bytes - kTailBytes) & ~(size_t)255);
  BandScan* dscan = reinterpret_cast<BandScan*>(tail);
  double* dscal = reinterpret_cast<double*>(tail + 256);  // 32 doubles: estimator scalars and partials
  int* dint = reinterpret_cast<int*>(tail + 512);
  unsigned long long* colmax = reinterpret_cast<unsigned long long*>(tail + 1024);
  int kl, ku;
  double norm1, norminf;
  if (a.AB) {
    BCK(cudaMemsetAsync(dscan, 0, sizeof(BandScan), st));
    k_bscan<<<1024, 256, 0, st>>>(a.AB, a.ldab, (int)a.kld, (int)a.kud, n, a.B, n * nrhs, dscan);
    BCK(cudaGetLastError());
    BandScan h;
    BCK(cudaMemcpyAsync(&h, dscan, sizeof(h), cudaMemcpyDeviceToHost, st));
    BCK(cudaStreamSynchronize(st));
    kl = h.kl;
    ku = h.ku;
    memcpy(&norm1, &h.norm1, 8);
    memcpy(&norminf, &h.norminf, 8);
    info->kl = kl;
    info->ku = ku;
    if (h.nonfinite || h.b_nonfinite) return info->status = ASOLVE_E_NONFINITE;
  } else {
    kl = (int)a.kl;
    ku = (int)a.ku;
    norm1 = a.norm1;
    norminf = a.norminf;
    info->kl = kl;
    info->ku = ku;
  }
  const int kv = kl + ku, ldf = 2 * kl + ku + 1;
  if (band_ws_bytes(n, kl, ku, nrhs) > ws_bytes) return info->status = ASOLVE_E_NOMEM;
  double* F = reinterpret_cast<double*>(base);
  int* piv = reinterpret_cast<int*>(base + round256(sizeof(double) * (size_t)ldf * n));
  double* ev = reinterpret_cast<double*>(reinterpret_cast<char*>(piv) + round256(sizeof(int) * (size_t)n));
  double* exi = ev + ((n + 31) & ~(int64_t)31);
  k_bpack<<<4 * 152, 256, 0, st>>>(a.AB, a.ldab, (int)a.kud, a.A, n, kl, ku, F);
  BCK(cudaGetLastError());
  const bool no_rcond = (a.flags & ASOLVE_NO_RCOND) != 0;
  const bool svd_ok = !(a.flags & ASOLVE_NO_APPROX) && n <= kSvdLargeMax;
  char* region = reinterpret_cast<char*>(exi + ((n + 31) & ~(int64_t)31));
  region = reinterpret_cast<char*>(((uintptr_t)region + 255) & ~(uintptr_t)255);
  double rc = NAN;
  bool spiked = false;
  double spike_be = NAN;
  int64_t spk_m = 0, spk_P = 0;
  // the tridiagonal specialisation (ASOLVE_TRIDIAG, kl = ku = 1): the
  // partitioned route below when it applies, else the elimination, whose
  // pivots and operations for kl = ku = 1 are xGTTRF's.  (Parallel cyclic
  // reduction was measured and left out: its O(n log n) FP64 divisions made
  // it 4x slower than the partitioned route at n = 10^6, and on weakly
  // dominant, ill-conditioned systems its backward error reached 4e-10.)
  const bool tridiag = (a.flags & ASOLVE_TRIDIAG) && kl == 1 && ku == 1;
  if (tridiag) info->route = ASOLVE_ROUTE_TRIDIAG;
  // dominant bands: the partitioned route (band_spike.cuh); blocks twice as
  // long on another attempt when the spikes have not decayed across them
  for (int level = 0; level < 3 && spike_enabled() && n >= kSpkMinN &&
                      spike_shape(n, kl, ku, level, &spk_m, &spk_P); ++level) {
    const SpikePlan sp = spike_layout(F, ldf, n, kl, ku, level, region);
    int outcome = SPK_NOT_DOMINANT;
    bool touched = false;
    int r = spike_prepare(sp, no_rcond, &outcome, &touched, st);
    if (r) return info->status = r;
    if (outcome == SPK_OK) {
      BCK(cudaMemcpyAsync(a.X, a.B, sizeof(double) * (size_t)(n * nrhs), cudaMemcpyDeviceToDevice, st));
      for (int64_t c = 0; c < nrhs; ++c)
        if ((r = spike_apply(sp, a.X + (size_t)c * n, false, st))) return info->status = r;
      // a posteriori check, whatever the scaling of A: the backward error
      if ((r = band_berr(a, kl, ku, norminf, colmax, &spike_be, st))) return info->status = r;
      if (!(spike_be <= kSpkBerrMax)) outcome = SPK_NUMERIC;
    }
    if (outcome == SPK_OK) {
      if (!no_rcond) {
        double est = NAN;
        auto apply = [&](double* v, bool tr) { return spike_apply(sp, v, tr, st); };
        const int erc = est_host<double>((int)n, ev, exi, dscal, dint, apply, st, &est);
        if (erc) return info->status = erc;
        rc = rcond_from_est(norm1, est);
      }
      spiked = true;
      info->detail |= 16;  // solved by the partitioned route
      break;
    }
    if (touched) {  // back to the original band for another attempt or the GBTRF-order path
      k_bpack<<<4 * 152, 256, 0, st>>>(a.AB, a.ldab, (int)a.kud, a.A, n, kl, ku, F);
      BCK(cudaGetLastError());
    }
    if (outcome != SPK_FAR_TIPS) break;
  }
  if (!spiked) {
    BCK(cudaMemsetAsync(dint, 0, sizeof(int) * 4, st));
    const size_t wsm = sizeof(double) * (size_t)(kv + 1 + kD) * ldf;
    const int R = window_r(kv);
    if (wsm <= kWinSmemMax) {
      BCK(ASV_SMEM_LIMIT_ONCE(k_band_lu_win, kWinSmemMax));
      k_band_lu_win<<<1, 32, wsm, st>>>(F, ldf, (int)n, kl, ku, piv, dint);
    } else {
      k_band_lu_glob<<<1, 32, 0, st>>>(F, ldf, (int)n, kl, ku, piv, dint);
    }
    BCK(cudaGetLastError());
    int fail = 0;
    BCK(cudaMemcpyAsync(&fail, dint, sizeof(int), cudaMemcpyDeviceToHost, st));
    BCK(cudaStreamSynchronize(st));
    if (fail) {
      BCK(cudaMemsetAsync(a.X, 0, sizeof(double) * (size_t)(n * nrhs), st));
      BCK(cudaStreamSynchronize(st));
      return info->status = svd_ok ? ASOLVE_PENDING : ASOLVE_E_SINGULAR;
    }
    BCK(cudaMemcpyAsync(a.X, a.B, sizeof(double) * (size_t)(n * nrhs), cudaMemcpyDeviceToDevice, st));
    // long systems with windows of up to kSwMaxWs: partitioned sweeps
    bool par = n >= kSwMinN && kv + 1 <= kSwMaxWs;
    SweepPlan pl{};
    if (par) {
      char* q = region;
      const int P0 = sw_blocks(n);
      pl.c = SweepCtx{F, ldf, (int)n, kl, ku, piv, 0, 0};
      pl.c.L = (int)((n + P0 - 1) / P0);
      pl.c.P = (int)((n + pl.c.L - 1) / pl.c.L);
      for (int k = 0; k < 4; ++k) {
        pl.T[k] = reinterpret_cast<double*>(q);
        const size_t ws = (size_t)sw_ws(k, kl, ku);
        q += round256(sizeof(double) * (size_t)pl.c.P * ws * ws);
      }
      pl.tv = reinterpret_cast<double*>(q);
      q += round256(sizeof(double) * (size_t)pl.c.P * (kv + 1));
      pl.Ws = reinterpret_cast<double*>(q);
      q += round256(sizeof(double) * (size_t)pl.c.P * (kv + 1));
      pl.tmp = reinterpret_cast<double*>(q);
      int src;
      if ((src = sw_run<SW_L>(pl, nullptr, nullptr, true, st)) || (src = sw_run<SW_U>(pl, nullptr, nullptr, true, st)))
        return info->status = src;
      if (!no_rcond &&
          ((src = sw_run<SW_UT>(pl, nullptr, nullptr, true, st)) || (src = sw_run<SW_LT>(pl, nullptr, nullptr, true, st))))
        return info->status = src;
      for (int64_t c = 0; c < nrhs; ++c)
        if ((src = sw_apply(pl, a.X + (size_t)c * n, false, st))) return info->status = src;
      // the sweeps chain transfer matrices, which can amplify rounding on a
      // band that is not dominant: their answer stands only with a backward
      // error below 2^-46.  Short of it, FP64 refinement with the same
      // sweeps (r = b - A x, x += A^-1 r; a few steps at O(n (kl + ku))
      // each), and if that does not get there either the sequential kernels
      // solve again (and estimate).
      double pbe = 0.0;
      if ((src = band_berr(a, kl, ku, norminf, colmax, &pbe, st))) return info->status = src;
      for (int it = 0; it < kSwRefineSteps && !(pbe <= kSpkBerrMax); ++it) {
        info->detail |= 128;
        const unsigned g = (unsigned)((n + 255) / 256 < 4 * 152 ? (n + 255) / 256 : 4 * 152);
        for (int64_t c = 0; c < nrhs; ++c) {
          k_band_resid<<<g, 256, 0, st>>>(a.AB, a.ldab, (int)a.kud, a.A, n, kl, ku, a.B + (size_t)c * n,
                                           a.X + (size_t)c * n, ev);
          BCK(cudaGetLastError());
          if ((src = sw_apply(pl, ev, false, st))) return info->status = src;
          k_band_xadd<<<g, 256, 0, st>>>(a.X + (size_t)c * n, ev, n);
          BCK(cudaGetLastError());
        }
        if ((src = band_berr(a, kl, ku, norminf, colmax, &pbe, st))) return info->status = src;
      }
      if (!(pbe <= kSpkBerrMax)) {
        BCK(cudaMemcpyAsync(a.X, a.B, sizeof(double) * (size_t)(n * nrhs), cudaMemcpyDeviceToDevice, st));
        par = false;
        info->detail |= 256;  // re-solved sequentially
      }
    }
    if (!par) switch (R) {
      case 1: k_band_solve<1><<<(unsigned)nrhs, 32, 0, st>>>(F, ldf, (int)n, kl, ku, piv, a.X); break;
      case 2: k_band_solve<2><<<(unsigned)nrhs, 32, 0, st>>>(F, ldf, (int)n, kl, ku, piv, a.X); break;
      case 4: k_band_solve<4><<<(unsigned)nrhs, 32, 0, st>>>(F, ldf, (int)n, kl, ku, piv, a.X); break;
      case 8: k_band_solve<8><<<(unsigned)nrhs, 32, 0, st>>>(F, ldf, (int)n, kl, ku, piv, a.X); break;
      default: k_band_solve_glob<<<(unsigned)nrhs, 32, 0, st>>>(F, ldf, (int)n, kl, ku, piv, a.X); break;
    }
    BCK(cudaGetLastError());
    if (!no_rcond && par) {
      double est = NAN;
      auto apply = [&](double* v, bool tr) { return sw_apply(pl, v, tr, st); };
      const int erc = est_host<double>((int)n, ev, exi, dscal, dint, apply, st, &est);
      if (erc) return info->status = erc;
      rc = rcond_from_est(norm1, est);
    } else if (!no_rcond) {
      switch (R) {
        case 1: k_band_est<1, false><<<1, 32, 0, st>>>(F, ldf, (int)n, kl, ku, piv, ev, exi, dscal); break;
        case 2: k_band_est<2, false><<<1, 32, 0, st>>>(F, ldf, (int)n, kl, ku, piv, ev, exi, dscal); break;
        case 4: k_band_est<4, false><<<1, 32, 0, st>>>(F, ldf, (int)n, kl, ku, piv, ev, exi, dscal); break;
        case 8: k_band_est<8, false><<<1, 32, 0, st>>>(F, ldf, (int)n, kl, ku, piv, ev, exi, dscal); break;
        default: k_band_est<1, true><<<1, 32, 0, st>>>(F, ldf, (int)n, kl, ku, piv, ev, exi, dscal); break;
      }
      BCK(cudaGetLastError());
      double est = NAN;
      BCK(cudaMemcpyAsync(&est, dscal, sizeof(double), cudaMemcpyDeviceToHost, st));
      BCK(cudaStreamSynchronize(st));
      rc = rcond_from_est(norm1, est);
    }
  }
  info->rcond = no_rcond ? NAN : rc;
  if (a.flags & ASOLVE_BERR) {
    double be = spike_be;
    if (!spiked) {
      const int r = band_berr(a, kl, ku, norminf, colmax, &be, st);
      if (r) return info->status = r;
    }
    info->berr = be;
  } else {
    BCK(cudaStreamSynchronize(st));
  }
  const bool poor = !no_rcond && !(rc >= a.rcond_threshold);
  if (!poor) return info->status = ASOLVE_OK;
  if (a.flags & ASOLVE_NO_APPROX) return info->status = ASOLVE_W_ILLCOND;
  return info->status = svd_ok ? ASOLVE_PENDING : ASOLVE_W_ILLCOND;
}

// Dense copy of a band-stored matrix (for the SVD fallback of small n).
int band_to_dense(const double* AB, int64_t ldab, int64_t kld, int64_t kud, int64_t n, double* A, cudaStream_t st) {
  k_band_to_dense<<<4 * 152, 256, 0, st>>>(AB, ldab, (int)kld, (int)kud, n, A);
  BCK(cudaGetLastError());
  return ASOLVE_OK;
}

}  // namespace asv
