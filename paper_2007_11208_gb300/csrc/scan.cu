// scan.cu -- one-pass property scan of A (paper Sec. 2.1, Sec. 2.2, Fig. 4).
//
// For every system the scan finds, in a single read of A:
//   kl, ku      sub/super-diagonal counts: the largest |i - j| over non-zero
//               elements below/above the diagonal (Sec. 2.1; the column
//               traversal there visits the same elements);
//   lower/upper ku == 0 / kl == 0 (Sec. 2.2);
//   likely_sympd  the Fig. 4 predicates: positive diagonal, symmetry within
//               100 eps (absolute and relative), the lower element below the
//               largest diagonal entry, |A_ij| + |A_ji| < A_ii + A_jj;
//   non-finite  any Inf/NaN in A or B;
//   ||A||_1, ||A||_inf  (for the condition estimate and the backward error).
//
// GB300 design: FP64 arithmetic runs at 1/70 of the FP32 rate, so the scan
// does no per-element FP64 work.  Non-zero tests, bandwidths and the
// "largest modulus" compare work on the IEEE bit patterns (integer order of
// non-negative doubles equals their numeric order); the symmetry and
// dominance predicates fall back to FP64 only for pairs an integer test
// cannot decide (unequal bit patterns, or exponents too close); the norms
// are summed from bit-truncated FP32 magnitudes in 32-element partials
// (relative error below 2^-18), which are combined with a compensated FP32
// sum in a fixed order, so the result does not depend on scheduling.  A is read once, tile pair by
// tile pair: tile (P,Q) is staged through shared memory and its mirror
// (Q,P) is read row-wise straight from global memory, which puts every
// element next to its transpose partner.
#include "asolve_internal.cuh"

namespace asv {

constexpr int kScanThreads = 256;
constexpr int kScanWarps = kScanThreads / kWarp;
constexpr int kTileLd = 33;  // padded column stride of a staged 32x32 FP64 tile

// |x| truncated to FP32 from its bit pattern; flags magnitudes outside the
// FP32 normal range (the caller then sums in FP64 instead).
__device__ __forceinline__ float abs_f32_trunc(uint64_t b, bool& range_bad) {
  uint32_t hi = (uint32_t)(b >> 32) & 0x7fffffffu, lo = (uint32_t)b;
  int e = (int)(hi >> 20);
  if ((hi | lo) == 0) return 0.0f;
  int fe = e - 1023 + 127;
  if (fe <= 0 || fe >= 255) { range_bad = true; return 0.0f; }
  return __uint_as_float(((uint32_t)fe << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}

struct ScanShared {
  double tile[kScanWarps][32 * kTileLd];
  int kl, ku;
  int sym_ok;
  int nonfinite;
  int range_bad;
  int diag_pos;
  double max_diag;
  double red[kScanWarps];
};

// Fig. 4 predicates for the pair (a = A_ij below the diagonal, b = A_ji).
// Returns true when the pair violates one of them.
// e_min: a biased exponent at which the symmetry test is decided without
// FP64 arithmetic: when the exponents of a and b differ by 2 or more, the
// larger magnitude m has |a - b| > m/2 > tol m, and when m's exponent is at
// least e_min also m/2 > tol — the pair fails exactly when the FP64 test
// would say so.
__device__ __forceinline__ bool pair_fails(double a, double b, double di, double dj,
                                           uint64_t hmd, double tol, int e_min) {
  const uint64_t kAbs = 0x7fffffffffffffffull;
  uint64_t ab = dbits(a), bb = dbits(b);
  uint64_t ha = ab & kAbs, hb = bb & kAbs;
  if (ab != bb) {  // symmetry within tol, absolute and relative
    const int ea = (int)(ha >> 52), eb = (int)(hb >> 52);
    if (abs(ea - eb) >= 2 && max(ea, eb) >= e_min) return true;
    double delta = fabs(__dadd_rn(a, -b));
    double mx = fabs(a) > fabs(b) ? fabs(a) : fabs(b);
    if (delta > tol && delta > __dmul_rn(tol, mx)) return true;
  }
  if (ha >= hmd) return true;  // |A_ij| >= max_diag
  int m = (int)((ha > hb ? ha : hb) >> 52);
  uint64_t hi_d = dbits(di) > dbits(dj) ? dbits(di) : dbits(dj);
  int ed = (int)(hi_d >> 52);
  if (m + 3 <= ed) return false;  // |a|+|b| < 2^(m-1021) <= 2^(ed-1023) <= d_i+d_j
  return __dadd_rn(fabs(a), fabs(b)) >= __dadd_rn(di, dj);
}

// Process tile pairs (P, Q), P >= Q, with linear index p = P(P+1)/2 + Q,
// for p = first, first + step, ...  One warp handles one pair at a time.
// colpart[R * n + c] receives the FP32 sum of |A(i, c)| over the rows i of
// row block R; rowpart[R * n + r] the sum of |A(r, j)| over column block R.
__device__ void scan_pairs(const double* __restrict__ A, int n, const double* diag,
                           int64_t first, int64_t step, float* colpart, float* rowpart,
                           ScanShared& sh, double tol, uint64_t hmd, int& kl_l, int& ku_l,
                           bool& nonfinite_l, bool& range_bad_l, bool& symfail_l) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int T = (n + 31) / 32;
  const int64_t npairs = (int64_t)T * (T + 1) / 2;
  double* ts = sh.tile[warp];
  const int e_min = tol <= 0.0 ? 0 : (tol < 0.25 ? ilogb(tol) + 1025 : 0x7fffffff);
  for (int64_t p = first; p < npairs; p += step) {
    // invert p = P(P+1)/2 + Q
    int64_t P = (int64_t)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
    while (P * (P + 1) / 2 > p) --P;
    while ((P + 1) * (P + 2) / 2 <= p) ++P;
    const int64_t Q = p - P * (P + 1) / 2;
    const int i0 = (int)P * 32, j0 = (int)Q * 32;
    // stage tile (P,Q): column c of the tile is column j0+c, rows i0..i0+31
    {
      const int row = i0 + lane;
#pragma unroll 8
      for (int c = 0; c < 32; ++c) {
        const int col = j0 + c;
        double v = 0.0;
        if (row < n && col < n) v = __ldg(A + (size_t)col * n + row);
        ts[c * kTileLd + lane] = v;
      }
    }
    __syncwarp();
    const bool check_sym = (*(volatile int*)&sh.sym_ok) != 0;
    float cs1 = 0.f, rs1 = 0.f, rs2 = 0.f;
    float v2[32];
    if (P == Q) {
      const int jc = i0 + lane;  // this lane's column (and row) index
      bool chk = check_sym;
      for (int k = 0; k < 32; ++k) {
        // once a pair of this warp failed, the predicate is decided
        if ((k & 7) == 0) chk = chk && !__any_sync(0xffffffffu, symfail_l);
        const int ir = i0 + k;
        double a = ts[lane * kTileLd + k];  // A(ir, jc)
        uint64_t ab = dbits(a);
        if (ir < n && jc < n) {
          if (is_nonfinite_bits(ab)) nonfinite_l = true;
          if (is_nonzero_bits(ab)) {
            if (k > lane) kl_l = max(kl_l, k - lane);
            if (k < lane) ku_l = max(ku_l, lane - k);
          }
          cs1 += abs_f32_trunc(ab, range_bad_l);
          if (chk && k > lane) {
            double b = ts[k * kTileLd + lane];  // A(jc, ir)
            if (pair_fails(a, b, diag[ir], diag[jc], hmd, tol, e_min)) symfail_l = true;
          }
        }
        double at = ts[k * kTileLd + lane];  // A(i0+lane, i0+k): row sums
        if (i0 + lane < n && i0 + k < n) rs1 += abs_f32_trunc(dbits(at), range_bad_l);
      }
      if (jc < n) {
        colpart[(size_t)P * n + jc] = cs1;
        rowpart[(size_t)P * n + jc] = rs1;
      }
    } else {
      // mirror tile (Q,P) held row-wise: lane owns row j0+lane, element k is
      // column i0+k, i.e. the transpose partner of staged element (i0+k, j0+lane)
      const int jr = j0 + lane;
      double bv[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        const int ic = i0 + k;
        bv[k] = (jr < n && ic < n) ? __ldg(A + (size_t)ic * n + jr) : 0.0;
      }
      bool chk = check_sym;
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        if ((k & 7) == 0) chk = chk && !__any_sync(0xffffffffu, symfail_l);
        const int ir = i0 + k;
        const bool valid = (ir < n) && (jr < n);
        double a = ts[lane * kTileLd + k];  // A(ir, jr): below the diagonal
        double b = bv[k];                   // A(jr, ir): above the diagonal
        uint64_t ab = dbits(a), bb = dbits(b);
        float fa = 0.f, fb = 0.f;
        if (valid) {
          if (is_nonfinite_bits(ab) || is_nonfinite_bits(bb)) nonfinite_l = true;
          if (is_nonzero_bits(ab)) kl_l = max(kl_l, ir - jr);
          if (is_nonzero_bits(bb)) ku_l = max(ku_l, ir - jr);
          fa = abs_f32_trunc(ab, range_bad_l);
          fb = abs_f32_trunc(bb, range_bad_l);
          if (chk && pair_fails(a, b, diag[ir], diag[jr], hmd, tol, e_min)) symfail_l = true;
        }
        cs1 += fa;   // column jr of tile (P,Q)
        rs2 += fb;   // row jr of tile (Q,P)
        v2[k] = fb;  // column ir of tile (Q,P): summed across lanes below
        double at = ts[k * kTileLd + lane];  // A(i0+lane, j0+k): row sums of (P,Q)
        if (i0 + lane < n && j0 + k < n) rs1 += abs_f32_trunc(dbits(at), range_bad_l);
      }
      // reduce-scatter: afterwards v2[0] of lane l = sum over lanes of v2[l]
#pragma unroll
      for (int s = 16; s >= 1; s >>= 1) {
        const bool upper = (lane & s) != 0;
#pragma unroll
        for (int i = 0; i < s; ++i) {
          float send = upper ? v2[i] : v2[i + s];
          float keep = upper ? v2[i + s] : v2[i];
          v2[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
      }
      if (jr < n) {
        colpart[(size_t)P * n + jr] = cs1;
        rowpart[(size_t)P * n + jr] = rs2;
      }
      if (i0 + lane < n) {
        colpart[(size_t)Q * n + i0 + lane] = v2[0];
        rowpart[(size_t)Q * n + i0 + lane] = rs1;
      }
    }
    if (symfail_l) sh.sym_ok = 0;
    __syncwarp();
  }
}

// Diagonal pass (Fig. 4: every A_jj > 0, and the largest one).
__device__ void scan_diag(const double* __restrict__ A, int n, double* diag, ScanShared& sh) {
  bool pos = true;
  double md = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double d = __ldg(A + (size_t)i * n + i);
    diag[i] = d;
    if (d <= 0.0) pos = false;
    if (d > md) md = d;
  }
  md = warp_max(md);
  pos = __all_sync(0xffffffffu, pos);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    sh.red[warp] = md;
    if (!pos) atomicAnd(&sh.diag_pos, 0);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = sh.red[w] > m ? sh.red[w] : m;
    sh.max_diag = m;
  }
  __syncthreads();
}

// Compensated (Kahan) FP32 sum of the T partials of column/row j: the FP64
// pipe is far too slow on this part to spend one FP64 add per partial.
__device__ __forceinline__ float kahan_partials(const float* part, int n, int T, int j) {
  float s = 0.f, c = 0.f;
  for (int R = 0; R < T; ++R) {
    const float y = part[(size_t)R * n + j] - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  return s;
}

// ||A||_1 and ||A||_inf from the partials (fixed summation order).
__device__ void reduce_norms(const float* colpart, const float* rowpart, int n, int T,
                             double& norm1, double& norminf, ScanShared& sh) {
  float c1f = 0.f, cif = 0.f;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const float s = kahan_partials(colpart, n, T, j), r = kahan_partials(rowpart, n, T, j);
    c1f = s > c1f ? s : c1f;
    cif = r > cif ? r : cif;
  }
  double c1 = (double)c1f, ci = (double)cif;
  c1 = warp_max(c1);
  ci = warp_max(ci);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh.red[warp] = c1;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = sh.red[w] > m ? sh.red[w] : m;
    norm1 = m;
  }
  __syncthreads();
  if (lane == 0) sh.red[warp] = ci;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = sh.red[w] > m ? sh.red[w] : m;
    norminf = m;
  }
  __syncthreads();
}

// Exact FP64 norms, used only when some magnitude falls outside FP32 range.
__device__ void norms_fp64(const double* __restrict__ A, int n, double& norm1, double& norminf,
                           ScanShared& sh) {
  double c1 = 0.0, ci = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double s = 0.0, r = 0.0;
    for (int i = 0; i < n; ++i) {
      s += fabs(A[(size_t)j * n + i]);
      r += fabs(A[(size_t)i * n + j]);
    }
    c1 = s > c1 ? s : c1;
    ci = r > ci ? r : ci;
  }
  c1 = warp_max(c1);
  ci = warp_max(ci);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh.red[warp] = c1;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = sh.red[w] > m ? sh.red[w] : m;
    norm1 = m;
  }
  __syncthreads();
  if (lane == 0) sh.red[warp] = ci;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = sh.red[w] > m ? sh.red[w] : m;
    norminf = m;
  }
  __syncthreads();
}

__device__ bool any_nonfinite(const double* __restrict__ X, int64_t cnt) {
  bool bad = false;
  for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x)
    if (is_nonfinite_bits(dbits(__ldg(X + i)))) bad = true;
  return __syncthreads_or(bad) != 0;
}

// Class from the scan flags: banded, lower, upper, sympd, general (Sec. 2).
__device__ __host__ inline int classify(int n, int flags) {
  if (n == 0) return ASOLVE_CLS_NONE;
  if (flags & SF_BANDED) return ASOLVE_CLS_BANDED;
  if (flags & SF_LOWER) return ASOLVE_CLS_LOWER;
  if (flags & SF_UPPER) return ASOLVE_CLS_UPPER;
  if (flags & SF_SYMPD) return ASOLVE_CLS_SYMPD;
  return ASOLVE_CLS_GENERAL;
}

__device__ int band_flag(int64_t n, int64_t kl, int64_t ku, double band_frac) {
  int64_t cnt = n * (kl + ku + 1) - kl * (kl + 1) / 2 - ku * (ku + 1) / 2;
  return ((double)cnt <= band_frac * (double)n * (double)n) ? SF_BANDED : 0;
}

// One CTA scans one whole system.
__device__ void cta_scan_system(const double* __restrict__ A, int n, const double* __restrict__ B,
                                int64_t nb, float* scratch, double tol, double band_frac,
                                double* diag, ScanShared& sh, ScanRes* out) {
  if (threadIdx.x == 0) {
    sh.kl = 0; sh.ku = 0; sh.sym_ok = 1; sh.nonfinite = 0; sh.range_bad = 0; sh.diag_pos = 1;
  }
  __syncthreads();
  scan_diag(A, n, diag, sh);
  if (!sh.diag_pos && threadIdx.x == 0) sh.sym_ok = 0;
  __syncthreads();
  const int T = (n + 31) / 32;
  float* colpart = scratch;
  float* rowpart = scratch + (size_t)T * n;
  int kl_l = 0, ku_l = 0;
  bool nf = false, rb = false, sf = false;
  scan_pairs(A, n, diag, threadIdx.x >> 5, kScanWarps, colpart, rowpart, sh, tol,
             dbits(sh.max_diag), kl_l, ku_l, nf, rb, sf);
  kl_l = __reduce_max_sync(0xffffffffu, kl_l);
  ku_l = __reduce_max_sync(0xffffffffu, ku_l);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&sh.kl, kl_l);
    atomicMax(&sh.ku, ku_l);
  }
  if (nf) sh.nonfinite = 1;
  if (rb) sh.range_bad = 1;
  __syncthreads();
  bool bbad = any_nonfinite(B, nb);
  double norm1 = 0.0, norminf = 0.0;
  if (sh.range_bad) {
    norms_fp64(A, n, norm1, norminf, sh);
  } else {
    reduce_norms(colpart, rowpart, n, T, norm1, norminf, sh);
  }
  if (threadIdx.x == 0) {
    ScanRes r;
    r.kl = sh.kl;
    r.ku = sh.ku;
    int f = 0;
    if (sh.nonfinite) f |= SF_NONFINITE;
    if (bbad) f |= SF_B_NONFINITE;
    if (n > 0 && sh.diag_pos && sh.sym_ok) f |= SF_SYMPD;
    if (sh.ku == 0) f |= SF_LOWER;
    if (sh.kl == 0) f |= SF_UPPER;
    if (sh.range_bad) f |= SF_NORM_FP64;
    f |= band_flag(n, sh.kl, sh.ku, band_frac);
    r.flags = f;
    r.cls = classify(n, f);
    r.norm1 = norm1;
    r.norminf = norminf;
    *out = r;
  }
  __syncthreads();
}

// Batched scan: persistent CTAs pull systems from a counter.
__global__ void __launch_bounds__(kScanThreads, 2) k_scan_batched(const BatchDesc* __restrict__ dp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ScanShared& sh = *reinterpret_cast<ScanShared*>(smem_raw);
  double* diag = reinterpret_cast<double*>(smem_raw + sizeof(ScanShared));
  __shared__ int64_t s_sys;
  const BatchDesc& d = *dp;
  float* scratch = reinterpret_cast<float*>(d.slot_base + (size_t)blockIdx.x * d.slot_bytes);
  for (;;) {
    if (threadIdx.x == 0) s_sys = atomicAdd(&d.work_ctr[0], 1);
    __syncthreads();
    int64_t s = s_sys;
    __syncthreads();
    if (s >= d.count) break;
    const int n = (int)d.n[s];
    const int64_t nr = d.nrhs[s];
    ScanRes* out = d.scan + s;
    if (n <= 0 || n > kBatchNMax || nr < 1 || nr > kBatchRhsMax) {
      if (threadIdx.x == 0) {
        ScanRes r{};
        r.cls = ASOLVE_CLS_NONE;
        r.flags = 0;
        *out = r;
      }
      continue;
    }
    cta_scan_system(sys_A(d, s), n, sys_B(d, s), (int64_t)n * nr, scratch,
                    d.sympd_tol, d.band_frac, diag, sh, out);
  }
}

// ---- large single system: tile pairs spread over the whole grid ----------
struct LargeScanState {
  int kl, ku, sym_fail, nonfinite, range_bad, b_nonfinite, diag_nonpos;
  int pad;
  double max_diag;
};

__global__ void __launch_bounds__(kScanThreads) k_scan_large_diag(const double* __restrict__ A,
                                                                  int64_t n, double* diag,
                                                                  LargeScanState* st) {
  double md = 0.0;
  bool pos = true;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v = __ldg(A + i * n + i);
    diag[i] = v;
    if (v <= 0.0) pos = false;
    if (v > md) md = v;
  }
  md = warp_max(md);
  if (!__all_sync(0xffffffffu, pos) && (threadIdx.x & 31) == 0) atomicOr(&st->diag_nonpos, 1);
  // max of non-negative doubles via their bit patterns
  if ((threadIdx.x & 31) == 0 && md > 0.0)
    atomicMax((unsigned long long*)&st->max_diag, (unsigned long long)dbits(md));
}

__global__ void __launch_bounds__(kScanThreads, 2) k_scan_large_pairs(const double* __restrict__ A,
                                                                   int64_t n64, const double* diag,
                                                                   float* colpart, float* rowpart,
                                                                   double tol, LargeScanState* st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ScanShared& sh = *reinterpret_cast<ScanShared*>(smem_raw);
  const int n = (int)n64;
  if (threadIdx.x == 0) sh.sym_ok = (st->diag_nonpos == 0 && st->sym_fail == 0) ? 1 : 0;
  __syncthreads();
  int kl_l = 0, ku_l = 0;
  bool nf = false, rb = false, sf = false;
  const int64_t warp_global = (int64_t)blockIdx.x * kScanWarps + (threadIdx.x >> 5);
  const int64_t nwarps = (int64_t)gridDim.x * kScanWarps;
  scan_pairs(A, n, diag, warp_global, nwarps, colpart, rowpart, sh, tol,
             dbits(st->max_diag), kl_l, ku_l, nf, rb, sf);
  kl_l = __reduce_max_sync(0xffffffffu, kl_l);
  ku_l = __reduce_max_sync(0xffffffffu, ku_l);
  if ((threadIdx.x & 31) == 0) {
    if (kl_l) atomicMax(&st->kl, kl_l);
    if (ku_l) atomicMax(&st->ku, ku_l);
  }
  if (nf) atomicOr(&st->nonfinite, 1);
  if (rb) atomicOr(&st->range_bad, 1);
  if (sf) atomicOr(&st->sym_fail, 1);
}

// Final reduction for the large scan: one CTA sums the partials in a fixed
// order, folds in the B check and writes the ScanRes.
__global__ void __launch_bounds__(1024) k_scan_large_final(const double* __restrict__ A,
                                                           int64_t n64, const double* __restrict__ B,
                                                           int64_t nb, const float* colpart,
                                                           const float* rowpart, double band_frac,
                                                           LargeScanState* st, ScanRes* out) {
  __shared__ double red[32];
  const int n = (int)n64;
  const int T = (n + 31) / 32;
  float c1f = 0.f, cif = 0.f;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const float s = kahan_partials(colpart, n, T, j), r = kahan_partials(rowpart, n, T, j);
    c1f = s > c1f ? s : c1f;
    cif = r > cif ? r : cif;
  }
  double c1 = (double)c1f, ci = (double)cif;
  bool bbad = false;
  for (int64_t i = threadIdx.x; i < nb; i += blockDim.x)
    if (is_nonfinite_bits(dbits(B[i]))) bbad = true;
  bbad = __syncthreads_or(bbad) != 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  c1 = warp_max(c1);
  if (lane == 0) red[warp] = c1;
  __syncthreads();
  double norm1 = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) norm1 = red[w] > norm1 ? red[w] : norm1;
  __syncthreads();
  ci = warp_max(ci);
  if (lane == 0) red[warp] = ci;
  __syncthreads();
  double norminf = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) norminf = red[w] > norminf ? red[w] : norminf;
  if (threadIdx.x == 0) {
    ScanRes r;
    r.kl = st->kl;
    r.ku = st->ku;
    int f = 0;
    if (st->nonfinite) f |= SF_NONFINITE;
    if (bbad) f |= SF_B_NONFINITE;
    if (n > 0 && !st->diag_nonpos && !st->sym_fail) f |= SF_SYMPD;
    if (r.ku == 0) f |= SF_LOWER;
    if (r.kl == 0) f |= SF_UPPER;
    if (st->range_bad) f |= SF_NORM_FP64;
    f |= band_flag(n, r.kl, r.ku, band_frac);
    r.flags = f;
    r.cls = classify(n, f);
    r.norm1 = norm1;
    r.norminf = norminf;
    *out = r;
  }
}

// FP64 norms over the whole grid (only when FP32 range is exceeded).
__global__ void k_norms_fp64_cols(const double* __restrict__ A, int64_t n, double* colsum,
                                  double* rowsum) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0, r = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      s += fabs(A[j * n + i]);
      r += fabs(A[i * n + j]);
    }
    colsum[j] = s;
    rowsum[j] = r;
  }
}

size_t scan_batched_smem(int nmax) { return sizeof(ScanShared) + sizeof(double) * (size_t)nmax; }
size_t scan_large_smem() { return sizeof(ScanShared); }
size_t scan_slot_bytes(int nmax) {
  size_t T = (size_t)(nmax + 31) / 32;
  return 2 * T * (size_t)nmax * sizeof(float);
}

}  // namespace asv

// Host-side launchers (used by api.cu).
namespace asv {
cudaError_t launch_scan_batched(const BatchDesc* d, int grid, cudaStream_t st) {
  size_t sm = scan_batched_smem(kBatchNMax);
  cudaError_t e = ASV_SMEM_LIMIT_ONCE(k_scan_batched, sm);
  if (e != cudaSuccess) return e;
  k_scan_batched<<<grid, kScanThreads, sm, st>>>(d);
  return cudaGetLastError();
}

size_t scan_large_workspace(int64_t n) {
  size_t T = (size_t)(n + 31) / 32;
  return sizeof(LargeScanState) + 256 + (size_t)n * sizeof(double) + 2 * T * (size_t)n * sizeof(float) +
         2 * (size_t)n * sizeof(double) + 1024;
}

cudaError_t launch_scan_large(const double* A, int64_t n, const double* B, int64_t nb, double band_frac,
                              double tol, void* ws, ScanRes* out, int num_sms, cudaStream_t st) {
  char* p = (char*)ws;
  LargeScanState* state = (LargeScanState*)p;
  p += 256;
  double* diag = (double*)p;
  p += (size_t)n * sizeof(double);
  size_t T = (size_t)(n + 31) / 32;
  float* colpart = (float*)p;
  p += T * (size_t)n * sizeof(float);
  float* rowpart = (float*)p;
  cudaError_t e = cudaMemsetAsync(state, 0, sizeof(LargeScanState), st);
  if (e != cudaSuccess) return e;
  int g = (int)((n + 255) / 256);
  if (g > num_sms * 4) g = num_sms * 4;
  if (g < 1) g = 1;
  k_scan_large_diag<<<g, kScanThreads, 0, st>>>(A, n, diag, state);
  size_t sm = scan_large_smem();
  e = ASV_SMEM_LIMIT_ONCE(k_scan_large_pairs, sm);
  if (e != cudaSuccess) return e;
  int64_t npairs = (int64_t)T * (T + 1) / 2;
  int64_t grid = (npairs + kScanWarps - 1) / kScanWarps;
  int64_t cap = (int64_t)num_sms * 3;
  if (grid > cap) grid = cap;
  k_scan_large_pairs<<<(int)grid, kScanThreads, sm, st>>>(A, n, diag, colpart, rowpart, tol, state);
  k_scan_large_final<<<1, 1024, 0, st>>>(A, n, B, nb, colpart, rowpart, band_frac, state, out);
  return cudaGetLastError();
}
}  // namespace asv
