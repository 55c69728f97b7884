// classes.cu -- the class-routed batched pipeline (paper Sec. 2, Fig. 2).
//
//   k_route       reads every system's scan result and applies the detection
//                 order of Sec. 2 (banded, lower, upper, sympd, general),
//                 writes the per-system info, and builds one work list per
//                 solver class, largest systems first.
//   k_band_class  Sec. 2.1: banded LU with partial pivoting in band storage
//                 (xGBTRF semantics), band solve, 1-norm estimate.  One warp
//                 per system.
//   k_tri_class   Sec. 2.2 / Eq. 3: forward or back substitution, estimate.
//   k_chol_class  Sec. 2.3: Cholesky; failure sends the system to the LU list.
//   k_lu_class    Sec. 2.4 / Eq. 4: LU with partial pivoting.
//   k_svd_class   Sec. 2.5: one-sided Jacobi SVD and minimum-norm solve for
//                 every system whose solver failed or whose rcond < threshold.
//
// Mixed precision (ASOLVE_PREC_MIXED): Cholesky and LU factor in FP32, the
// solution is refined with FP64 residuals until the normwise backward error
// reaches the target; a factor whose estimated rcond is below 1/kappa_limit,
// or a refinement that stalls, is redone in FP64.  Every class kernel is a
// persistent kernel pulling systems from its list; per-CTA scratch slots
// hold the factors.
#include "cta_linalg.cuh"
#include "cta_ldlt.cuh"
#include "band_warp.cuh"

namespace asv {

__device__ __forceinline__ int round4(int x) { return (x + 3) & ~3; }

__device__ __forceinline__ void write_info_init(asolve_info* inf, const ScanRes& sr, int route,
                                                int status, int precision) {
  asolve_info i;
  i.cls = sr.cls;
  i.route = route;
  i.status = status;
  i.ir_iters = 0;
  i.kl = sr.kl;
  i.ku = sr.ku;
  i.rcond = __longlong_as_double(0x7ff8000000000000ll);
  i.berr = __longlong_as_double(0x7ff8000000000000ll);
  i.svd_rank = -1;
  i.precision = precision;
  i.detail = 0;
  *inf = i;
}

// ------------------------------------------------------------------ router
// One CTA of 1024 threads.  Lists are sorted by n, descending (counting sort).
__global__ void __launch_bounds__(1024) k_route(const BatchDesc* __restrict__ dp) {
  const BatchDesc& d = *dp;
  __shared__ int hist[4][kBatchNMax + 1];
  for (int e = threadIdx.x; e < 4 * (kBatchNMax + 1); e += blockDim.x) (&hist[0][0])[e] = 0;
  __syncthreads();
  const int64_t cap = d.capacity;
  for (int64_t s = threadIdx.x; s < d.count; s += blockDim.x) {
    const int64_t n = d.n[s], nr = d.nrhs[s];
    ScanRes sr = d.scan[s];
    int list = -1, route = ASOLVE_ROUTE_NONE, status = ASOLVE_OK;
    if (n < 0 || nr < 1) {
      status = ASOLVE_E_INVALID;
      sr = ScanRes{};
    } else if (n > kBatchNMax || nr > kBatchRhsMax) {
      status = ASOLVE_E_UNSUPPORTED;
      sr = ScanRes{};
    } else if (n == 0) {
      sr = ScanRes{};
    } else if (sr.flags & (SF_NONFINITE | SF_B_NONFINITE)) {
      status = ASOLVE_E_NONFINITE;
    } else if (d.flags & ASOLVE_FORCE_SVD) {
      list = L_SVD;
      route = ASOLVE_ROUTE_SVD;
    } else if (d.flags & ASOLVE_FORCE_LU) {
      list = L_LU;
      route = ASOLVE_ROUTE_LU;
    } else {
      switch (sr.cls) {
        case ASOLVE_CLS_BANDED:
          list = L_BAND;
          // the tridiagonal specialisation runs the band kernel with kl = ku = 1,
          // whose pivots and operations are xGTTRF's
          route = ((d.flags & ASOLVE_TRIDIAG) && sr.kl == 1 && sr.ku == 1) ? ASOLVE_ROUTE_TRIDIAG
                                                                            : ASOLVE_ROUTE_BAND_LU;
          break;
        case ASOLVE_CLS_LOWER: list = L_TRI; route = ASOLVE_ROUTE_TRI_LOWER; break;
        case ASOLVE_CLS_UPPER: list = L_TRI; route = ASOLVE_ROUTE_TRI_UPPER; break;
        case ASOLVE_CLS_SYMPD: list = L_CHOL; route = ASOLVE_ROUTE_CHOL; break;
        default: list = L_LU; route = ASOLVE_ROUTE_LU; break;
      }
    }
    write_info_init(d.info + s, sr, route, status, ASOLVE_PREC_FP64);
    if (list >= 0 && list < 4) atomicAdd(&hist[list][n], 1);
    if (list == L_SVD) {
      int pos = atomicAdd(&d.list_len[L_SVD], 1);
      d.lists[(int64_t)L_SVD * cap + pos] = (int32_t)s;
    }
  }
  __syncthreads();
  // exclusive prefix over n descending, per list
  if (threadIdx.x < 4) {
    const int l = threadIdx.x;
    int acc = 0;
    for (int n = kBatchNMax; n >= 0; --n) {
      int h = hist[l][n];
      hist[l][n] = acc;
      acc += h;
    }
    d.list_len[l] = acc;
  }
  __syncthreads();
  for (int64_t s = threadIdx.x; s < d.count; s += blockDim.x) {
    const int64_t n = d.n[s];
    const asolve_info& inf = d.info[s];
    if (inf.status != ASOLVE_OK || n <= 0 || n > kBatchNMax || d.nrhs[s] > kBatchRhsMax) continue;
    int list;
    switch (inf.route) {
      case ASOLVE_ROUTE_BAND_LU:
      case ASOLVE_ROUTE_TRIDIAG: list = L_BAND; break;
      case ASOLVE_ROUTE_TRI_LOWER:
      case ASOLVE_ROUTE_TRI_UPPER: list = L_TRI; break;
      case ASOLVE_ROUTE_CHOL: list = L_CHOL; break;
      case ASOLVE_ROUTE_LU: list = L_LU; break;
      default: list = -1;
    }
    if (list < 0) continue;
    int pos = atomicAdd(&hist[list][n], 1);
    d.lists[(int64_t)list * cap + pos] = (int32_t)s;
  }
}

// ------------------------------------------------------------ shared tail
// Primary solver finished: decide on the SVD fallback (Sec. 2.5).  CTA scope.
__device__ void finish_primary(const BatchDesc& d, int64_t s, bool failed, double rc, double* X,
                               int64_t xcount) {
  asolve_info* inf = d.info + s;
  const bool no_rcond = (d.flags & ASOLVE_NO_RCOND) != 0;
  const bool poor = !failed && !no_rcond && !(rc >= d.rcond_threshold);
  if (threadIdx.x == 0)
    inf->rcond = (failed || no_rcond) ? __longlong_as_double(0x7ff8000000000000ll) : rc;
  if (!failed && !poor) {
    if (threadIdx.x == 0) inf->status = ASOLVE_OK;
    return;
  }
  if (d.flags & ASOLVE_NO_APPROX) {
    if (failed)
      for (int64_t i = threadIdx.x; i < xcount; i += blockDim.x) X[i] = 0.0;
    if (threadIdx.x == 0) inf->status = failed ? ASOLVE_E_SINGULAR : ASOLVE_W_ILLCOND;
    return;
  }
  if (threadIdx.x == 0) {
    int pos = atomicAdd(&d.list_len[L_SVD], 1);
    d.lists[(int64_t)L_SVD * d.capacity + pos] = (int32_t)s;
  }
}

// Warp-scope variant of finish_primary for warp-per-system kernels.
__device__ void finish_primary_warp(const BatchDesc& d, int64_t s, bool failed, double rc, double* X,
                                    int64_t xcount) {
  asolve_info* inf = d.info + s;
  const int lane = threadIdx.x & 31;
  const bool no_rcond = (d.flags & ASOLVE_NO_RCOND) != 0;
  const bool poor = !failed && !no_rcond && !(rc >= d.rcond_threshold);
  if (lane == 0) inf->rcond = (failed || no_rcond) ? __longlong_as_double(0x7ff8000000000000ll) : rc;
  if (!failed && !poor) {
    if (lane == 0) inf->status = ASOLVE_OK;
    return;
  }
  if (d.flags & ASOLVE_NO_APPROX) {
    if (failed)
      for (int64_t i = lane; i < xcount; i += 32) X[i] = 0.0;
    if (lane == 0) inf->status = failed ? ASOLVE_E_SINGULAR : ASOLVE_W_ILLCOND;
    return;
  }
  if (lane == 0) {
    int pos = atomicAdd(&d.list_len[L_SVD], 1);
    d.lists[(int64_t)L_SVD * d.capacity + pos] = (int32_t)s;
  }
}

__device__ __forceinline__ int next_item(const BatchDesc& d, int ctr, int* s_item) {
  if (threadIdx.x == 0) *s_item = atomicAdd(&d.work_ctr[ctr], 1);
  __syncthreads();
  int it = *s_item;
  __syncthreads();
  return it;
}

// Dense-class dynamic shared memory: 110 KB (two blocks per SM).
constexpr int kDenseSmem = 110 * 1024;
// FP64 estimates: v (two columns) and xi (3 x 1024 doubles) first, then the 8 warps'
// 32 x 33 tiles of the transposed triangular updates.
constexpr int kEstStageOff = 3 * 1024 * 8 + 64;
static_assert(kEstStageOff + kWarps * 32 * 33 * 8 <= kDenseSmem, "estimate stage");

// Panel width: the n x nb panel plus the 32 x 33 inverse and two 32 x 64
// tiles must fit in kDenseSmem; within that, the autotuner's table may
// choose a narrower panel per size bucket.
template <typename T>
__device__ __forceinline__ int pick_nb(int n, const BatchDesc& d, int kind) {
  const size_t extra = (32 * 33 + 8 + 32 * 65 + 8 + 32 * 64) * sizeof(T) + 64;
  int nb = 32;
  while (nb > 4 && (size_t)n * nb * sizeof(T) + extra > (size_t)kDenseSmem) nb >>= 1;
  // a tuned width (a power of two) may only narrow the panel
  const int t = d.nb_tab[kind + (sizeof(T) == 8 ? 2 : 0)][(n - 1) >> 5];
  if (t >= 4 && t < nb) nb = t >= 16 ? 16 : (t >= 8 ? 8 : 4);
  return nb;
}

// Slot layout of the dense classes: [W (8 * ldw * n)] [piv | perm] [R] [tmp]
// [Linv] [Uinv]; R and tmp hold n x 8 doubles, Linv/Uinv 32 x 32 blocks.
struct DenseSlot {
  void* W;
  int* piv;
  int* perm;
  double* R;
  double* tmp;
  void* Linv;
  void* Uinv;
};
__device__ __forceinline__ DenseSlot dense_slot(const BatchDesc& d, int n) {
  char* base = d.slot_base + (size_t)blockIdx.x * d.slot_bytes;
  DenseSlot s;
  const size_t wbytes = ((size_t)8 * round4(n) * n + 255) & ~(size_t)255;
  s.W = base;
  s.piv = reinterpret_cast<int*>(base + wbytes);
  s.perm = s.piv + 1024;
  s.R = reinterpret_cast<double*>(base + wbytes + 8192);
  s.tmp = s.R + (size_t)8 * 1024;
  s.Linv = reinterpret_cast<void*>(s.tmp + (size_t)8 * 1024);
  s.Uinv = reinterpret_cast<char*>(s.Linv) + (size_t)8 * 32 * 1024;
  return s;
}

template <typename T>
__device__ __noinline__ void copy_to_work(const double* __restrict__ A, int n, T* W, int ldw) {
  cta_copy_block<T, double>(W, ldw, A, n, n, n);
  __syncthreads();
}

// ----------------------------------------------------- mixed refinement
// Solve with FP32 factors, refine with FP64 residuals (Sec. 2.4 / 2.3 solve
// steps, used as the correction solver).  xd, xs: smem.  Returns true when
// every column reached berr <= target; *berr_out = max column berr.
template <typename ApplyF>
__device__ bool refine(const BatchDesc& d, const double* __restrict__ A, const double* __restrict__ B,
                       int n, int nrhs, double norminf, double* xd, float* xs, double* R,
                       ApplyF apply32, double& berr_out, int& iters, CtaRed& red) {
  // column scales are powers of two (exact to apply and to undo); the
  // reciprocal is kept so the per-element scaling is one multiplication
  __shared__ double s_scale[8], s_iscale[8], s_rmax[8];
  // x0 = inv(A32) b, with each column scaled to max-norm in [1, 2) first
  for (int c = 0; c < nrhs; ++c) {
    double m = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(B[(size_t)c * n + i]));
    m = cta_max(m, red);
    if (threadIdx.x == 0) {
      const int k = m > 0.0 ? ilogb(m) : 0;
      s_scale[c] = ldexp(1.0, k);
      s_iscale[c] = ldexp(1.0, -k);
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * nrhs; e += blockDim.x) {
    int c = e / n;
    xs[e] = (float)(B[e] * s_iscale[c]);
  }
  apply32(xs);
  for (int e = threadIdx.x; e < n * nrhs; e += blockDim.x) xd[e] = (double)xs[e] * s_scale[e / n];
  __syncthreads();
  double berr_prev = INFINITY;
  iters = 0;
  bool ok = false;
  for (int it = 0;; ++it) {
    cta_residual(A, n, n, B, xd, nrhs, R, s_rmax);
    double berr = 0.0;
    for (int c = 0; c < nrhs; ++c) {
      double xm = 0.0, bm = 0.0;
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        xm = fmax(xm, fabs(xd[(size_t)c * n + i]));
        bm = fmax(bm, fabs(B[(size_t)c * n + i]));
      }
      xm = cta_max(xm, red);
      bm = cta_max(bm, red);
      double den = norminf * xm + bm;
      double be = den > 0.0 ? s_rmax[c] / den : (s_rmax[c] > 0.0 ? INFINITY : 0.0);
      if (!(be <= berr)) berr = be;  // NaN propagates as "not converged"
    }
    berr_out = berr;
    const bool conv = berr <= d.ir_target_berr;
    if (!conv && (it >= d.ir_max_iter || !(berr < 0.5 * berr_prev))) break;  // stalled
    berr_prev = berr;
    if (threadIdx.x < nrhs) {
      const double m = s_rmax[threadIdx.x];
      const int k = m > 0.0 ? ilogb(m) : 0;
      s_scale[threadIdx.x] = ldexp(1.0, k);
      s_iscale[threadIdx.x] = ldexp(1.0, -k);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * nrhs; e += blockDim.x) {
      int c = e / n;
      xs[e] = (float)(R[e] * s_iscale[c]);
    }
    apply32(xs);
    for (int e = threadIdx.x; e < n * nrhs; e += blockDim.x) {
      int c = e / n;
      xd[e] += (double)xs[e] * s_scale[c];
    }
    __syncthreads();
    ++iters;
    // converged: the correction just applied used the verified residual,
    // so it only removes the remaining O(kappa u32) part of the error
    if (conv) { ok = true; break; }
  }
  __syncthreads();
  return ok;
}

// FP64 backward error of the solution in xd (smem), max over columns.
__device__ double berr_fp64(const double* __restrict__ A, const double* __restrict__ B, int n, int nrhs,
                            double norminf, const double* xd, double* R, CtaRed& red) {
  __shared__ double s_rmax[8];
  cta_residual(A, n, n, B, xd, nrhs, R, s_rmax);
  double berr = 0.0;
  for (int c = 0; c < nrhs; ++c) {
    double xm = 0.0, bm = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      xm = fmax(xm, fabs(xd[(size_t)c * n + i]));
      bm = fmax(bm, fabs(B[(size_t)c * n + i]));
    }
    xm = cta_max(xm, red);
    bm = cta_max(bm, red);
    double den = norminf * xm + bm;
    double be = den > 0.0 ? s_rmax[c] / den : (s_rmax[c] > 0.0 ? INFINITY : 0.0);
    if (!(be <= berr)) berr = be;
  }
  return berr;
}

// --------------------------------------------------------------- LU / Chol
// kind 0: LU, kind 1: Cholesky.  Returns for Cholesky whether the FP64
// factorisation failed (the caller then moves the system to the LU list).
template <int KIND>
__device__ bool dense_system(const BatchDesc& d, int64_t s, unsigned char* smem, CtaRed& red) {
  const int n = (int)d.n[s], nrhs = (int)d.nrhs[s];
  const double* A = sys_A(d, s);
  const double* B = sys_B(d, s);
  double* X = sys_X(d, s);
  const ScanRes sr = d.scan[s];
  asolve_info* inf = d.info + s;
  DenseSlot sl = dense_slot(d, n);
  const int ldw = round4(n);
  const bool no_rcond = (d.flags & ASOLVE_NO_RCOND) != 0;
  int detail = 0;
  // ---- mixed precision attempt (not when magnitudes leave the FP32 range)
  // (the 16-bit modes differ only in the large path's tensor-core updates:
  // here they factor in FP32 as MIXED does)
  if (d.precision != ASOLVE_PREC_FP64 && d.precision != ASOLVE_PREC_FP64_OZ && !(sr.flags & SF_NORM_FP64)) {
    float* W = reinterpret_cast<float*>(sl.W);
    copy_to_work<float>(A, n, W, ldw);
    const int nb = pick_nb<float>(n, d, KIND);
    int f = KIND == 0 ? cta_lu_factor<float>(W, ldw, n, sl.piv, reinterpret_cast<float*>(smem), nb)
                      : cta_chol_factor<float>(W, ldw, n, reinterpret_cast<float*>(smem), nb);
    if (KIND == 0 && f == 0) cta_build_perm(sl.piv, n, sl.perm, reinterpret_cast<int*>(smem));
    if (f == 0) {
      float* Li = reinterpret_cast<float*>(sl.Linv);
      float* Ui = reinterpret_cast<float*>(sl.Uinv);
      float* tmp = reinterpret_cast<float*>(sl.tmp);
      cta_block_inverses<float>(W, ldw, n, true, KIND == 0, Li);
      if (KIND == 0) cta_block_inverses<float>(W, ldw, n, false, false, Ui);
      float* v = reinterpret_cast<float*>(smem);
      float* xi = v + 2 * n;
      float* stage = reinterpret_cast<float*>(smem + 8192 * 2 + 64);  // after v, xi (n <= 1024)
      // the factor's transpose, in the second half of the slot's working
      // area (sized for an FP64 factor): the transposed solves of the
      // estimate and of the Cholesky applications read it coalesced
      float* WT = W + (size_t)ldw * n;
      if (KIND == 1 || !no_rcond) cta_transpose<float>(W, ldw, n, WT, stage);
      auto apply_est = [&](float* x, bool tr, int k) {
        if (KIND == 0) cta_lu_apply<float, float>(W, ldw, n, sl.perm, x, n, k, tr, tmp, Li, Ui, stage, WT);
        else cta_chol_apply<float, float>(W, ldw, n, x, n, k, Li, stage, WT);
      };
      double rc = __longlong_as_double(0x7ff8000000000000ll);
      bool gate_ok = true;
      if (!no_rcond) {
        double est = cta_est_inv_norm1<float>(n, v, xi, apply_est, red);
        rc = rcond_from(sr.norm1, est);
        gate_ok = rc >= 1.0 / d.ir_kappa_limit;
      }
      if (gate_ok) {
        // FP64 iterate lives in X (global); FP32 correction and the
        // transposed-update stage in shared memory
        float* xs = reinterpret_cast<float*>(smem);
        float* stage = reinterpret_cast<float*>(smem + (size_t)4 * 1024 * 8 + 64);
        auto apply32 = [&](float* x) {
          if (KIND == 0) cta_lu_apply<float, float>(W, ldw, n, sl.perm, x, n, nrhs, false, tmp, Li, Ui, stage);
          else cta_chol_apply<float, float>(W, ldw, n, x, n, nrhs, Li, stage, WT);
        };
        double berr;
        int iters;
        bool ok = refine(d, A, B, n, nrhs, sr.norminf, X, xs, sl.R, apply32, berr, iters, red);
        if (ok) {
          if (threadIdx.x == 0) {
            inf->rcond = rc;
            inf->berr = berr;
            inf->ir_iters = iters;
            inf->precision = ASOLVE_PREC_MIXED;
            inf->status = ASOLVE_OK;
            inf->detail |= detail;
          }
          __syncthreads();
          return false;
        }
        detail |= 2;
      } else {
        detail |= 1;
      }
    } else if (KIND == 1) {
      detail |= 4;
    }
  }
  // ---- FP64 path
  double* W = reinterpret_cast<double*>(sl.W);
  copy_to_work<double>(A, n, W, ldw);
  const int nb = pick_nb<double>(n, d, KIND);
  int f = KIND == 0 ? cta_lu_factor<double>(W, ldw, n, sl.piv, reinterpret_cast<double*>(smem), nb)
                    : cta_chol_factor<double>(W, ldw, n, reinterpret_cast<double*>(smem), nb);
  if (KIND == 0 && f == 0) cta_build_perm(sl.piv, n, sl.perm, reinterpret_cast<int*>(smem));
  if (threadIdx.x == 0) {
    inf->detail |= detail;
    inf->precision = ASOLVE_PREC_FP64;
  }
  if (KIND == 1 && f != 0) {
    __syncthreads();
    return true;  // not sympd after all (Sec. 2.3): general solver
  }
  const bool failed = f != 0;
  double rc = __longlong_as_double(0x7ff8000000000000ll);
  if (!failed) {
    double* xd = reinterpret_cast<double*>(smem);
    for (int e = threadIdx.x; e < n * nrhs; e += blockDim.x) xd[e] = B[e];
    if (KIND == 0) cta_lu_apply<double, double>(W, ldw, n, sl.perm, xd, n, nrhs, false, sl.tmp);
    else cta_chol_apply<double, double>(W, ldw, n, xd, n, nrhs);
    for (int e = threadIdx.x; e < n * nrhs; e += blockDim.x) X[e] = xd[e];
    __syncthreads();
    if (d.flags & ASOLVE_BERR) {
      double be = berr_fp64(A, B, n, nrhs, sr.norminf, xd, sl.R, red);
      if (threadIdx.x == 0) inf->berr = be;
    }
    if (!no_rcond) {
      // FP64 estimate by substitution: on an ill-conditioned factor a
      // product with explicit block inverses would corrupt the estimate
      double* v = reinterpret_cast<double*>(smem);
      double* xi = v + 2 * n;
      double* stage = reinterpret_cast<double*>(smem + kEstStageOff);
      auto apply_est = [&](double* x, bool tr, int k) {
        if (KIND == 0) cta_lu_apply<double, double>(W, ldw, n, sl.perm, x, n, k, tr, sl.tmp, nullptr, nullptr, stage);
        else cta_chol_apply<double, double>(W, ldw, n, x, n, k, nullptr, stage);
      };
      double est = cta_est_inv_norm1<double>(n, v, xi, apply_est, red);
      rc = rcond_from(sr.norm1, est);
    }
  }
  __syncthreads();
  finish_primary(d, s, failed, rc, X, (int64_t)n * nrhs);
  __syncthreads();
  return false;
}

// The symmetric-indefinite route (ASOLVE_SYM_INDEF): Bunch-Kaufman LDL^T
// in FP64, solve, FP64 backward error, estimate, then the SVD decision of
// Sec. 2.5 as for every route.
__device__ void dense_ldlt(const BatchDesc& d, int64_t s, unsigned char* smem, CtaRed& red, int route) {
  const int n = (int)d.n[s], nrhs = (int)d.nrhs[s];
  const double* A = sys_A(d, s);
  const double* B = sys_B(d, s);
  double* X = sys_X(d, s);
  const ScanRes sr = d.scan[s];
  asolve_info* inf = d.info + s;
  DenseSlot sl = dense_slot(d, n);
  const int ldw = round4(n);
  double* W = reinterpret_cast<double*>(sl.W);
  copy_to_work<double>(A, n, W, ldw);
  const int f = cta_ldlt_factor(W, ldw, n, sl.piv, reinterpret_cast<double*>(smem), red);
  if (threadIdx.x == 0) {
    inf->route = route;
    inf->precision = ASOLVE_PREC_FP64;
  }
  const bool failed = f != 0;
  double rc = __longlong_as_double(0x7ff8000000000000ll);
  if (!failed) {
    double* xd = reinterpret_cast<double*>(smem);
    for (int e = threadIdx.x; e < n * nrhs; e += blockDim.x) xd[e] = B[e];
    cta_ldlt_solve(W, ldw, n, sl.piv, xd, n, nrhs);
    for (int e = threadIdx.x; e < n * nrhs; e += blockDim.x) X[e] = xd[e];
    __syncthreads();
    if (d.flags & ASOLVE_BERR) {
      const double be = berr_fp64(A, B, n, nrhs, sr.norminf, xd, sl.R, red);
      if (threadIdx.x == 0) inf->berr = be;
    }
    if (!(d.flags & ASOLVE_NO_RCOND)) {
      double* v = reinterpret_cast<double*>(smem);
      double* xi = v + 2 * n;
      auto apply_est = [&](double* x, bool, int k) { cta_ldlt_solve(W, ldw, n, sl.piv, x, n, k); };
      const double est = cta_est_inv_norm1<double>(n, v, xi, apply_est, red);
      rc = rcond_from(sr.norm1, est);
    }
  }
  __syncthreads();
  finish_primary(d, s, failed, rc, X, (int64_t)n * nrhs);
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads, 2) k_chol_class(const BatchDesc* __restrict__ dp) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ CtaRed red;
  __shared__ int s_item;
  const BatchDesc& d = *dp;
  const int len = d.list_len[L_CHOL];
  for (;;) {
    int it = next_item(d, 8 + L_CHOL, &s_item);
    if (it >= len) break;
    int64_t s = d.lists[(int64_t)L_CHOL * d.capacity + it];
    bool to_lu = dense_system<1>(d, s, smem, red);
    if (to_lu && threadIdx.x == 0) {
      // not positive definite after all (Sec. 2.3): the general solver, or
      // with ASOLVE_SYM_INDEF the symmetric-indefinite one
      d.info[s].route = (d.flags & ASOLVE_SYM_INDEF) ? ASOLVE_ROUTE_CHOL_FAIL_LDLT : ASOLVE_ROUTE_CHOL_FAIL_LU;
      int pos = atomicAdd(&d.list_len[L_LU], 1);
      d.lists[(int64_t)L_LU * d.capacity + pos] = (int32_t)s;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kThreads, 2) k_lu_class(const BatchDesc* __restrict__ dp) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ CtaRed red;
  __shared__ int s_item;
  const BatchDesc& d = *dp;
  const int len = d.list_len[L_LU];
  for (;;) {
    int it = next_item(d, 8 + L_LU, &s_item);
    if (it >= len) break;
    int64_t s = d.lists[(int64_t)L_LU * d.capacity + it];
    const int rt = d.info[s].route;
    if (rt == ASOLVE_ROUTE_CHOL_FAIL_LDLT ||
        (rt == ASOLVE_ROUTE_LU && (d.flags & ASOLVE_SYM_INDEF) && !(d.flags & ASOLVE_FORCE_LU) &&
         cta_is_symmetric(sys_A(d, s), (int)d.n[s], d.sympd_tol))) {
      dense_ldlt(d, s, smem, red, rt == ASOLVE_ROUTE_CHOL_FAIL_LDLT ? rt : ASOLVE_ROUTE_LDLT);
      continue;
    }
    dense_system<0>(d, s, smem, red);
  }
}

// ------------------------------------------------------------- triangular
__global__ void __launch_bounds__(kThreads, 2) k_tri_class(const BatchDesc* __restrict__ dp) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ CtaRed red;
  __shared__ int s_item;
  const BatchDesc& d = *dp;
  const int len = d.list_len[L_TRI];
  for (;;) {
    int it = next_item(d, 8 + L_TRI, &s_item);
    if (it >= len) break;
    const int64_t s = d.lists[(int64_t)L_TRI * d.capacity + it];
    const int n = (int)d.n[s], nrhs = (int)d.nrhs[s];
    const double* A = sys_A(d, s);
    const double* B = sys_B(d, s);
    double* X = sys_X(d, s);
    const ScanRes sr = d.scan[s];
    const bool lower = d.info[s].route == ASOLVE_ROUTE_TRI_LOWER;
    DenseSlot sl = dense_slot(d, n);
    bool zero = false;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      if (A[(size_t)i * n + i] == 0.0) zero = true;
    const bool failed = __syncthreads_or(zero) != 0;
    double rc = __longlong_as_double(0x7ff8000000000000ll);
    if (!failed) {
      double* xd = reinterpret_cast<double*>(smem);
      for (int e = threadIdx.x; e < n * nrhs; e += blockDim.x) xd[e] = B[e];
      cta_tri_solve<double, double>(A, n, n, lower, false, false, xd, n, nrhs);
      for (int e = threadIdx.x; e < n * nrhs; e += blockDim.x) X[e] = xd[e];
      __syncthreads();
      if (d.flags & ASOLVE_BERR) {
        double be = berr_fp64(A, B, n, nrhs, sr.norminf, xd, sl.R, red);
        if (threadIdx.x == 0) d.info[s].berr = be;
      }
      if (!(d.flags & ASOLVE_NO_RCOND)) {
        double* v = reinterpret_cast<double*>(smem);
        double* xi = v + 2 * n;
        double* stage = reinterpret_cast<double*>(smem + kEstStageOff);
        auto apply_est = [&](double* x, bool tr, int k) {
          cta_tri_solve<double, double>(A, n, n, lower, tr, false, x, n, k, nullptr, stage);
        };
        double est = cta_est_inv_norm1<double>(n, v, xi, apply_est, red);
        rc = rcond_from(sr.norm1, est);
      }
    }
    __syncthreads();
    finish_primary(d, s, failed, rc, X, (int64_t)n * nrhs);
    __syncthreads();
  }
}

// ------------------------------------------------------------------ banded
// Band storage, warp_band_lu and the sweeps live in band_warp.cuh.  The
// batched band kernel gives every warp a ring for register windows of up
// to kBandR registers (kl + ku < 32 kBandR); wider bands use the
// global-memory sweep.
constexpr int kBandR = 2;
constexpr int kBandCols = 2;  // vectors per sweep: the estimator's first product
constexpr int kBandRingBytes = band_ring_doubles(kBandR, kBandCols) * 8 + 64;  // ring + pivot ring, per warp

// x (n x k, ld n, k = 1 or 2) <- inv(A) x: the k columns share one pair of
// sweeps when the register window fits, else column by column on the
// global-memory routine.  (The right-hand sides of a solve go one sweep
// each: sweeping all of them at once measured slower, the SM's FP64 pipe
// and issue slots being shared by every warp's sweep.)
__device__ void band_solve_cols(const WarpBand& b, double* x, int k, double* ring, int* pring) {
  // the factor and x were written with ordinary stores; the sweeps read
  // them through cp.async
  __syncwarp();
  __threadfence();
  const int need = (b.kv + 1 + 31) / 32;
  if (need <= kBandR) {
    if (k == 2) {
      if (need <= 1) band_apply<1, 2, true>(b.F, b.ldf, b.n, b.kl, b.ku, b.piv, x, ring, pring, b.n, b.rd);
      else band_apply<2, 2, true>(b.F, b.ldf, b.n, b.kl, b.ku, b.piv, x, ring, pring, b.n, b.rd);
    } else {
      if (need <= 1) band_apply<1, 1, true>(b.F, b.ldf, b.n, b.kl, b.ku, b.piv, x, ring, pring, b.n, b.rd);
      else band_apply<2, 1, true>(b.F, b.ldf, b.n, b.kl, b.ku, b.piv, x, ring, pring, b.n, b.rd);
    }
  } else {
    for (int c = 0; c < k; ++c) warp_band_apply(b, x + (size_t)c * b.n, false);
  }
}

// Warp-scope estimator (same iteration as cta_est_inv_norm1, whose closing
// vector of alternating signs likewise rides along the first product, as
// the second column: xi = v + n).
__device__ double warp_est_inv_norm1(const WarpBand& b, double* v, double* xi, double* ring, int* pring) {
  const int lane = threadIdx.x & 31;
  const int n = b.n;
  if (n == 1) {
    if (lane == 0) v[0] = 1.0;
    band_solve_cols(b, v, 1, ring, pring);
    return fabs(v[0]);
  }
  for (int i = lane; i < n; i += 32) {
    v[i] = 1.0 / (double)n;
    xi[i] = ((i & 1) ? -1.0 : 1.0) * (1.0 + (double)i / (double)(n - 1));
  }
  band_solve_cols(b, v, 2, ring, pring);
  double temp = 0.0;
  for (int i = lane; i < n; i += 32) temp += fabs(xi[i]);
  temp = 2.0 * warp_sum(temp) / (double)(3 * n);
  auto sum_abs = [&]() {
    double s = 0.0;
    for (int i = lane; i < n; i += 32) s += fabs(v[i]);
    return warp_sum(s);
  };
  auto argmax = [&]() {
    double best = -1.0;
    int bi = 0x7fffffff;
    for (int i = lane; i < n; i += 32) {
      double a = fabs(v[i]);
      if (a > best) { best = a; bi = i; }
    }
    warp_argmax_first(best, bi);
    return bi;
  };
  double est = sum_abs();
  for (int i = lane; i < n; i += 32) {
    double sg = v[i] >= 0.0 ? 1.0 : -1.0;
    xi[i] = sg;
    v[i] = sg;
  }
  __syncwarp();
  band_sweep_any(b, v, true, ring, pring, kBandR);
  int k = 2;
  for (;;) {
    const int j = argmax();
    if (j < 0 || j >= n) return __longlong_as_double(0x7ff8000000000000ll);
    __syncwarp();
    for (int i = lane; i < n; i += 32) v[i] = (i == j) ? 1.0 : 0.0;
    __syncwarp();
    band_sweep_any(b, v, false, ring, pring, kBandR);
    const double estold = est;
    est = sum_abs();
    bool same = true;
    for (int i = lane; i < n; i += 32)
      if ((v[i] >= 0.0 ? 1.0 : -1.0) != xi[i]) same = false;
    same = __all_sync(0xffffffffu, same);
    if (same || est <= estold) break;
    for (int i = lane; i < n; i += 32) {
      double sg = v[i] >= 0.0 ? 1.0 : -1.0;
      xi[i] = sg;
      v[i] = sg;
    }
    __syncwarp();
    band_sweep_any(b, v, true, ring, pring, kBandR);
    const int jn = argmax();
    ++k;
    if (jn < 0 || jn >= n) return __longlong_as_double(0x7ff8000000000000ll);
    const double vj = v[j], vjn = fabs(v[jn]);
    __syncwarp();
    if (vj == vjn || k > 5) break;
  }
  __syncwarp();
  return temp > est ? temp : est;
}

// One warp per banded system.  Each warp owns 1/8 of its CTA's slot; a
// system whose band storage does not fit there is left for the second
// phase, where warp 0 of a CTA uses the whole slot.
__global__ void __launch_bounds__(kThreads) k_band_class(const BatchDesc* __restrict__ dp) {
  extern __shared__ __align__(16) unsigned char band_smem[];
  const BatchDesc& d = *dp;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double* ring = reinterpret_cast<double*>(band_smem + (size_t)w * kBandRingBytes);
  int* pring = reinterpret_cast<int*>(band_smem + (size_t)w * kBandRingBytes + band_ring_doubles(kBandR, kBandCols) * 8);
  const int len = d.list_len[L_BAND];
  const size_t sub = (size_t)d.slot_bytes / kWarps;
  for (int phase = 0; phase < 2; ++phase) {
    if (phase == 1) {
      __syncthreads();
      if (w != 0) return;
    }
    char* base = d.slot_base + (size_t)blockIdx.x * d.slot_bytes + (phase == 0 ? w * sub : 0);
    const size_t avail = phase == 0 ? sub : (size_t)d.slot_bytes;
    for (;;) {
      int it = 0;
      if (lane == 0) it = atomicAdd(&d.work_ctr[8 + L_BAND + (phase ? 8 : 0)], 1);
      it = __shfl_sync(0xffffffffu, it, 0);
      if (it >= len) break;
      const int64_t s = d.lists[(int64_t)L_BAND * d.capacity + it];
      const int n = (int)d.n[s], nrhs = (int)d.nrhs[s];
      const ScanRes sr = d.scan[s];
      WarpBand b;
      b.n = n; b.kl = sr.kl; b.ku = sr.ku; b.kv = sr.kl + sr.ku; b.ldf = 2 * sr.kl + sr.ku + 1;
      const size_t fbytes = ((size_t)b.ldf * n * 8 + 255) & ~(size_t)255;
      const size_t need = fbytes + (size_t)n * 4 + 3 * (size_t)n * 8 + 1024;
      const bool fits = need <= sub;
      if (phase == 0 ? !fits : (fits || need > avail)) {
        if (phase == 1 && !fits && need > avail && lane == 0) {
          d.info[s].status = ASOLVE_E_UNSUPPORTED;  // cannot happen for n <= 1024
        }
        continue;
      }
      b.F = reinterpret_cast<double*>(base);
      b.piv = reinterpret_cast<int*>(base + fbytes);
      double* v = reinterpret_cast<double*>(base + fbytes + (((size_t)n * 4 + 255) & ~(size_t)255));
      double* xi = v + n;
      b.rd = xi + n;  // 1 / U(j,j) of the factorisation, for the sweeps
      const double* A = sys_A(d, s);
      const double* B = sys_B(d, s);
      double* X = sys_X(d, s);
      // pack (Sec. 2.1 compact storage) with zeroed fill rows
      for (int64_t e = lane; e < (int64_t)b.ldf * n; e += 32) b.F[e] = 0.0;
      __syncwarp();
      for (int j = 0; j < n; ++j) {
        const int lo = max(0, j - b.ku), hi = min(n - 1, j + b.kl);
        for (int i = lo + lane; i <= hi; i += 32) b.at(i, j) = A[(size_t)j * n + i];
      }
      __syncwarp();
      const int f = warp_band_lu(b);
      const bool failed = f != 0;
      double rc = __longlong_as_double(0x7ff8000000000000ll);
      if (!failed) {
        for (int64_t e = lane; e < (int64_t)n * nrhs; e += 32) X[e] = B[e];
        for (int c = 0; c < nrhs; ++c) band_solve_cols(b, X + (size_t)c * n, 1, ring, pring);
        __syncwarp();
        if (!(d.flags & ASOLVE_NO_RCOND)) rc = rcond_from(sr.norm1, warp_est_inv_norm1(b, v, xi, ring, pring));
        if (d.flags & ASOLVE_BERR) {
          // FP64 backward error over the band: r = b - A x, A read in band form
          double berr = 0.0;
          for (int c = 0; c < nrhs; ++c) {
            const double* xc = X + (size_t)c * n;
            const double* bc = B + (size_t)c * n;
            double rm = 0.0, xm = 0.0, bm = 0.0;
            for (int i = lane; i < n; i += 32) {
              double acc = 0.0;
              const int lo = max(0, i - sr.kl), hi = min(n - 1, i + sr.ku);
              for (int j = lo; j <= hi; ++j) acc = fma(A[(size_t)j * n + i], xc[j], acc);
              rm = fmax(rm, fabs(bc[i] - acc));
              xm = fmax(xm, fabs(xc[i]));
              bm = fmax(bm, fabs(bc[i]));
            }
            rm = warp_max(rm);
            xm = warp_max(xm);
            bm = warp_max(bm);
            const double den = sr.norminf * xm + bm;
            const double be = den > 0.0 ? rm / den : (rm > 0.0 ? INFINITY : 0.0);
            if (!(be <= berr)) berr = be;
          }
          if (lane == 0) d.info[s].berr = berr;
        }
      }
      finish_primary_warp(d, s, failed, rc, X, (int64_t)n * nrhs);
      __syncwarp();
    }
  }
}

// ------------------------------------------------------------------- SVD
// One-sided Jacobi (Hestenes) with the round-robin parallel ordering; a pair
// (p < q) is rotated when |g_p.g_q| > n eps ||g_p|| ||g_q||; sweeps end after
// one without rotation (at most 30).  Then x = sum_{sigma_i > tau} v_i
// (u_i^T b) / sigma_i with u_i = g_i / sigma_i (Sec. 2.5).
//
// A thread-block cluster of kSvdCluster CTAs works on one system: the
// pairs of a round are spread over all warps of the cluster and rounds are
// separated by hardware cluster barriers.  G = A V and V live in the
// leader CTA's scratch slot (global memory, L2-resident).
constexpr int kSvdCluster = 8;

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
__device__ __forceinline__ unsigned cluster_ctarank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// address of `p` (this CTA's shared variable) in the shared memory of CTA `rank`
__device__ __forceinline__ unsigned dsmem_addr(const void* p, unsigned rank) {
  unsigned a = (unsigned)__cvta_generic_to_shared(p), r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ int dsmem_ld(unsigned addr) {
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ void dsmem_or(unsigned addr, int v) {
  asm volatile("red.shared::cluster.or.b32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// One warp rotates the column pair (p, q) of G and V if they are not yet
// orthogonal to the tolerance.  Returns true when it rotated.
__device__ bool jacobi_pair(double* G, double* V, int n, int p, int q, double tol) {
  const int lane = threadIdx.x & 31;
  double* gp = G + (size_t)p * n;
  double* gq = G + (size_t)q * n;
  double xr[32], yr[32];
#pragma unroll
  for (int t = 0; t < 32; ++t) {
    const int k = lane + 32 * t;
    xr[t] = (k < n) ? gp[k] : 0.0;
    yr[t] = (k < n) ? gq[k] : 0.0;
  }
  double al = 0.0, be = 0.0, ga = 0.0;
#pragma unroll
  for (int t = 0; t < 32; ++t) {
    al = fma(xr[t], xr[t], al);
    be = fma(yr[t], yr[t], be);
    ga = fma(xr[t], yr[t], ga);
  }
  al = warp_sum(al);
  be = warp_sum(be);
  ga = warp_sum(ga);
  if (!(fabs(ga) > tol * sqrt(al) * sqrt(be))) return false;
  const double zeta = (be - al) / (2.0 * ga);
  const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  const double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
#pragma unroll
  for (int u = 0; u < 32; ++u) {
    const int k = lane + 32 * u;
    if (k < n) {
      gp[k] = c * xr[u] - sn * yr[u];
      gq[k] = sn * xr[u] + c * yr[u];
    }
  }
  double* vp = V + (size_t)p * n;
  double* vq = V + (size_t)q * n;
#pragma unroll
  for (int u = 0; u < 32; ++u) {
    const int k = lane + 32 * u;
    xr[u] = (k < n) ? vp[k] : 0.0;
    yr[u] = (k < n) ? vq[k] : 0.0;
  }
#pragma unroll
  for (int u = 0; u < 32; ++u) {
    const int k = lane + 32 * u;
    if (k < n) {
      vp[k] = c * xr[u] - sn * yr[u];
      vq[k] = sn * xr[u] + c * yr[u];
    }
  }
  return true;
}

__global__ void __cluster_dims__(kSvdCluster, 1, 1) __launch_bounds__(kThreads, 1)
    k_svd_class(const BatchDesc* __restrict__ dp) {
  __shared__ int s_item, s_rot;
  __shared__ double s_red[kWarps];
  const BatchDesc& d = *dp;
  const unsigned crank = cluster_ctarank();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int cw = (int)crank * kWarps + w;        // warp index within the cluster
  const int ncw = kSvdCluster * kWarps;           // warps per cluster
  const int ctid = (int)crank * kThreads + threadIdx.x;
  const int nct = kSvdCluster * kThreads;
  const int leader_block = blockIdx.x - (int)crank;
  const unsigned item_addr = dsmem_addr(&s_item, 0);
  const unsigned rot_addr = dsmem_addr(&s_rot, 0);
  const int len = *(volatile int*)&d.list_len[L_SVD];
  for (;;) {
    if (crank == 0 && threadIdx.x == 0) s_item = atomicAdd(&d.work_ctr[8 + L_SVD], 1);
    cluster_sync_all();
    const int it = dsmem_ld(item_addr);
    cluster_sync_all();
    if (it >= len) break;
    const int64_t s = d.lists[(int64_t)L_SVD * d.capacity + it];
    const int n = (int)d.n[s], nrhs = (int)d.nrhs[s];
    const double* A = sys_A(d, s);
    const double* B = sys_B(d, s);
    double* X = sys_X(d, s);
    char* base = d.slot_base + (size_t)leader_block * d.slot_bytes;
    double* G = reinterpret_cast<double*>(base);
    double* V = G + (size_t)n * n;
    double* sigma = V + (size_t)n * n;
    double* wv = sigma + n;
    for (int64_t e = ctid; e < (int64_t)n * n; e += nct) {
      G[e] = A[e];
      V[e] = ((e % n) == (e / n)) ? 1.0 : 0.0;
    }
    cluster_sync_all();
    const int np = (n + 1) & ~1;  // players; index n (odd n) is a dummy
    const double tol = (double)n * kEps;
    for (int sweep = 0; sweep < 30; ++sweep) {
      if (crank == 0 && threadIdx.x == 0) s_rot = 0;
      cluster_sync_all();
      bool rotated = false;
      for (int r = 0; r < np - 1; ++r) {
        for (int pi = cw; pi < np / 2; pi += ncw) {
          int a, b;
          if (pi == 0) { a = 0; b = 1 + r % (np - 1); }
          else { a = 1 + (pi + r) % (np - 1); b = 1 + (np - 1 - pi + r) % (np - 1); }
          const int p = min(a, b), q = max(a, b);
          if (q >= n) continue;
          if (jacobi_pair(G, V, n, p, q, tol)) rotated = true;
        }
        cluster_sync_all();
      }
      if (__syncthreads_or(rotated) && threadIdx.x == 0) dsmem_or(rot_addr, 1);
      cluster_sync_all();
      const int any = dsmem_ld(rot_addr);
      cluster_sync_all();
      if (!any) break;
    }
    for (int j = cw; j < n; j += ncw) {
      double sacc = 0.0;
      const double* g = G + (size_t)j * n;
      for (int k = lane; k < n; k += 32) sacc = fma(g[k], g[k], sacc);
      sacc = warp_sum(sacc);
      if (lane == 0) sigma[j] = sqrt(sacc);
    }
    cluster_sync_all();
    // truncation threshold and rank (every CTA computes them redundantly)
    double smax = 0.0;
    for (int i = threadIdx.x; i < n; i += kThreads) smax = fmax(smax, sigma[i]);
    smax = warp_max(smax);
    if (lane == 0) s_red[w] = smax;
    __syncthreads();
    smax = 0.0;
    for (int k = 0; k < kWarps; ++k) smax = fmax(smax, s_red[k]);
    const double tau = (d.svd_trunc_rel > 0.0 ? d.svd_trunc_rel : (double)n * kEps) * smax;
    int rank = 0;
    for (int i = threadIdx.x; i < n; i += kThreads) rank += sigma[i] > tau ? 1 : 0;
    __syncthreads();
    {
      int rr = warp_sum(rank);
      __shared__ int s_rank[kWarps];
      if (lane == 0) s_rank[w] = rr;
      __syncthreads();
      rank = 0;
      for (int k = 0; k < kWarps; ++k) rank += s_rank[k];
    }
    for (int c = 0; c < nrhs; ++c) {
      const double* bc = B + (size_t)c * n;
      for (int i = cw; i < n; i += ncw) {
        const double si = sigma[i];
        double wi = 0.0;
        if (si > tau) {
          const double* g = G + (size_t)i * n;
          double dsum = 0.0;
          for (int k = lane; k < n; k += 32) dsum += (g[k] / si) * bc[k];
          dsum = warp_sum(dsum);
          wi = dsum / si;
        }
        if (lane == 0) wv[i] = wi;
      }
      cluster_sync_all();
      for (int r = ctid; r < n; r += nct) {
        double x = 0.0;
        for (int i = 0; i < n; ++i) x += V[(size_t)i * n + r] * wv[i];
        X[(size_t)c * n + r] = x;
      }
      cluster_sync_all();
    }
    if (crank == 0 && threadIdx.x == 0) {
      d.info[s].svd_rank = rank;
      d.info[s].status = ASOLVE_W_APPROX;
    }
    cluster_sync_all();
  }
}

// --------------------------------------------------------------- launchers
size_t dense_slot_bytes(int nmax) {
  size_t w = ((size_t)8 * ((nmax + 3) & ~3) * nmax + 255) & ~(size_t)255;
  size_t svd = 2 * (size_t)8 * nmax * nmax + 2 * (size_t)8 * nmax + 1024;
  size_t dense = w + 8192 + 2 * (size_t)8 * 8 * 1024 + 2 * (size_t)8 * 32 * 1024 + 1024;
  return ((svd > dense ? svd : dense) + 4095) & ~(size_t)4095;
}

// Shared memory limits of the class kernels on the current device (once per
// device; contexts on several devices each call it).
cudaError_t set_class_attrs() {
  static PerDeviceOnce once;
  return once.run([]() {
    cudaError_t e;
    e = cudaFuncSetAttribute(k_chol_class, cudaFuncAttributeMaxDynamicSharedMemorySize, kDenseSmem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_lu_class, cudaFuncAttributeMaxDynamicSharedMemorySize, kDenseSmem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_tri_class, cudaFuncAttributeMaxDynamicSharedMemorySize, kDenseSmem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_band_class, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kWarps * kBandRingBytes);
  });
}

cudaError_t launch_route(const BatchDesc* d, cudaStream_t st) {
  k_route<<<1, 1024, 0, st>>>(d);
  return cudaGetLastError();
}
cudaError_t launch_band(const BatchDesc* d, int grid, cudaStream_t st) {
  k_band_class<<<grid, kThreads, kWarps * kBandRingBytes, st>>>(d);
  return cudaGetLastError();
}
cudaError_t launch_tri(const BatchDesc* d, int grid, cudaStream_t st) {
  k_tri_class<<<grid, kThreads, kDenseSmem, st>>>(d);
  return cudaGetLastError();
}
cudaError_t launch_chol(const BatchDesc* d, int grid, cudaStream_t st) {
  k_chol_class<<<grid, kThreads, kDenseSmem, st>>>(d);
  return cudaGetLastError();
}
cudaError_t launch_lu(const BatchDesc* d, int grid, cudaStream_t st) {
  k_lu_class<<<grid, kThreads, kDenseSmem, st>>>(d);
  return cudaGetLastError();
}
cudaError_t launch_svd(const BatchDesc* d, int grid, cudaStream_t st) {
  grid = (grid + kSvdCluster - 1) / kSvdCluster * kSvdCluster;
  k_svd_class<<<grid, kThreads, 0, st>>>(d);
  return cudaGetLastError();
}

}  // namespace asv
