// band_spike.cuh -- partitioned band solve without pivoting (truncated
// SPIKE) for long band systems that are diagonally dominant.
//
// Sec. 2.1 solves a band system with GBTRF / GBTRS / GBCON: LU with partial
// pivoting, whose every step depends on the previous one.  On a matrix that
// is diagonally dominant by rows or by columns, elimination without
// pivoting is stable (growth factor at most 2), and by columns partial
// pivoting takes no interchange at all.  Such a matrix is cut into P blocks
// of m rows; with D = diag(A_bb):
//   A x = f  <=>  x_b + V_b x_{b+1}^T + W_b x_{b-1}^B = g_b,  g_b = A_bb^-1 f_b,
// V_b = A_bb^-1 A_{b,b+1} (its columns: the first ku columns of block b+1),
// W_b = A_bb^-1 A_{b,b-1} (the last kl columns of block b-1), x^T the first
// ku and x^B the last kl entries of a block.  On dominant matrices the
// spikes decay away from the coupling corner; when the far rows (V_b's top
// ku, W_b's bottom kl) are below a bound, dropping them leaves one
// independent system of order kl + ku per block boundary b:
//   [ I      VB_b ] [ x_b^B     ]   [ g_b^B     ]
//   [ WT_b+1  I   ] [ x_{b+1}^T ] = [ g_{b+1}^T ]
// (VB: V's bottom kl rows, WT: W's top ku rows), and then
//   x_b = A_bb^-1 (f_b - A_{b,b+1} x_{b+1}^T - A_{b,b-1} x_{b-1}^B).
// A^T is a band matrix with kl and ku exchanged and the same diagonal
// blocks (A_bb^T = U^T L^T), so the solves with A^T that the condition
// estimate needs take the same steps on the transposed couplings.
//
// Every routine here is the work of one thread on plain pointers, so that
// the kernels in band_large.cu are one call per thread and the same code
// also compiles as host C++.
#pragma once

#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define SPK_HD __host__ __device__ __forceinline__
#else
#define SPK_HD inline
#endif

namespace asv {
namespace spk {

// Factor storage: LAPACK band layout with fill rows, ldf = 2kl+ku+1,
// A(i,j) at F[kv + i - j + j*ldf], kv = kl + ku.  Without pivoting the fill
// rows stay zero; entries coupling two blocks are never written, so F keeps
// the original couplings beside the blocks' factors.
struct Ctx {
  double* F;
  int64_t ldf;
  int64_t n;
  int kl, ku;
  int64_t m;  // block length; the last block also takes the remainder
  int64_t P;  // number of blocks (>= 2)
};

SPK_HD int64_t imin(int64_t a, int64_t b) { return a < b ? a : b; }
SPK_HD int64_t imax(int64_t a, int64_t b) { return a > b ? a : b; }
SPK_HD double dabs(double v) { return v < 0.0 ? -v : v; }

// Tests on a double's bits, for the inner loops: on this GPU an FP64
// comparison issues on the (narrow) FP64 pipe, an integer test does not.
SPK_HD uint64_t dbits(double v) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(v);
#else
  uint64_t b;
  memcpy(&b, &v, sizeof(b));
  return b;
#endif
}
SPK_HD bool nonzero(double v) { return (dbits(v) << 1) != 0; }                            // v != 0 (NaN: true)
SPK_HD bool zero_or_nan(double v) { return (dbits(v) << 1) == 0 || (dbits(v) << 1) > (0x7ff0000000000000ull << 1); }

SPK_HD double& fa(const Ctx& c, int64_t i, int64_t j) {
  return c.F[(size_t)(c.kl + c.ku + i - j) + (size_t)j * (size_t)c.ldf];
}
SPK_HD int64_t blk_s(const Ctx& c, int64_t b) { return b * c.m; }
SPK_HD int64_t blk_e(const Ctx& c, int64_t b) { return b == c.P - 1 ? c.n : (b + 1) * c.m; }

// Bandwidths of the system solved: A, or A^T (kl and ku exchanged).
SPK_HD int sys_kl(const Ctx& c, bool tr) { return tr ? c.ku : c.kl; }
SPK_HD int sys_ku(const Ctx& c, bool tr) { return tr ? c.kl : c.ku; }
// Entry (i, j) of the system matrix outside the diagonal blocks.
SPK_HD double sys_at(const Ctx& c, bool tr, int64_t i, int64_t j) { return tr ? fa(c, j, i) : fa(c, i, j); }

// LU without pivoting of block b in place.  Returns 0, or 1 + the block-local
// column of the first pivot that is zero or not a number.
SPK_HD int factor_block(const Ctx& c, int64_t b) {
  const int64_t s = blk_s(c, b), e = blk_e(c, b);
  for (int64_t j = s; j < e; ++j) {
    const double p = fa(c, j, j);
    if (!(p != 0.0) || p != p) return (int)(j - s) + 1;
    const int64_t lo = imin(e - 1, j + c.kl), hi = imin(e - 1, j + c.ku);
    for (int64_t i = j + 1; i <= lo; ++i) fa(c, i, j) = fa(c, i, j) / p;
    for (int64_t q = j + 1; q <= hi; ++q) {
      const double u = fa(c, j, q);
      if (u == 0.0) continue;
      for (int64_t i = j + 1; i <= lo; ++i) fa(c, i, q) -= fa(c, i, j) * u;
    }
  }
  return 0;
}

// xl[0 .. e-s) := A_bb^-1 xl  (tr: A_bb^-T), with the block's factors;
// xl[k] is row s + k of the block.
SPK_HD void solve_block(const Ctx& c, int64_t b, bool tr, double* xl) {
  const int64_t s = blk_s(c, b), e = blk_e(c, b);
  if (!tr) {
    for (int64_t j = s; j < e; ++j) {  // L y = x, unit diagonal
      const double xj = xl[j - s];
      if (xj == 0.0) continue;
      const int64_t lo = imin(e - 1, j + c.kl);
      for (int64_t i = j + 1; i <= lo; ++i) xl[i - s] -= fa(c, i, j) * xj;
    }
    for (int64_t j = e - 1; j >= s; --j) {  // U x = y
      xl[j - s] = xl[j - s] / fa(c, j, j);
      const double xj = xl[j - s];
      if (xj == 0.0) continue;
      for (int64_t i = imax(s, j - c.ku); i < j; ++i) xl[i - s] -= fa(c, i, j) * xj;
    }
  } else {
    for (int64_t j = s; j < e; ++j) {  // U^T z = x
      double t = xl[j - s];
      for (int64_t i = imax(s, j - c.ku); i < j; ++i) t -= fa(c, i, j) * xl[i - s];
      xl[j - s] = t / fa(c, j, j);
    }
    for (int64_t j = e - 1; j >= s; --j) {  // L^T y = z, unit diagonal
      double t = xl[j - s];
      const int64_t lo = imin(e - 1, j + c.kl);
      for (int64_t i = j + 1; i <= lo; ++i) t -= fa(c, i, j) * xl[i - s];
      xl[j - s] = t;
    }
  }
}

// The largest far-tip entry: a maximum over the bit patterns of
// non-negative doubles (their integer order is their numeric order).
SPK_HD void max_bits(unsigned long long* slot, double v) {
#ifdef __CUDA_ARCH__
  atomicMax(slot, (unsigned long long)__double_as_longlong(v));
#else
  unsigned long long bits;
  memcpy(&bits, &v, sizeof(bits));
  if (bits > *slot) *slot = bits;
#endif
}

// Order of every boundary system.
SPK_HD int64_t q_of(const Ctx& c) { return (int64_t)c.kl + c.ku; }

// One spike column per thread: t in [0, P*q).  Block b = t / q, column
// r = t % q: r < ku' is column r of V_b (right spike, exists for b < P-1),
// else column r - ku' of W_b (left spike, exists for b > 0), where kl', ku'
// are the bandwidths of the system solved.  The column is solved in the
// scratch area at offset s_b*q + r*m_b (m_b doubles); its near tip goes to
// boundary system M (q x q, column-major, one per boundary, zeroed before),
// the largest |entry| of its far tip to *far.
SPK_HD void spike_column(const Ctx& c, bool tr, int64_t t, double* scr, double* M, unsigned long long* far) {
  const int64_t q = q_of(c);
  const int64_t b = t / q;
  const int r = (int)(t % q);
  const int kl = sys_kl(c, tr), ku = sys_ku(c, tr);
  const int64_t s = blk_s(c, b), e = blk_e(c, b), mb = e - s;
  double* v = scr + (size_t)s * (size_t)q + (size_t)r * (size_t)mb;  // v[i - s], i in [s, e)
  double fm = 0.0;
  if (r < ku) {  // V_b column r: column J = e + r, in block b+1
    if (b + 1 >= c.P) return;
    const int64_t J = e + r;
    for (int64_t i = s; i < e; ++i) v[i - s] = 0.0;
    for (int64_t i = imax(s, J - ku); i < e; ++i) v[i - s] = sys_at(c, tr, i, J);
    solve_block(c, b, tr, v);
    double* Mb = M + (size_t)b * (size_t)(q * q);  // boundary b: [x_b^B (kl'); x_{b+1}^T (ku')]
    for (int i = 0; i < kl; ++i) Mb[i + (size_t)(kl + r) * q] = v[mb - kl + i];
    for (int i = 0; i < ku; ++i) fm = fm < dabs(v[i]) ? dabs(v[i]) : fm;
  } else {  // W_b column r - ku': column J = s - kl' + (r - ku'), in block b-1
    if (b == 0) return;
    const int cc = r - ku;
    const int64_t J = s - kl + cc;
    for (int64_t i = s; i < e; ++i) v[i - s] = 0.0;
    for (int64_t i = s; i < imin(e, J + kl + 1); ++i) v[i - s] = sys_at(c, tr, i, J);
    solve_block(c, b, tr, v);
    double* Mb = M + (size_t)(b - 1) * (size_t)(q * q);  // boundary b-1
    for (int i = 0; i < ku; ++i) Mb[(kl + i) + (size_t)cc * q] = v[i];
    for (int i = 0; i < kl; ++i) fm = fm < dabs(v[mb - kl + i]) ? dabs(v[mb - kl + i]) : fm;
  }
  max_bits(far, fm);
}

// Boundary system b (b < P-1): M += I, then LU with partial pivoting in
// place (first largest |a|).  Returns 0 or 1 + the singular column.
SPK_HD int factor_boundary(const Ctx& c, int64_t b, double* M, int* ipiv) {
  const int64_t q = q_of(c);
  double* A = M + (size_t)b * (size_t)(q * q);
  int* pv = ipiv + (size_t)b * (size_t)q;
  for (int64_t i = 0; i < q; ++i) A[i + i * q] += 1.0;
  for (int64_t j = 0; j < q; ++j) {
    int64_t p = j;
    double best = dabs(A[j + j * q]);
    for (int64_t i = j + 1; i < q; ++i)
      if (dabs(A[i + j * q]) > best) { best = dabs(A[i + j * q]); p = i; }
    pv[j] = (int)p;
    if (!(best > 0.0)) return (int)j + 1;
    if (p != j)
      for (int64_t k = 0; k < q; ++k) {
        const double tmp = A[j + k * q];
        A[j + k * q] = A[p + k * q];
        A[p + k * q] = tmp;
      }
    const double d = A[j + j * q];
    for (int64_t i = j + 1; i < q; ++i) A[i + j * q] = A[i + j * q] / d;
    for (int64_t k = j + 1; k < q; ++k) {
      const double u = A[j + k * q];
      if (u == 0.0) continue;
      for (int64_t i = j + 1; i < q; ++i) A[i + k * q] -= A[i + j * q] * u;
    }
  }
  return 0;
}

// Solve step 1 (one thread per block): G[s..e) = A_bb^-1 x[s..e) (tr: A_bb^-T).
SPK_HD void solve_step1(const Ctx& c, bool tr, int64_t b, const double* x, double* G) {
  const int64_t s = blk_s(c, b), e = blk_e(c, b);
  for (int64_t i = s; i < e; ++i) G[i] = x[i];
  solve_block(c, b, tr, G + s);
}

// Solve step 2 (one thread per boundary b < P-1): the boundary unknowns
// [x_b^B; x_{b+1}^T] into Y[b*q ..].
SPK_HD void solve_step2(const Ctx& c, bool tr, int64_t b, const double* G, const double* M, const int* ipiv,
                        double* Y) {
  const int64_t q = q_of(c);
  const int kl = sys_kl(c, tr), ku = sys_ku(c, tr);
  const double* A = M + (size_t)b * (size_t)(q * q);
  const int* pv = ipiv + (size_t)b * (size_t)q;
  double* u = Y + (size_t)b * (size_t)q;
  const int64_t e = blk_e(c, b), s1 = blk_s(c, b + 1);
  for (int i = 0; i < kl; ++i) u[i] = G[e - kl + i];
  for (int i = 0; i < ku; ++i) u[kl + i] = G[s1 + i];
  for (int64_t j = 0; j < q; ++j) {  // P, then unit L
    const int64_t p = pv[j];
    if (p != j) {
      const double tmp = u[j];
      u[j] = u[p];
      u[p] = tmp;
    }
    const double uj = u[j];
    for (int64_t i = j + 1; i < q; ++i) u[i] -= A[i + j * q] * uj;
  }
  for (int64_t j = q - 1; j >= 0; --j) {  // U
    u[j] = u[j] / A[j + j * q];
    const double uj = u[j];
    for (int64_t i = 0; i < j; ++i) u[i] -= A[i + j * q] * uj;
  }
}

// Solve step 3 (one thread per block): x_b = A_bb^-1 (f_b - couplings with
// the neighbours' boundary unknowns), in place on x (which holds f).
SPK_HD void solve_step3(const Ctx& c, bool tr, int64_t b, const double* Y, double* x) {
  const int64_t q = q_of(c);
  const int kl = sys_kl(c, tr), ku = sys_ku(c, tr);
  const int64_t s = blk_s(c, b), e = blk_e(c, b);
  if (b + 1 < c.P) {  // columns e .. e+ku-1 hold x_{b+1}^T = Y[b*q + kl ..]
    const double* y = Y + (size_t)b * (size_t)q + kl;
    for (int r = 0; r < ku; ++r) {
      const int64_t J = e + r;
      const double xj = y[r];
      for (int64_t i = imax(s, J - ku); i < e; ++i) x[i] -= sys_at(c, tr, i, J) * xj;
    }
  }
  if (b > 0) {  // columns s-kl .. s-1 hold x_{b-1}^B = Y[(b-1)*q ..]
    const double* y = Y + (size_t)(b - 1) * (size_t)q;
    for (int r = 0; r < kl; ++r) {
      const int64_t J = s - kl + r;
      const double xj = y[r];
      for (int64_t i = s; i < imin(e, J + kl + 1); ++i) x[i] -= sys_at(c, tr, i, J) * xj;
    }
  }
  solve_block(c, b, tr, x + s);
}

// ---------------------------------------------------------------- warps
// Warp-cooperative versions of the block factorisation and the block
// solves, for wide bands.  Each is a sequence of phases over lanes
// 0..31: within a phase every lane writes entries no other lane touches and
// reads only entries that no lane writes in that phase; the kernels put a
// __syncwarp() between phases, and running the lanes of a phase one after
// another gives the same result.  `red` is 32 doubles of per-warp scratch.

// Factorisation, column j: (1) multipliers, rows j+1+lane, j+33+lane, ...
SPK_HD void wlu_mult(const Ctx& c, int64_t e, int64_t j, int lane) {
  const double p = fa(c, j, j);
  const int64_t lo = imin(e - 1, j + c.kl);
  for (int64_t i = j + 1 + lane; i <= lo; i += 32) fa(c, i, j) = fa(c, i, j) / p;
}
// (2) rank-1 update of the same rows, columns j+1 .. j+ku
SPK_HD void wlu_update(const Ctx& c, int64_t e, int64_t j, int lane) {
  const int64_t lo = imin(e - 1, j + c.kl), hi = imin(e - 1, j + c.ku);
  for (int64_t i = j + 1 + lane; i <= lo; i += 32) {
    const double l = fa(c, i, j);
    if (l == 0.0) continue;
    for (int64_t q = j + 1; q <= hi; ++q) fa(c, i, q) -= l * fa(c, j, q);
  }
}

// Solve with A_bb, column j of L (forward): one phase.
SPK_HD void wsolve_l(const Ctx& c, int64_t s, int64_t e, int64_t j, int lane, double* xl) {
  const double xj = xl[j - s];
  const int64_t lo = imin(e - 1, j + c.kl);
  for (int64_t i = j + 1 + lane; i <= lo; i += 32) xl[i - s] -= fa(c, i, j) * xj;
}
// Column j of U (backward): (1) lane 0 divides, (2) the rows above update.
SPK_HD void wsolve_u_div(const Ctx& c, int64_t s, int64_t j, int lane, double* xl) {
  if (lane == 0) xl[j - s] = xl[j - s] / fa(c, j, j);
}
SPK_HD void wsolve_u_upd(const Ctx& c, int64_t s, int64_t j, int lane, double* xl) {
  const double xj = xl[j - s];
  for (int64_t i = imax(s, j - c.ku) + lane; i < j; i += 32) xl[i - s] -= fa(c, i, j) * xj;
}
// Solve with A_bb^T, row j of U^T (forward): (1) partial dot products,
// (2) lane 0 sums them in lane order and divides.
SPK_HD void wsolve_ut_dot(const Ctx& c, int64_t s, int64_t j, int lane, const double* xl, double* red) {
  double t = 0.0;
  for (int64_t i = imax(s, j - c.ku) + lane; i < j; i += 32) t += fa(c, i, j) * xl[i - s];
  red[lane] = t;
}
SPK_HD void wsolve_ut_fin(const Ctx& c, int64_t s, int64_t j, int lane, double* xl, const double* red) {
  if (lane != 0) return;
  double t = 0.0;
  for (int k = 0; k < 32; ++k) t += red[k];
  xl[j - s] = (xl[j - s] - t) / fa(c, j, j);
}
// Row j of L^T (backward): (1) partial dot products, (2) lane 0 subtracts.
SPK_HD void wsolve_lt_dot(const Ctx& c, int64_t s, int64_t e, int64_t j, int lane, const double* xl, double* red) {
  double t = 0.0;
  const int64_t lo = imin(e - 1, j + c.kl);
  for (int64_t i = j + 1 + lane; i <= lo; i += 32) t += fa(c, i, j) * xl[i - s];
  red[lane] = t;
}
SPK_HD void wsolve_lt_fin(int64_t s, int64_t j, int lane, double* xl, const double* red) {
  if (lane != 0) return;
  double t = 0.0;
  for (int k = 0; k < 32; ++k) t += red[k];
  xl[j - s] = xl[j - s] - t;
}

// Block drivers over a phase runner: run(f) calls f(lane) for this thread's
// lane and then __syncwarp() (device), or f(0) .. f(31) in turn (host).
#ifdef __CUDACC__
#pragma nv_exec_check_disable
#endif
template <class Run>
SPK_HD int wfactor_block(const Ctx& c, int64_t b, Run&& run) {
  const int64_t s = blk_s(c, b), e = blk_e(c, b);
  for (int64_t j = s; j < e; ++j) {
    const double p = fa(c, j, j);  // every lane reads the same value: a uniform branch
    if (!(p != 0.0) || p != p) return (int)(j - s) + 1;
    run([&](int lane) { wlu_mult(c, e, j, lane); });
    run([&](int lane) { wlu_update(c, e, j, lane); });
  }
  return 0;
}

#ifdef __CUDACC__
#pragma nv_exec_check_disable
#endif
template <class Run>
SPK_HD void wsolve_block(const Ctx& c, int64_t b, bool tr, double* xl, double* red, Run&& run) {
  const int64_t s = blk_s(c, b), e = blk_e(c, b);
  if (!tr) {
    for (int64_t j = s; j < e; ++j)
      if (xl[j - s] != 0.0) run([&](int lane) { wsolve_l(c, s, e, j, lane, xl); });
    for (int64_t j = e - 1; j >= s; --j) {
      run([&](int lane) { wsolve_u_div(c, s, j, lane, xl); });
      run([&](int lane) { wsolve_u_upd(c, s, j, lane, xl); });
    }
  } else {
    for (int64_t j = s; j < e; ++j) {
      run([&](int lane) { wsolve_ut_dot(c, s, j, lane, xl, red); });
      run([&](int lane) { wsolve_ut_fin(c, s, j, lane, xl, red); });
    }
    for (int64_t j = e - 1; j >= s; --j) {
      run([&](int lane) { wsolve_lt_dot(c, s, e, j, lane, xl, red); });
      run([&](int lane) { wsolve_lt_fin(s, j, lane, xl, red); });
    }
  }
}

// Step 3's couplings with the neighbours' boundary unknowns, rows split
// over the lanes (only rows within kl' of the block's start or ku' of its
// end are reached).
SPK_HD void step3_couplings(const Ctx& c, bool tr, int64_t b, const double* Y, double* x, int lane) {
  const int64_t q = q_of(c);
  const int kl = sys_kl(c, tr), ku = sys_ku(c, tr);
  const int64_t s = blk_s(c, b), e = blk_e(c, b);
  for (int64_t i = s + lane; i < e; i += 32) {
    if (i < e - ku && i >= s + kl) {  // skip to the rows the couplings reach
      const int64_t nxt = e - ku > s + kl ? e - ku : s + kl;
      i += ((nxt - i + 31) / 32 - 1) * 32;
      continue;
    }
    double t = x[i];
    if (b + 1 < c.P)
      for (int r = 0; r < ku; ++r) {
        const int64_t J = e + r;
        if (i >= J - ku) t -= sys_at(c, tr, i, J) * Y[(size_t)b * (size_t)q + kl + r];
      }
    if (b > 0)
      for (int r = 0; r < kl; ++r) {
        const int64_t J = s - kl + r;
        if (i <= J + kl) t -= sys_at(c, tr, i, J) * Y[(size_t)(b - 1) * (size_t)q + r];
      }
    x[i] = t;
  }
}

// Solve steps 1 and 3 with one warp per block (steps 2 is per boundary).
#ifdef __CUDACC__
#pragma nv_exec_check_disable
#endif
template <class Run>
SPK_HD void wsolve_step1(const Ctx& c, bool tr, int64_t b, const double* x, double* G, double* red, Run&& run) {
  const int64_t s = blk_s(c, b), e = blk_e(c, b);
  run([&](int lane) {
    for (int64_t i = s + lane; i < e; i += 32) G[i] = x[i];
  });
  wsolve_block(c, b, tr, G + s, red, run);
}

#ifdef __CUDACC__
#pragma nv_exec_check_disable
#endif
template <class Run>
SPK_HD void wsolve_step3(const Ctx& c, bool tr, int64_t b, const double* Y, double* x, double* red, Run&& run) {
  run([&](int lane) { step3_couplings(c, tr, b, Y, x, lane); });
  wsolve_block(c, b, tr, x + blk_s(c, b), red, run);
}

// ------------------------------------------------------- sliding windows
// Spike columns for bandwidths kl', ku' <= 32, in dot-product form over a
// circular window of the last kWin unknowns computed (a per-thread array:
// local memory on the GPU, where one index across the 32 lanes is one
// contiguous line, so every access is coalesced and stays in L1).  Only
// what the route needs is kept: V's near tip (bottom kl' rows) goes to M and
// its far tip (top ku' rows) into *far, and V's forward values live in the
// window alone (the right-hand side starts at most ku' rows above the
// block's end).  W's forward values are stored once, lane-interleaved in the
// scratch area (row i of column r at (i - s) q + r), for its backward pass.
constexpr int kWin = 64;
constexpr int kWinMaxBand = 32;

// Entry (i, j), i != j, of the system's block factors: for A the unit-lower
// L and the upper U (fa(i, j)); for A^T = U^T L^T the lower U^T and the
// unit-upper L^T (fa(j, i)).
SPK_HD double blkf(const Ctx& c, bool tr, int64_t i, int64_t j) { return tr ? fa(c, j, i) : fa(c, i, j); }

// Forward row i of the lower factor: (rhs - sum over j in [max(lo0, i-bl), i)
// of L'(i, j) w_j) / d_i, d_i = 1 for A (unit L), U_ii for A^T; the
// division is a product with rd_i = 1 / U_ii.
SPK_HD double fwd_row(const Ctx& c, bool tr, int64_t i, int64_t lo0, int bl, double rhs, const double* w,
                      const double* rd) {
  double t = rhs;
  const int64_t j0 = imax(lo0, i - bl);
  const int cnt = (int)(i - j0);
  // L'(i, j0 + k): for A fa(i, j) (stride ldf - 1 in j), for A^T fa(j, i) (stride 1)
  const double* f = tr ? &fa(c, j0, i) : &fa(c, i, j0);
  const int st = tr ? 1 : (int)c.ldf - 1;
  int wi = (int)(j0 & (kWin - 1));
  for (int k = 0, o = 0; k < cnt; ++k, o += st, wi = (wi + 1) & (kWin - 1)) t -= f[o] * w[wi];
  return tr ? t * rd[i] : t;
}
// Backward row i of the upper factor: (y - sum over j in (i, min(hi0, i+bu)]
// of U'(i, j) w_j) / d_i, d_i = U_ii for A, 1 for A^T (unit L^T).
SPK_HD double bwd_row(const Ctx& c, bool tr, int64_t i, int64_t hi0, int bu, double y, const double* w,
                      const double* rd) {
  double t = y;
  const int cnt = (int)(imin(hi0, i + bu) - i);
  // U'(i, i + 1 + k): for A fa(i, j) (stride ldf - 1 in j), for A^T fa(j, i) (stride 1)
  const double* f = tr ? &fa(c, i + 1, i) : &fa(c, i, i + 1);
  const int st = tr ? 1 : (int)c.ldf - 1;
  int wi = (int)((i + 1) & (kWin - 1));
  for (int k = 0, o = 0; k < cnt; ++k, o += st, wi = (wi + 1) & (kWin - 1)) t -= f[o] * w[wi];
  return tr ? t : t * rd[i];
}

// One spike column per thread, t in [0, P q), as spike_column, with the
// window solves above; rd: the reciprocals of the blocks' U diagonals.
SPK_HD void spike_column_win(const Ctx& c, bool tr, int64_t t, double* scr, double* M, unsigned long long* far,
                             const double* rd) {
  const int64_t q = q_of(c);
  const int64_t b = t / q;
  const int r = (int)(t % q);
  const int kl = sys_kl(c, tr), ku = sys_ku(c, tr);
  const int64_t s = blk_s(c, b), e = blk_e(c, b);
  double w[kWin];
  double fm = 0.0;
  if (r < ku) {  // V_b column r: column J = e + r (block b+1); right-hand side rows [i0, e)
    if (b + 1 >= c.P) return;
    const int64_t J = e + r, i0 = imax(s, J - ku);
    for (int64_t i = i0; i < e; ++i) w[i & (kWin - 1)] = fwd_row(c, tr, i, i0, kl, sys_at(c, tr, i, J), w, rd);
    double* Mb = M + (size_t)b * (size_t)(q * q);  // boundary b: [x_b^B (kl'); x_{b+1}^T (ku')]
    for (int64_t i = e - 1; i >= s; --i) {
      const double v = bwd_row(c, tr, i, e - 1, ku, i >= i0 ? w[i & (kWin - 1)] : 0.0, w, rd);
      w[i & (kWin - 1)] = v;
      if (i >= e - kl) Mb[(i - (e - kl)) + (size_t)(kl + r) * q] = v;
      if (i < s + ku) fm = fm < dabs(v) ? dabs(v) : fm;
    }
  } else {  // W_b column r - ku': column J = s - kl' + (r - ku') (block b-1); right-hand side rows [s, i1)
    if (b == 0) return;
    const int cc = r - ku;
    const int64_t J = s - kl + cc, i1 = imin(e, J + kl + 1);
    double* ys = scr + (size_t)s * (size_t)q + (size_t)r;
    for (int64_t i = s; i < e; ++i) {
      const double v = fwd_row(c, tr, i, s, kl, i < i1 ? sys_at(c, tr, i, J) : 0.0, w, rd);
      w[i & (kWin - 1)] = v;
      ys[(size_t)(i - s) * (size_t)q] = v;
    }
    double* Mb = M + (size_t)(b - 1) * (size_t)(q * q);  // boundary b-1
    for (int64_t i = e - 1; i >= s; --i) {
      const double v = bwd_row(c, tr, i, e - 1, ku, ys[(size_t)(i - s) * (size_t)q], w, rd);
      w[i & (kWin - 1)] = v;
      if (i >= e - kl) fm = fm < dabs(v) ? dabs(v) : fm;
      if (i < s + ku) Mb[(kl + (i - s)) + (size_t)cc * q] = v;
    }
  }
  max_bits(far, fm);
}

// Block factorisation by one warp, one phase per column j: lane l takes row
// i = j + 1 + l (kl <= 32), forms its multiplier with the pivot's
// reciprocal rd[j] and updates its row from the pivot row j, which no lane
// writes in that phase; the lane that finishes row j + 1 (lane 0) then
// forms rd[j + 1].  The loads of a row are issued together before any of
// its stores.
SPK_HD void wlu_step(const Ctx& c, int64_t e, int64_t j, int lane, double* rd) {
  const int64_t i = j + 1 + lane;
  if (i <= imin(e - 1, j + c.kl)) {
    const double l = fa(c, i, j) * rd[j];
    fa(c, i, j) = l;
    if (nonzero(l)) {
      const int cnt = (int)(imin(e - 1, j + c.ku) - j);  // columns j+1 .. j+cnt
      // rows j and i from column j + 1 on: stride ldf - 1 per column
      const double* pu = &fa(c, j, j + 1);
      double* pa = &fa(c, i, j + 1);
      const int st = (int)c.ldf - 1;
      double u[kWinMaxBand], a[kWinMaxBand];
      for (int k = 0; k < kWinMaxBand; ++k)
        if (k < cnt) {
          u[k] = pu[k * st];
          a[k] = pa[k * st];
        }
      for (int k = 0; k < kWinMaxBand; ++k)
        if (k < cnt && nonzero(u[k])) pa[k * st] = a[k] - l * u[k];
    }
  }
  if (lane == 0 && i < e) rd[i] = 1.0 / fa(c, i, i);  // row j + 1 is final
}

#ifdef __CUDACC__
#pragma nv_exec_check_disable
#endif
template <class Run>
SPK_HD int wfactor_block_step(const Ctx& c, int64_t b, double* rd, Run&& run) {
  const int64_t s = blk_s(c, b), e = blk_e(c, b);
  run([&](int lane) {
    if (lane == 0) rd[s] = 1.0 / fa(c, s, s);
  });
  for (int64_t j = s; j < e; ++j) {
    // final after the previous phase; uniform across the lanes
    if (zero_or_nan(fa(c, j, j))) return (int)(j - s) + 1;
    run([&](int lane) { wlu_step(c, e, j, lane, rd); });
  }
  return 0;
}

// Boundary system b by one warp (lanes over rows, then over columns for the
// interchange): M += I, then LU with partial pivoting, the first largest
// |a| as in factor_boundary.  rv, ri: 33 entries of per-warp scratch.
#ifdef __CUDACC__
#pragma nv_exec_check_disable
#endif
template <class Run>
SPK_HD int wfactor_boundary(const Ctx& c, int64_t b, double* M, int* ipiv, double* rv, int* ri, Run&& run) {
  const int64_t q = q_of(c);
  double* A = M + (size_t)b * (size_t)(q * q);
  int* pv = ipiv + (size_t)b * (size_t)q;
  run([&](int lane) {
    for (int64_t i = lane; i < q; i += 32) A[i + i * q] += 1.0;
  });
  for (int64_t j = 0; j < q; ++j) {
    run([&](int lane) {  // the first largest |a| among this lane's rows
      double best = -1.0;
      int at = -1;
      for (int64_t i = j + lane; i < q; i += 32)
        if (dabs(A[i + j * q]) > best) {
          best = dabs(A[i + j * q]);
          at = (int)i;
        }
      rv[lane] = best;
      ri[lane] = at;
    });
    run([&](int lane) {  // lane 0: the largest over the lanes, ties to the first row
      if (lane != 0) return;
      double best = -1.0;
      int at = -1;
      for (int k = 0; k < 32; ++k)
        if (ri[k] >= 0 && (rv[k] > best || (rv[k] == best && ri[k] < at))) {
          best = rv[k];
          at = ri[k];
        }
      rv[32] = best;
      ri[32] = at;
      pv[j] = at;
    });
    const double best = rv[32];
    const int64_t p = ri[32];
    if (!(best > 0.0)) return (int)j + 1;
    if (p != j)
      run([&](int lane) {
        for (int64_t k = lane; k < q; k += 32) {
          const double tmp = A[j + k * q];
          A[j + k * q] = A[p + k * q];
          A[p + k * q] = tmp;
        }
      });
    run([&](int lane) {  // rows below the pivot: multiplier and row update
      const double d = A[j + j * q];
      for (int64_t i = j + 1 + lane; i < q; i += 32) {
        const double l = A[i + j * q] / d;
        A[i + j * q] = l;
        for (int64_t k = j + 1; k < q; ++k) {
          const double u = A[j + k * q];
          if (nonzero(u)) A[i + k * q] -= l * u;
        }
      }
    });
  }
  return 0;
}

// Solve step 2 by one warp per boundary (as solve_step2; u in Y).
#ifdef __CUDACC__
#pragma nv_exec_check_disable
#endif
template <class Run>
SPK_HD void wsolve_step2(const Ctx& c, bool tr, int64_t b, const double* G, const double* M, const int* ipiv,
                         double* Y, Run&& run) {
  const int64_t q = q_of(c);
  const int kl = sys_kl(c, tr), ku = sys_ku(c, tr);
  const double* A = M + (size_t)b * (size_t)(q * q);
  const int* pv = ipiv + (size_t)b * (size_t)q;
  double* u = Y + (size_t)b * (size_t)q;
  const int64_t e = blk_e(c, b), s1 = blk_s(c, b + 1);
  run([&](int lane) {
    for (int i = lane; i < kl; i += 32) u[i] = G[e - kl + i];
    for (int i = lane; i < ku; i += 32) u[kl + i] = G[s1 + i];
  });
  for (int64_t j = 0; j < q; ++j) {  // P, then unit L
    const int64_t p = pv[j];
    if (p != j)
      run([&](int lane) {
        if (lane != 0) return;
        const double tmp = u[j];
        u[j] = u[p];
        u[p] = tmp;
      });
    run([&](int lane) {
      const double uj = u[j];
      for (int64_t i = j + 1 + lane; i < q; i += 32) u[i] -= A[i + j * q] * uj;
    });
  }
  for (int64_t j = q - 1; j >= 0; --j) {  // U
    run([&](int lane) {
      if (lane == 0) u[j] = u[j] / A[j + j * q];
    });
    run([&](int lane) {
      const double uj = u[j];
      for (int64_t i = lane; i < j; i += 32) u[i] -= A[i + j * q] * uj;
    });
  }
}

// Diagonal dominance of the original matrix in F (before any factoring):
// row i (by rows) and column i (by columns); one thread per index.
SPK_HD void dominance(const Ctx& c, int64_t i, int* rowdom, int* coldom) {
  const double d = dabs(fa(c, i, i));
  double rs = 0.0, cs = 0.0;
  for (int64_t j = imax(0, i - c.kl); j <= imin(c.n - 1, i + c.ku); ++j)
    if (j != i) rs += dabs(fa(c, i, j));
  for (int64_t r = imax(0, i - c.ku); r <= imin(c.n - 1, i + c.kl); ++r)
    if (r != i) cs += dabs(fa(c, r, i));
  *rowdom = d >= rs && d > 0.0;
  *coldom = d >= cs && d > 0.0;
}

}  // namespace spk
}  // namespace asv
