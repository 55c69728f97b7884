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
  const int64_t q = q_of(c);
  const int kl = sys_kl(c, tr), ku = sys_ku(c, tr);
  const int64_t s = blk_s(c, b), e = blk_e(c, b);
  // couplings with the neighbours' boundary unknowns: rows split over lanes
  run([&](int lane) {
    for (int64_t i = s + lane; i < e; i += 32) {
      if (i < e - ku && i >= s + kl) continue;  // rows no coupling reaches
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
  });
  wsolve_block(c, b, tr, x + s, red, run);
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
