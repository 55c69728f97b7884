// band_warp.cuh -- banded LU with partial pivoting in band storage (Sec. 2.1,
// xGBTRF semantics) and the solve with its factors (xGBTRS), performed by one
// warp directly on global (or L2-resident) memory.  Used by the batched band
// class and, as the general-bandwidth fallback, by the large banded route.
#pragma once
#include "asolve_internal.cuh"

namespace asv {
namespace {

// Band factor storage (xGBTRF layout): element (i,j) at F[(kv+i-j) + j*ldf],
// ldf = 2kl+ku+1, kv = kl+ku; rows 0..kl-1 are fill room for U.
struct WarpBand {
  double* F;
  int* piv;
  double* rd = nullptr;  // optional: 1 / U(j,j), written by warp_band_lu
  int n, kl, ku, kv, ldf;
  __device__ double& at(int i, int j) const { return F[(size_t)(kv + i - j) + (size_t)j * ldf]; }
};

// Warp-scope GBTRF-equivalent.  Returns 0 or j+1 at an exact zero pivot.
__device__ int warp_band_lu(WarpBand& b) {
  const int lane = threadIdx.x & 31;
  int ju = 0;
  for (int j = 0; j < b.n; ++j) {
    const int km = min(b.kl, b.n - 1 - j);
    // the first largest |a(j+t, j)|, t = 0..km, in passes of 32 candidates
    int jp = -1;
    unsigned long long kbest = 0ull;
    for (int t0 = 0; t0 <= km; t0 += 32) {
      const int t = t0 + lane;
      unsigned long long kp;
      const int l = warp_first_max_key(t <= km ? abs_key(b.at(j + t, j)) : 0ull, kp);
      if (l >= 0 && kp > kbest) { kbest = kp; jp = t0 + l; }
    }
    if (jp < 0 || jp > km) return j + 1;  // only NaN candidates
    if (lane == 0) b.piv[j] = j + jp;
    const double pv = b.at(j + jp, j);
    if (pv == 0.0 || pv != pv) return j + 1;
    ju = max(ju, min(j + b.ku + jp, b.n - 1));
    __syncwarp();
    if (jp != 0)
      for (int c = j + lane; c <= ju; c += 32) {
        double t0 = b.at(j, c);
        b.at(j, c) = b.at(j + jp, c);
        b.at(j + jp, c) = t0;
      }
    __syncwarp();
    const double inv = 1.0 / b.at(j, j);
    if (b.rd && lane == 0) b.rd[j] = inv;
    for (int t = 1 + lane; t <= km; t += 32) b.at(j + t, j) *= inv;
    __syncwarp();
    // rank-1 update of rows j+1..j+km, columns j+1..ju
    const int ncol = ju - j;
    if (km > 0)
      for (int e = lane; e < km * ncol; e += 32) {
      const int t = 1 + e % km, c = j + 1 + e / km;
      b.at(j + t, c) -= b.at(j + t, j) * b.at(j, c);
    }
    __syncwarp();
  }
  return 0;
}

// x <- inv(A) x (trans: inv(A)^T x) with the band factors, one vector.
__device__ void warp_band_apply(const WarpBand& b, double* x, bool trans) {
  const int lane = threadIdx.x & 31;
  const int n = b.n;
  if (!trans) {
    for (int j = 0; j < n; ++j) {
      const int km = min(b.kl, n - 1 - j);
      const int p = b.piv[j];
      __syncwarp();
      double xj;
      if (p != j) {
        double a = x[j], c = x[p];
        __syncwarp();
        if (lane == 0) { x[j] = c; x[p] = a; }
        xj = c;
      } else {
        xj = x[j];
      }
      __syncwarp();
      for (int t = 1 + lane; t <= km; t += 32) x[j + t] -= b.at(j + t, j) * xj;
    }
    __syncwarp();
    for (int i = n - 1; i >= 0; --i) {  // U x = y, column-oriented
      __syncwarp();
      const double xi = x[i] / b.at(i, i);
      __syncwarp();
      if (lane == 0) x[i] = xi;
      const int lo = max(0, i - b.kv);
      for (int r = lo + lane; r < i; r += 32) x[r] -= b.at(r, i) * xi;
    }
    __syncwarp();
  } else {
    for (int i = 0; i < n; ++i) {  // U^T z = b
      const int lo = max(0, i - b.kv);
      double sacc = 0.0;
      for (int r = lo + lane; r < i; r += 32) sacc += b.at(r, i) * x[r];
      sacc = warp_sum(sacc);
      __syncwarp();
      if (lane == 0) x[i] = (x[i] - sacc) / b.at(i, i);
      __syncwarp();
    }
    for (int j = n - 1; j >= 0; --j) {  // L_j^T then P_j, in reverse
      const int km = min(b.kl, n - 1 - j);
      double sacc = 0.0;
      for (int t = 1 + lane; t <= km; t += 32) sacc += b.at(j + t, j) * x[j + t];
      sacc = warp_sum(sacc);
      __syncwarp();
      if (lane == 0) {
        double v = x[j] - sacc;
        const int p = b.piv[j];
        x[j] = x[p];
        x[p] = v;
        if (p == j) x[j] = v;
      }
      __syncwarp();
    }
  }
  __syncwarp();
}


// ---------------------------------------------------- register-window sweeps
// The solve of Sec. 2.1 with the band factors as a chain of n dependent
// steps run by one warp: the window of the vector being eliminated sits in
// registers across the lanes (element e in register e >> 5 of lane e & 31),
// and the factor columns stream through a cp.async ring kD steps ahead.
constexpr int kD = 16;          // cp.async prefetch distance (column steps)
constexpr int kMaxR = 8;        // register-window width: kl+ku+1 <= 32 * kMaxR

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// ------------------------------------------------------------ sweeps
// The vector window: element e sits in register e >> 5 of lane e & 31.
template <int R>
struct Win {
  double w[R];
  // (selects on shuffled copies keep every w[r] in a register)
  __device__ __forceinline__ double get(int e) const {
    const int re = e >> 5, le = e & 31;
    double v = __shfl_sync(0xffffffffu, w[0], le);
#pragma unroll
    for (int r = 1; r < R; ++r) {
      const double t = __shfl_sync(0xffffffffu, w[r], le);
      v = (r == re) ? t : v;
    }
    return v;
  }
  __device__ __forceinline__ void set(int e, double v) {
    const int lane = threadIdx.x & 31;
    const bool mine = lane == (e & 31);
#pragma unroll
    for (int r = 0; r < R; ++r) w[r] = (mine && r == (e >> 5)) ? v : w[r];
  }
  // element e <- element e+1; the top element becomes 0
  __device__ __forceinline__ void shift_down() {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const double nxt = (r + 1 < R) ? __shfl_sync(0xffffffffu, w[(r + 1 < R) ? r + 1 : r], 0) : 0.0;
      w[r] = __shfl_down_sync(0xffffffffu, w[r], 1);
      if (lane == 31) w[r] = nxt;
    }
  }
  // element e <- element e-1; element 0 becomes v0
  __device__ __forceinline__ void shift_up(double v0) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int r = R - 1; r >= 0; --r) {
      const double prv = (r > 0) ? __shfl_sync(0xffffffffu, w[r > 0 ? r - 1 : 0], 31) : v0;
      w[r] = __shfl_up_sync(0xffffffffu, w[r], 1);
      if (lane == 0) w[r] = prv;
    }
  }
};

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// x <- inv(A) x with the band factors (Sec. 2.1 solve), one warp; NC
// vectors at once (x column-major, ld ldx): the columns share the chain of
// steps, each step's column work is independent, so NC columns cost far
// less than NC sweeps.  With RD, rd[i] = 1 / U(i,i) (from the
// factorisation) turns each step's FP64 division into a multiplication:
// GB300's FP64 pipe, shared by every warp of the SM, bounds the batched
// sweeps, and a division is several of its instructions.  ring: kD * (kv + 1
// + NC + RD) doubles + kD ints of shared memory.
template <int R, int NC = 1, bool RD = false>
__device__ void band_apply(const double* __restrict__ F, int ldf, int n, int kl, int ku, const int* __restrict__ piv,
                           double* x, double* ring, int* pring, int ldx = 0, const double* __restrict__ rd = nullptr) {
  const int lane = threadIdx.x & 31;
  const int kv = kl + ku, SL = kv + 1 + NC + (RD ? 1 : 0);
  Win<R> W[NC];
  // ---- forward: apply P_j then L_j, j = 0..n-1; element t = x[j+t], t <= kl
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int t = r * 32 + lane;
      W[c].w[r] = (t <= kl && t < n) ? x[(size_t)c * ldx + t] : 0.0;
    }
  __syncwarp();
  auto pre_f = [&](int cs) {
    if (cs < n) {
      double* sl = ring + (size_t)(cs % kD) * SL;
      const int kmc = min(kl, n - 1 - cs);
      for (int t = 1 + lane; t <= kmc; t += 32) cp_async8(sl + t - 1, F + (size_t)kv + t + (size_t)cs * ldf);
      if (lane < NC && cs + kl + 1 < n) cp_async8(sl + kl + lane, x + (size_t)lane * ldx + cs + kl + 1);
      if (lane == 0) cp_async4(pring + cs % kD, piv + cs);
    }
    cp_commit();
  };
  for (int cs = 0; cs < kD; ++cs) pre_f(cs);
  for (int j = 0; j < n; ++j) {
    cp_wait<kD - 1>();
    __syncwarp();
    const double* sl = ring + (size_t)(j % kD) * SL;
    const int km = min(kl, n - 1 - j);
    const int d = pring[j % kD] - j;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const double e0 = W[c].get(0);
      const double ed = W[c].get(d);
      if (d) {
        W[c].set(0, ed);
        W[c].set(d, e0);
      }
      const double xj = d ? ed : e0;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int t = r * 32 + lane;
        if (t >= 1 && t <= km) W[c].w[r] = fma(-sl[t - 1], xj, W[c].w[r]);
      }
      if (lane == 0) x[(size_t)c * ldx + j] = xj;
      const double inc = (j + kl + 1 < n) ? sl[kl + c] : 0.0;
      W[c].shift_down();
      W[c].set(kl, inc);
    }
    __syncwarp();
    pre_f(j + kD);
  }
  cp_wait_all();
  __syncwarp();
  __threadfence();
  // ---- backward: U x = y, i = n-1..0; element s = y[i-s], s <= kv
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int s = r * 32 + lane;
      W[c].w[r] = (s <= kv && n - 1 - s >= 0) ? x[(size_t)c * ldx + n - 1 - s] : 0.0;
    }
  __syncwarp();
  auto pre_b = [&](int q) {
    const int i = n - 1 - q;
    if (i >= 0) {
      double* sl = ring + (size_t)(q % kD) * SL;
      for (int t = lane; t <= kv; t += 32) cp_async8(sl + t, F + (size_t)t + (size_t)i * ldf);
      if (lane < NC && i - kv - 1 >= 0) cp_async8(sl + kv + 1 + lane, x + (size_t)lane * ldx + i - kv - 1);
      if (RD && lane == 31) cp_async8(sl + kv + 1 + NC, rd + i);
    }
    cp_commit();
  };
  for (int q = 0; q < kD; ++q) pre_b(q);
  for (int q = 0; q < n; ++q) {
    const int i = n - 1 - q;
    cp_wait<kD - 1>();
    __syncwarp();
    const double* sl = ring + (size_t)(q % kD) * SL;
    const int lim = min(kv, i);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const double xi = RD ? W[c].get(0) * sl[kv + 1 + NC] : W[c].get(0) / sl[kv];
      if (lane == 0) x[(size_t)c * ldx + i] = xi;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int s = r * 32 + lane;
        if (s >= 1 && s <= lim) W[c].w[r] = fma(-sl[kv - s], xi, W[c].w[r]);
      }
      const double inc = (i - kv - 1 >= 0) ? sl[kv + 1 + c] : 0.0;
      W[c].shift_down();
      W[c].set(kv, inc);
    }
    __syncwarp();
    pre_b(q + kD);
  }
  cp_wait_all();
  __syncwarp();
  __threadfence();
}

// x <- inv(A)^T x: U^T z = x forward, then L_j^T and P_j backward.
template <int R, bool RD = false>
__device__ void band_apply_t(const double* __restrict__ F, int ldf, int n, int kl, int ku,
                             const int* __restrict__ piv, double* x, double* ring, int* pring,
                             const double* __restrict__ rd = nullptr) {
  const int lane = threadIdx.x & 31;
  const int kv = kl + ku, SL = kv + 2 + (RD ? 1 : 0);
  Win<R> W;
  // ---- U^T z = b, i = 0..n-1: element 0 = b_i, element s = z_{i-s}
#pragma unroll
  for (int r = 0; r < R; ++r) W.w[r] = (r == 0 && lane == 0) ? x[0] : 0.0;
  __syncwarp();
  auto pre_u = [&](int c) {
    if (c < n) {
      double* sl = ring + (size_t)(c % kD) * SL;
      for (int t = lane; t <= kv; t += 32) cp_async8(sl + t, F + (size_t)t + (size_t)c * ldf);
      if (lane == 0 && c + 1 < n) cp_async8(sl + kv + 1, x + c + 1);
      if (RD && lane == 31) cp_async8(sl + kv + 2, rd + c);
    }
    cp_commit();
  };
  for (int c = 0; c < kD; ++c) pre_u(c);
  for (int i = 0; i < n; ++i) {
    cp_wait<kD - 1>();
    __syncwarp();
    const double* sl = ring + (size_t)(i % kD) * SL;
    const int lim = min(kv, i);
    double acc = 0.0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int s = r * 32 + lane;
      if (s >= 1 && s <= lim) acc = fma(sl[kv - s], W.w[r], acc);
    }
    acc = warp_sum_d(acc);
    const double zi = RD ? (W.get(0) - acc) * sl[kv + 2] : (W.get(0) - acc) / sl[kv];
    if (lane == 0) x[i] = zi;
    W.set(0, zi);
    const double inc = (i + 1 < n) ? sl[kv + 1] : 0.0;
    W.shift_up(inc);
    __syncwarp();
    pre_u(i + kD);
  }
  cp_wait_all();
  __syncwarp();
  __threadfence();
  // ---- L^T with interchanges, j = n-1..0: element t = x[j+t], t <= kl
#pragma unroll
  for (int r = 0; r < R; ++r) W.w[r] = (r == 0 && lane == 0) ? x[n - 1] : 0.0;
  __syncwarp();
  auto pre_l = [&](int q) {
    const int j = n - 1 - q;
    if (j >= 0) {
      double* sl = ring + (size_t)(q % kD) * SL;
      const int kmc = min(kl, n - 1 - j);
      for (int t = 1 + lane; t <= kmc; t += 32) cp_async8(sl + t - 1, F + (size_t)kv + t + (size_t)j * ldf);
      if (lane == 0) {
        if (j - 1 >= 0) cp_async8(sl + kl, x + j - 1);
        cp_async4(pring + q % kD, piv + j);
      }
    }
    cp_commit();
  };
  for (int q = 0; q < kD; ++q) pre_l(q);
  for (int q = 0; q < n; ++q) {
    const int j = n - 1 - q;
    cp_wait<kD - 1>();
    __syncwarp();
    const double* sl = ring + (size_t)(q % kD) * SL;
    const int km = min(kl, n - 1 - j);
    double acc = 0.0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int t = r * 32 + lane;
      if (t >= 1 && t <= km) acc = fma(sl[t - 1], W.w[r], acc);
    }
    acc = warp_sum_d(acc);
    const double v = W.get(0) - acc;
    const int d = pring[q % kD] - j;
    if (d) {
      const double ed = W.get(d);
      W.set(0, ed);
      W.set(d, v);
    } else {
      W.set(0, v);
    }
    if (j == 0) break;
    // element kl (x[j+kl]) is final: no later step reads or swaps it
    const double ek = W.get(kl);
    if (lane == 0 && j + kl < n) x[j + kl] = ek;
    const double inc = sl[kl];
    W.shift_up(inc);
    __syncwarp();
    pre_l(q + kD);
  }
  cp_wait_all();
  __syncwarp();
  // flush the window: elements 0..kl are x[0..kl]
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int t = r * 32 + lane;
    if (t <= kl && t < n) x[t] = W.w[r];
  }
  __syncwarp();
  __threadfence();
}


// Ring storage of the sweeps for a window of R registers and up to NC
// vectors at once.
__host__ __device__ constexpr int band_ring_doubles(int R, int NC = 1) { return kD * (32 * R + 2 + NC); }

// x <- inv(A) x (trans: inv(A)^T x) for one vector, choosing the register
// window from the bandwidth; beyond 32 * rmax elements the global-memory
// routine is used.
__device__ __forceinline__ void band_sweep_any(const WarpBand& b, double* x, bool trans, double* ring, int* pring,
                                               int rmax) {
  // the factor and x were written with ordinary stores; the sweeps read
  // them through cp.async
  __syncwarp();
  __threadfence();
  const int need = (b.kv + 1 + 31) / 32;
  if (need <= 1 && rmax >= 1) {
    if (b.rd)
      trans ? band_apply_t<1, true>(b.F, b.ldf, b.n, b.kl, b.ku, b.piv, x, ring, pring, b.rd)
            : band_apply<1, 1, true>(b.F, b.ldf, b.n, b.kl, b.ku, b.piv, x, ring, pring, 0, b.rd);
    else
      trans ? band_apply_t<1>(b.F, b.ldf, b.n, b.kl, b.ku, b.piv, x, ring, pring)
            : band_apply<1>(b.F, b.ldf, b.n, b.kl, b.ku, b.piv, x, ring, pring);
  } else if (need <= 2 && rmax >= 2) {
    if (b.rd)
      trans ? band_apply_t<2, true>(b.F, b.ldf, b.n, b.kl, b.ku, b.piv, x, ring, pring, b.rd)
            : band_apply<2, 1, true>(b.F, b.ldf, b.n, b.kl, b.ku, b.piv, x, ring, pring, 0, b.rd);
    else
      trans ? band_apply_t<2>(b.F, b.ldf, b.n, b.kl, b.ku, b.piv, x, ring, pring)
            : band_apply<2>(b.F, b.ldf, b.n, b.kl, b.ku, b.piv, x, ring, pring);
  } else {
    warp_band_apply(b, x, trans);
  }
}
}  // namespace
}  // namespace asv
