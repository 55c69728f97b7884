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
  int n, kl, ku, kv, ldf;
  __device__ double& at(int i, int j) const { return F[(size_t)(kv + i - j) + (size_t)j * ldf]; }
};

// Warp-scope GBTRF-equivalent.  Returns 0 or j+1 at an exact zero pivot.
__device__ int warp_band_lu(WarpBand& b) {
  const int lane = threadIdx.x & 31;
  int ju = 0;
  for (int j = 0; j < b.n; ++j) {
    const int km = min(b.kl, b.n - 1 - j);
    double best = -1.0;
    int bi = 0x7fffffff;
    for (int t = lane; t <= km; t += 32) {
      double v = fabs(b.at(j + t, j));
      if (v > best) { best = v; bi = t; }
    }
    warp_argmax_first(best, bi);
    const int jp = bi;
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

}  // namespace
}  // namespace asv
