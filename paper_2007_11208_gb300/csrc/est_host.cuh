// est_host.cuh -- the 1-norm estimate of inv(A) (Hager 1984; Higham 1988,
// the xLACN2 iteration used by xGECON / xPOCON / xGBCON), driven from the
// host for one large system: the vector steps are small kernels, and
// apply(v, trans) -- a callback that overwrites the device vector v with
// inv(A) v or inv(A)^T v through the route's factors -- does the solves.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "asolve_internal.cuh"

namespace asv {
namespace {

#define ECK(x)                                      \
  do {                                              \
    cudaError_t _e = (x);                           \
    if (_e != cudaSuccess) return ASOLVE_E_CUDA;    \
  } while (0)

// Estimator reductions over a device vector, spread over kEstBlocks CTAs
// and deterministic: the sum of |x| from per-CTA partials (a fixed split of
// the index range, a fixed order inside each CTA) added in CTA order; the
// first index of max |x| from an atomic maximum of the magnitudes' bit
// patterns (order-free: the integer order of non-negative doubles is their
// numeric order) and then an atomic minimum over the indices that reach it.
// Scratch: dscal[0] the sum, dscal[1..2] the values of the argmax step,
// dscal[3] the maximum's bits, dscal[8 .. 8 + kEstBlocks) the partials;
// dint[1] the index.
constexpr int kEstBlocks = 24;
constexpr int kEstThreads = 1024;

template <typename V>
__global__ void __launch_bounds__(kEstThreads) k_vec_sumabs_part(const V* x, int n, double* part) {
  __shared__ double red[32];
  const int per = (n + kEstBlocks - 1) / kEstBlocks;
  const int lo = blockIdx.x * per, hi = min(n, lo + per);
  double s = 0.0;
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) s += fabs((double)x[i]);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    part[blockIdx.x] = t;
  }
}
__global__ void k_vec_sum_final(const double* part, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int b = 0; b < kEstBlocks; ++b) t += part[b];
    *out = t;
  }
}
template <typename V>
__global__ void __launch_bounds__(kEstThreads) k_vec_absmax_bits(const V* x, int n, unsigned long long* mbits) {
  unsigned long long m = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double a = fabs((double)x[i]);
    const unsigned long long b = (unsigned long long)__double_as_longlong(a);
    if (a == a && b > m) m = b;  // NaN entries never win
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
    m = t > m ? t : m;
  }
  if ((threadIdx.x & 31) == 0 && m) atomicMax(mbits, m);
}
template <typename V>
__global__ void __launch_bounds__(kEstThreads) k_vec_first_at(const V* x, int n, const unsigned long long* mbits,
                                                              int* idx) {
  const unsigned long long m = *mbits;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double a = fabs((double)x[i]);
    if ((unsigned long long)__double_as_longlong(a) == m) atomicMin(idx, i);
  }
}
template <typename V>
__global__ void k_vec_argmax_fin(const V* x, int n, int* out, double* vals, int jprev) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int ii = *out;
  vals[0] = (ii >= 0 && ii < n) ? fabs((double)x[ii]) : 0.0;
  vals[1] = (jprev >= 0 && jprev < n) ? (double)x[jprev] : 0.0;
}

// mode 0: x = 1/n; 1: x = e_j; 2: alternating test vector;
// 3: xi = sign(x), x = xi, flag[0] |= (sign changed)
template <typename V>
__global__ void k_vec_set(V* x, V* xi, int n, int mode, int j, int* flag) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (mode == 0) x[i] = V(1) / V(n);
    else if (mode == 1) x[i] = (i == j) ? V(1) : V(0);
    else if (mode == 2) x[i] = ((i & 1) ? V(-1) : V(1)) * (V(1) + V(i) / V(n - 1));
    else {
      const V sg = x[i] >= V(0) ? V(1) : V(-1);
      if (sg != xi[i]) atomicOr(flag, 1);
      xi[i] = sg;
      x[i] = sg;
    }
  }
}

// 1-norm estimate of inv(A) (Hager 1984, Higham 1988), the iteration driven
// from the host; apply(v, trans) overwrites the device vector v.
template <typename V, typename Apply>
int est_host(int n, V* v, V* xi, double* dscal, int* dint, Apply apply, cudaStream_t st, double* out) {
  auto sumabs = [&](double* r) -> int {
    k_vec_sumabs_part<V><<<kEstBlocks, kEstThreads, 0, st>>>(v, n, dscal + 8);
    k_vec_sum_final<<<1, 32, 0, st>>>(dscal + 8, dscal);
    ECK(cudaMemcpyAsync(r, dscal, sizeof(double), cudaMemcpyDeviceToHost, st));
    ECK(cudaStreamSynchronize(st));
    return ASOLVE_OK;
  };
  // first index of max |v| into dint[1]; |v[j]| and v[jprev] into dscal[1..2]
  auto argmax = [&](int jp) -> int {
    unsigned long long* mb = reinterpret_cast<unsigned long long*>(dscal + 3);
    ECK(cudaMemsetAsync(mb, 0, sizeof(unsigned long long), st));
    ECK(cudaMemsetAsync(dint + 1, 0x7f, sizeof(int), st));  // 0x7f7f7f7f: above any index
    k_vec_absmax_bits<V><<<kEstBlocks, kEstThreads, 0, st>>>(v, n, mb);
    k_vec_first_at<V><<<kEstBlocks, kEstThreads, 0, st>>>(v, n, mb, dint + 1);
    k_vec_argmax_fin<V><<<1, 32, 0, st>>>(v, n, dint + 1, dscal + 1, jp);
    return ASOLVE_OK;
  };
  const int g = (n + 255) / 256;
  k_vec_set<V><<<g, 256, 0, st>>>(v, xi, n, 0, 0, dint);
  int rc = apply(v, false);
  if (rc) return rc;
  double est;
  if (n == 1) {
    V h;
    ECK(cudaMemcpyAsync(&h, v, sizeof(V), cudaMemcpyDeviceToHost, st));
    ECK(cudaStreamSynchronize(st));
    *out = fabs((double)h);
    return ASOLVE_OK;
  }
  if ((rc = sumabs(&est))) return rc;
  k_vec_set<V><<<g, 256, 0, st>>>(v, xi, n, 3, 0, dint);
  if ((rc = apply(v, true))) return rc;
  int k = 2;
  int jprev = -1;
  for (;;) {
    int j;
    if ((rc = argmax(jprev))) return rc;
    ECK(cudaMemcpyAsync(&j, dint + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    ECK(cudaStreamSynchronize(st));
    if (j < 0 || j >= n) { est = NAN; break; }
    k_vec_set<V><<<g, 256, 0, st>>>(v, xi, n, 1, j, dint);
    if ((rc = apply(v, false))) return rc;
    const double estold = est;
    if ((rc = sumabs(&est))) return rc;
    ECK(cudaMemsetAsync(dint, 0, sizeof(int), st));
    k_vec_set<V><<<g, 256, 0, st>>>(v, xi, n, 3, 0, dint);
    int changed = 0;
    ECK(cudaMemcpyAsync(&changed, dint, sizeof(int), cudaMemcpyDeviceToHost, st));
    ECK(cudaStreamSynchronize(st));
    if (!changed || est <= estold) break;
    if ((rc = apply(v, true))) return rc;
    double vals[2];
    int jn;
    if ((rc = argmax(j))) return rc;
    ECK(cudaMemcpyAsync(&jn, dint + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    ECK(cudaMemcpyAsync(vals, dscal + 1, sizeof(vals), cudaMemcpyDeviceToHost, st));
    ECK(cudaStreamSynchronize(st));
    ++k;
    if (jn < 0 || jn >= n) { est = NAN; break; }
    jprev = j;
    if (vals[1] == vals[0] || k > 5) break;
  }
  k_vec_set<V><<<g, 256, 0, st>>>(v, xi, n, 2, 0, dint);
  if ((rc = apply(v, false))) return rc;
  double s2;
  if ((rc = sumabs(&s2))) return rc;
  const double temp = 2.0 * s2 / (double)(3 * n);
  if (temp > est) est = temp;
  *out = est;
  return ASOLVE_OK;
}

#undef ECK

}  // namespace
}  // namespace asv
