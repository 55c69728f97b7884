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

// estimator helpers (one CTA of 1024 threads each)
template <typename V>
__global__ void k_vec_sumabs(const V* x, int n, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += fabs((double)x[i]);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    *out = t;
  }
}
template <typename V>
__global__ void k_vec_argmax(const V* x, int n, int* out, double* vals, int jprev) {
  __shared__ double rv[32];
  __shared__ int ri[32];
  double best = -1.0;
  int bi = 0x7fffffff;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double a = fabs((double)x[i]);
    if (a > best) { best = a; bi = i; }
  }
  warp_argmax_first(best, bi);
  if ((threadIdx.x & 31) == 0) { rv[threadIdx.x >> 5] = best; ri[threadIdx.x >> 5] = bi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = rv[0];
    int ii = ri[0];
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k)
      if (rv[k] > b || (rv[k] == b && ri[k] < ii)) { b = rv[k]; ii = ri[k]; }
    *out = ii;
    vals[0] = (ii >= 0 && ii < n) ? fabs((double)x[ii]) : 0.0;
    vals[1] = (jprev >= 0 && jprev < n) ? (double)x[jprev] : 0.0;
  }
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
    k_vec_sumabs<V><<<1, 1024, 0, st>>>(v, n, dscal);
    ECK(cudaMemcpyAsync(r, dscal, sizeof(double), cudaMemcpyDeviceToHost, st));
    ECK(cudaStreamSynchronize(st));
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
    k_vec_argmax<V><<<1, 1024, 0, st>>>(v, n, dint + 1, dscal + 1, jprev);
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
    k_vec_argmax<V><<<1, 1024, 0, st>>>(v, n, dint + 1, dscal + 1, j);
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
