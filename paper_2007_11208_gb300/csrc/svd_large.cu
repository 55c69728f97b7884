// svd_large.cu -- the SVD fallback of Sec. 2.5 for one large system
// (1024 < n <= kSvdLargeMax): when the routed solver fails or its rcond is
// below the threshold, X is the minimum-norm solution through the SVD of A
// (xGELSD semantics: singular values sigma_i <= tau dropped).
//
// One-sided Jacobi (Hestenes): G = A is rotated by pairs of columns until
// every pair is orthogonal to the tolerance n eps (relative to the two
// column norms); then sigma_j = ||G_j||, U_j = G_j / sigma_j, and V
// accumulates the rotations.  The minimum-norm solution is
//   x = sum_{sigma_j > tau} V_j (U_j . b) / sigma_j.
// The pairs are visited in the round-robin (tournament) order: in each of
// the n - 1 rounds of a sweep the n/2 pairs are disjoint, so one launch
// rotates all of them at once, a warp per pair, the columns streamed from
// global memory (coalesced).  A sweep ends with one flag read by the host;
// at most 30 sweeps.  Sums over a column run in lane order and then across
// the warp in a fixed tree, so results do not depend on scheduling.  The
// rotation rule (the tolerance test and the angle) is the batched SVD
// kernel's; only the pair order differs from the oracle's cyclic order,
// which changes results within the SVD tolerance, not the kept rank on
// gapped spectra.
//
// GB300: the work is FP64 (the Jacobi rotations cannot be split into lower
// precision without losing the small singular values).  Each round reads
// every column of G and V twice and writes the rotated ones once; at
// n = 8192 (1 GB for G and V) a round is bound by HBM, about 0.5 ms, and a
// sweep by its n - 1 rounds.  This is a fallback: its cost is stated, not
// hidden (seconds at n = 4096, tens of seconds at n = 8192).
#include <cuda_runtime.h>
#include <math.h>

#include <vector>

#include "asolve_internal.cuh"

namespace asv {

constexpr int kSvdThreads = 256;
constexpr int kSvdMaxSweeps = 30;

namespace {

__global__ void k_svdl_init(const double* __restrict__ A, int64_t n, double* __restrict__ G, int64_t ldg,
                            double* __restrict__ V) {
  const int64_t total = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / n, i = e - j * n;
    G[j * ldg + i] = A[e];
    V[j * ldg + i] = (i == j) ? 1.0 : 0.0;
  }
}

// Round r of the round-robin order over np players (np even; player n is a
// dummy when n is odd): pair index pi -> (a, b).
__device__ __forceinline__ void rr_pair(int pi, int r, int np, int& p, int& q) {
  int a, b;
  if (pi == 0) {
    a = 0;
    b = 1 + r % (np - 1);
  } else {
    a = 1 + (pi + r) % (np - 1);
    b = 1 + (np - 1 - pi + r) % (np - 1);
  }
  p = a < b ? a : b;
  q = a < b ? b : a;
}

__global__ void __launch_bounds__(kSvdThreads) k_svdl_round(double* __restrict__ G, double* __restrict__ V,
                                                            int64_t ldg, int n, int np, int r, double tol,
                                                            int* rotated) {
  const int lane = threadIdx.x & 31;
  const int pi = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (pi >= np / 2) return;  // the whole warp
  int p, q;
  rr_pair(pi, r, np, p, q);
  if (q >= n) return;
  double* gp = G + (size_t)p * ldg;
  double* gq = G + (size_t)q * ldg;
  double al = 0.0, be = 0.0, ga = 0.0;
  for (int k = lane; k < n; k += 32) {
    const double x = gp[k], y = gq[k];
    al = fma(x, x, al);
    be = fma(y, y, be);
    ga = fma(x, y, ga);
  }
  al = warp_sum(al);
  be = warp_sum(be);
  ga = warp_sum(ga);
  if (!(fabs(ga) > tol * sqrt(al) * sqrt(be))) return;
  const double zeta = (be - al) / (2.0 * ga);
  const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  const double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
  for (int k = lane; k < n; k += 32) {
    const double x = gp[k], y = gq[k];
    gp[k] = c * x - sn * y;
    gq[k] = sn * x + c * y;
  }
  double* vp = V + (size_t)p * ldg;
  double* vq = V + (size_t)q * ldg;
  for (int k = lane; k < n; k += 32) {
    const double x = vp[k], y = vq[k];
    vp[k] = c * x - sn * y;
    vq[k] = sn * x + c * y;
  }
  if (lane == 0) atomicOr(rotated, 1);
}

// sigma_j = ||G_j||_2, a warp per column.
__global__ void __launch_bounds__(kSvdThreads) k_svdl_sigma(const double* __restrict__ G, int64_t ldg, int n,
                                                            double* __restrict__ sigma) {
  const int lane = threadIdx.x & 31;
  const int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (j >= n) return;
  const double* g = G + (size_t)j * ldg;
  double s = 0.0;
  for (int k = lane; k < n; k += 32) s = fma(g[k], g[k], s);
  s = warp_sum(s);
  if (lane == 0) sigma[j] = sqrt(s);
}

// W(j, c) = (U_j . b_c) / sigma_j for sigma_j > tau, else 0; a warp per
// (column j, right-hand side c).
__global__ void __launch_bounds__(kSvdThreads) k_svdl_coef(const double* __restrict__ G, int64_t ldg, int n,
                                                           const double* __restrict__ B, int nrhs,
                                                           const double* __restrict__ sigma, double tau,
                                                           double* __restrict__ W) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (w >= (int64_t)n * nrhs) return;
  const int j = (int)(w % n), c = (int)(w / n);
  const double sj = sigma[j];
  double wj = 0.0;
  if (sj > tau) {
    const double* g = G + (size_t)j * ldg;
    const double* b = B + (size_t)c * n;
    double s = 0.0;
    for (int k = lane; k < n; k += 32) s += (g[k] / sj) * b[k];
    s = warp_sum(s);
    wj = s / sj;
  }
  if (lane == 0) W[(size_t)c * n + j] = wj;
}

// X(:, c) = V W(:, c): a thread per row, the columns of V in order.
__global__ void __launch_bounds__(kSvdThreads) k_svdl_apply(const double* __restrict__ V, int64_t ldg, int n,
                                                            const double* __restrict__ W, int nrhs,
                                                            double* __restrict__ X) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * nrhs) return;
  const int r = (int)(e % n), c = (int)(e / n);
  const double* wc = W + (size_t)c * n;
  double x = 0.0;
  for (int i = 0; i < n; ++i) {
    const double wi = wc[i];
    if (wi != 0.0) x += V[(size_t)i * ldg + r] * wi;
  }
  X[(size_t)c * n + r] = x;
}

unsigned blocks_for(int64_t threads) { return (unsigned)((threads + kSvdThreads - 1) / kSvdThreads); }

}  // namespace

size_t large_svd_ws_bytes(int64_t n, int64_t nrhs) {
  const size_t ldg = (size_t)((n + 3) & ~3);
  return sizeof(double) * ldg * (size_t)n + 256 +  // V
         sizeof(double) * (size_t)n + 256 +         // sigma
         sizeof(double) * (size_t)n * nrhs + 256 +  // W
         256;                                        // flag
}

// Minimum-norm solution of A X = B through the one-sided Jacobi SVD.
// G: device buffer of ldg * n doubles (ldg = n rounded up to 4) that the
// routine overwrites; ws: large_svd_ws_bytes(n, nrhs) bytes.  trunc_rel:
// tau = trunc_rel * sigma_max (0: n eps).  *rank: the number of singular
// values kept; *sweeps: the sweeps run.  Returns ASOLVE_OK or an error.
int large_svd(const double* A, int64_t n64, const double* B, double* X, int64_t nrhs, double trunc_rel,
              double* G, void* ws, int64_t* rank, int* sweeps, cudaStream_t st) {
  if (n64 <= 0 || n64 > kSvdLargeMax || nrhs < 1) return ASOLVE_E_UNSUPPORTED;
  const int n = (int)n64;
  const int64_t ldg = (n + 3) & ~3;
  char* p = static_cast<char*>(ws);
  auto take = [&](size_t b) {
    char* r = p;
    p += (b + 255) & ~(size_t)255;
    return r;
  };
  double* V = reinterpret_cast<double*>(take(sizeof(double) * (size_t)ldg * n));
  double* sigma = reinterpret_cast<double*>(take(sizeof(double) * (size_t)n));
  double* W = reinterpret_cast<double*>(take(sizeof(double) * (size_t)n * nrhs));
  int* rotated = reinterpret_cast<int*>(take(sizeof(int)));
  k_svdl_init<<<1024, kSvdThreads, 0, st>>>(A, n64, G, ldg, V);
  if (cudaGetLastError() != cudaSuccess) return ASOLVE_E_CUDA;
  const int np = (n + 1) & ~1;
  const double tol = (double)n * kEps;
  const unsigned grid = blocks_for((int64_t)32 * (np / 2));
  int sw = 0;
  for (; sw < kSvdMaxSweeps; ++sw) {
    if (cudaMemsetAsync(rotated, 0, sizeof(int), st) != cudaSuccess) return ASOLVE_E_CUDA;
    for (int r = 0; r < np - 1; ++r) k_svdl_round<<<grid, kSvdThreads, 0, st>>>(G, V, ldg, n, np, r, tol, rotated);
    if (cudaGetLastError() != cudaSuccess) return ASOLVE_E_CUDA;
    int h = 0;
    if (cudaMemcpyAsync(&h, rotated, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return ASOLVE_E_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return ASOLVE_E_CUDA;
    if (!h) {
      ++sw;
      break;
    }
  }
  k_svdl_sigma<<<blocks_for((int64_t)32 * n), kSvdThreads, 0, st>>>(G, ldg, n, sigma);
  std::vector<double> hs((size_t)n);
  if (cudaMemcpyAsync(hs.data(), sigma, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return ASOLVE_E_CUDA;
  double smax = 0.0;
  for (double s : hs) smax = fmax(smax, s);
  const double tau = (trunc_rel > 0.0 ? trunc_rel : (double)n * kEps) * smax;
  int64_t kept = 0;
  for (double s : hs) kept += s > tau ? 1 : 0;
  k_svdl_coef<<<blocks_for((int64_t)32 * n * nrhs), kSvdThreads, 0, st>>>(G, ldg, n, B, (int)nrhs, sigma, tau, W);
  k_svdl_apply<<<blocks_for((int64_t)n * nrhs), kSvdThreads, 0, st>>>(V, ldg, n, W, (int)nrhs, X);
  if (cudaGetLastError() != cudaSuccess) return ASOLVE_E_CUDA;
  if (rank) *rank = kept;
  if (sweeps) *sweeps = sw;
  return ASOLVE_OK;
}

}  // namespace asv
