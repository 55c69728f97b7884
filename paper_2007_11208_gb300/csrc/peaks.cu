// peaks.cu -- issue-rate probes of the arithmetic pipes the solver's
// latency-bound kernels run on: FP32 FMA, FP64 FMA and the FP64 tensor
// instruction mma.sync m8n8k4.  They give the roofline denominators of the
// kernels that no copy or cuBLAS measurement bounds (the batched class
// kernels factor in FP32 on the FMA pipe and refine in FP64).
//
// Each probe runs a grid of several CTAs per SM; every thread (every warp
// for the tensor instruction) keeps 8 independent accumulator chains so
// that the pipe, not the dependency latency, sets the rate.  The chains
// start from values the compiler cannot fold and are stored at the end,
// so no operation is removed.  flops are counted as 2 per FMA and
// 2 * 8 * 8 * 4 per m8n8k4.
#include <cuda_runtime.h>

#include "asolve_internal.cuh"

namespace asv {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kPeakThreads) k_peak_ffma(float* out, int iters, float a, float b) {
  float c[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) c[k] = (float)(threadIdx.x + k) * 1e-7f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int k = 0; k < kChains; ++k) c[k] = fmaf(c[k], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += c[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_dfma(double* out, int iters, double a, double b) {
  double c[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) c[k] = (double)(threadIdx.x + k) * 1e-7;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int k = 0; k < kChains; ++k) c[k] = fma(c[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += c[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_dmma(double* out, int iters, double a, double b) {
  double c0[kChains], c1[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) c0[k] = c1[k] = (double)(threadIdx.x + k) * 1e-9;
  const double av = a * (double)(threadIdx.x & 3), bv = b;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int k = 0; k < kChains; ++k)
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                     : "+d"(c0[k]), "+d"(c1[k])
                     : "d"(av), "d"(bv));
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += c0[k] + c1[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace asv

using namespace asv;

extern "C" int asolve_pipe_peak(int pipe, int iters, double* tflops, double* ms_out) {
  if (!tflops || iters < 1 || pipe < ASOLVE_PIPE_FFMA || pipe > ASOLVE_PIPE_DMMA) return ASOLVE_E_INVALID;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ASOLVE_E_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return ASOLVE_E_CUDA;
  const int grid = sms * 8;  // 8 CTAs of 256 threads: 64 warps per SM
  const size_t cnt = (size_t)grid * kPeakThreads;
  void* out = nullptr;
  if (cudaMalloc(&out, cnt * sizeof(double)) != cudaSuccess) return ASOLVE_E_NOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto launch = [&](int it) {
    if (pipe == ASOLVE_PIPE_FFMA)
      k_peak_ffma<<<grid, kPeakThreads>>>(static_cast<float*>(out), it, 0.999999f, 1e-6f);
    else if (pipe == ASOLVE_PIPE_DFMA)
      k_peak_dfma<<<grid, kPeakThreads>>>(static_cast<double*>(out), it, 0.999999, 1e-6);
    else
      k_peak_dmma<<<grid, kPeakThreads>>>(static_cast<double*>(out), it, 1e-3, 0.5);
  };
  launch(iters / 8 + 1);  // warm-up (clocks ramp, module load)
  cudaEventRecord(e0);
  launch(iters);
  cudaEventRecord(e1);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  if (err == cudaSuccess) err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return ASOLVE_E_CUDA;
  double flops;
  if (pipe == ASOLVE_PIPE_DMMA)  // per warp: iters * 4 * kChains instructions of 512 flops
    flops = (double)grid * (kPeakThreads / 32) * iters * 4.0 * kChains * 512.0;
  else
    flops = (double)cnt * iters * 16.0 * kChains * 2.0;
  *tflops = flops / (ms * 1e-3) / 1e12;
  if (ms_out) *ms_out = ms;
  return ASOLVE_OK;
}
