// noalloc.cu -- a property scan that allocates no device memory.
//
// Some callers cannot allocate: code running where the allocator must not
// be entered (a real-time or latency-critical loop, a host application
// that hands out all device memory itself through its own pool, a plugin
// that is not allowed to grow the process's footprint), or code that has
// no asolve context to own a workspace.  asolve_scan_noalloc serves them:
// it runs the same scan kernels as asolve_scan, but its workspace is a
// fixed file-scope device array instead of memory the library allocates.
//
// That array is part of the module: every GPU that loads the library holds
// it until the process exits, and every call shares it.  Calls that overlap
// on the GPU (two streams, two host threads) therefore race on it; callers
// must order them.  Each call clears the part that has to start at zero.
#include <cuda_runtime.h>
#include <mutex>

#include "asolve_internal.cuh"

namespace asv {
cudaError_t launch_scan_large(const double* A, int64_t n, const double* B, int64_t nb, double band_frac,
                              double tol, void* ws, ScanRes* out, int num_sms, cudaStream_t st);
size_t scan_large_workspace(int64_t n);
}  // namespace asv

using namespace asv;

namespace {

constexpr int64_t kNoAllocNMax = 2048;         // largest n this entry point accepts
constexpr size_t kNoAllocBytes = 1152 * 1024;  // scan workspace for n <= 2048, plus the result
constexpr int kMaxDevices = 64;

// The workspace.  In host code the name below is only a handle for the
// runtime; its device address is looked up once per device.
static __device__ __align__(256) unsigned char g_noalloc_ws[kNoAllocBytes];

std::mutex g_setup_mu;
void* g_ws_addr[kMaxDevices] = {};
int g_num_sms[kMaxDevices] = {};

// Copy the internal scan record into the public layout (device to device).
__global__ void k_scan_result_out(const ScanRes* in, asolve_scan_result* out, int64_t n) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  asolve_scan_result r = {};
  if (n > 0) {
    const ScanRes s = *in;
    r.kl = s.kl;
    r.ku = s.ku;
    r.lower = (s.flags & SF_LOWER) != 0;
    r.upper = (s.flags & SF_UPPER) != 0;
    r.sympd = (s.flags & SF_SYMPD) != 0;
    r.banded = (s.flags & SF_BANDED) != 0;
    r.nonfinite = (s.flags & SF_NONFINITE) != 0;
    r.cls = s.cls;
    r.norm1 = s.norm1;
    r.norminf = s.norminf;
  }
  *out = r;
}

// Device address of the workspace on the current device (set up on the
// first call for that device).
int workspace_for_current_device(void** ws, int* num_sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ASOLVE_E_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return ASOLVE_E_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_ws_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_ws) != cudaSuccess || !p) return ASOLVE_E_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return ASOLVE_E_CUDA;
    g_ws_addr[dev] = p;
    g_num_sms[dev] = sms;
  }
  *ws = g_ws_addr[dev];
  *num_sms = g_num_sms[dev];
  return ASOLVE_OK;
}

}  // namespace

extern "C" int asolve_scan_noalloc(const double* A, int64_t n, asolve_scan_result* out, void* stream) {
  if (!out || n < 0 || (n > 0 && !A)) return ASOLVE_E_INVALID;
  if (n > kNoAllocNMax) return ASOLVE_E_UNSUPPORTED;
  const size_t need = ((scan_large_workspace(n) + 255) & ~(size_t)255) + 256;
  if (need > kNoAllocBytes) return ASOLVE_E_UNSUPPORTED;
  void* ws = nullptr;
  int sms = 0;
  int rc = workspace_for_current_device(&ws, &sms);
  if (rc != ASOLVE_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  ScanRes* res = reinterpret_cast<ScanRes*>(static_cast<char*>(ws) + (need - 256));
  if (n > 0) {
    // the launcher clears the scan's accumulators on the stream itself
    if (launch_scan_large(A, n, A, 0, 0.25, 100.0 * kEps, ws, res, sms, st) != cudaSuccess)
      return ASOLVE_E_CUDA;
  }
  k_scan_result_out<<<1, 32, 0, st>>>(res, out, n);
  if (cudaGetLastError() != cudaSuccess) return ASOLVE_E_CUDA;
  return ASOLVE_OK;
}
