// gemm_tc.cu -- trailing-update GEMM of the large dense factorisations on the
// 5th-generation tensor cores (tcgen05, accumulators in tensor memory).
//
//   C (M x N) -= A (M x K) * B (K x N),   all FP32, column-major.
//
// The products run as kind::tf32 MMAs with FP32 accumulation.  With
// passes = 3 every operand is split into a TF32 head and its FP32 remainder
// and the three significant products (head*head, head*rest, rest*head) are
// accumulated, which recovers FP32-level accuracy (relative error ~2^-21)
// at three times the tensor work.
//
// One CTA (4 warps) computes one 128 x 128 tile of C.  For each 32-wide K
// chunk the warps stage A and B into shared memory in the K-major,
// non-swizzled core-matrix layout (8 rows x 16 bytes per core matrix;
// K-adjacent core matrices 128 B apart, 8-row groups 1024 B apart), one
// elected thread issues the MMAs, and tcgen05.commit signals an mbarrier
// when they have consumed the stage.  The epilogue reads the accumulator
// from tensor memory with tcgen05.ld (warp w owns rows 32w..32w+31) and
// writes C - acc with coalesced stores.  Every wait is bounded: on timeout
// the kernel raises the error flag, frees its tensor memory and returns.
#include "asolve_internal.cuh"

namespace asv {

constexpr int kTcM = 128, kTcN = 128, kTcK = 32;
constexpr int kTcThreads = 128;
constexpr int kTileBytes = kTcM * kTcK * 4;  // 16 KB per operand copy
constexpr long long kSpinLimit = 20000000;   // mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: K-major, no swizzle, version 1.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor: D = F32, A = B = TF32, both K-major, N = 128, M = 128.
constexpr uint32_t kIdescTf32 =
    (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);

__device__ __forceinline__ void tc_mma_tf32(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t accum) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(ad), "l"(bd), "r"(kIdescTf32), "r"(accum));
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  uint32_t done = 0;
  for (long long it = 0; it < kSpinLimit; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// byte offset of element (row r, k) of a 128 x 32 K-major tile
__device__ __forceinline__ uint32_t tc_off(int r, int k) {
  return (uint32_t)((((r >> 3) * 8 + (k >> 2)) * 128) + ((r & 7) * 16) + ((k & 3) * 4));
}

// TF32 head of x (low 13 mantissa bits cleared) and the remainder.
__device__ __forceinline__ void tf32_split(float x, float& hi, float& lo) {
  hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
  lo = x - hi;
}

// TRANS_B: B is given transposed, element (k, n) at B[k * ldb + n].
// LOWER: C is square and only its lower triangle is needed; tiles strictly
// above the diagonal are skipped.
template <bool TRANS_B, bool LOWER>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_gemm_tc(float* __restrict__ C, int ldc, const float* __restrict__ A, int lda, const float* __restrict__ B,
              int ldb, int M, int N, int K, int passes, int* err) {
  if (LOWER && blockIdx.y > blockIdx.x) return;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kTcM, n0 = blockIdx.y * kTcN;
  // stage layout: A head, B head, [A rest, B rest]
  unsigned char* sAh = smem;
  unsigned char* sBh = smem + kTileBytes;
  unsigned char* sAl = smem + 2 * kTileBytes;
  unsigned char* sBl = smem + 3 * kTileBytes;
  const uint32_t mbar_a = smem_u32(&mbar);
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                 "r"(kTcN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar_a));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_base;
  bool ok = true;
  uint32_t phase = 0;
  const int nchunks = (K + kTcK - 1) / kTcK;
  for (int ch = 0; ch < nchunks && ok; ++ch) {
    const int k0 = ch * kTcK;
    // stage A: element (r, k) = A[(k0 + k) * lda + m0 + r]; lanes over r
    for (int e = tid; e < kTcM * kTcK; e += kTcThreads) {
      const int r = e & (kTcM - 1), k = e >> 7;
      const float v = (m0 + r < M && k0 + k < K) ? __ldg(A + (size_t)(k0 + k) * lda + m0 + r) : 0.f;
      float hi, lo;
      tf32_split(v, hi, lo);
      *reinterpret_cast<float*>(sAh + tc_off(r, k)) = (passes == 3) ? hi : v;
      if (passes == 3) *reinterpret_cast<float*>(sAl + tc_off(r, k)) = lo;
    }
    // stage B: element (n, k) = B[(n0 + n) * ldb + k0 + k] (lanes over k),
    // or B[(k0 + k) * ldb + n0 + n] when transposed (lanes over n)
    for (int e = tid; e < kTcN * kTcK; e += kTcThreads) {
      const int k = TRANS_B ? (e >> 7) : (e & (kTcK - 1)), n = TRANS_B ? (e & (kTcN - 1)) : (e >> 5);
      float v = 0.f;
      if (n0 + n < N && k0 + k < K)
        v = TRANS_B ? __ldg(B + (size_t)(k0 + k) * ldb + n0 + n) : __ldg(B + (size_t)(n0 + n) * ldb + k0 + k);
      float hi, lo;
      tf32_split(v, hi, lo);
      *reinterpret_cast<float*>(sBh + tc_off(n, k)) = (passes == 3) ? hi : v;
      if (passes == 3) *reinterpret_cast<float*>(sBl + tc_off(n, k)) = lo;
    }
    // generic-proxy writes -> visible to the tensor core's async proxy
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
      for (int j = 0; j < kTcK / 8; ++j) {  // K = 8 per tf32 MMA: two core matrices
        const uint32_t off = (uint32_t)j * 256;
        const uint64_t ah = tc_desc(smem_u32(sAh) + off, 128, 1024);
        const uint64_t bh = tc_desc(smem_u32(sBh) + off, 128, 1024);
        tc_mma_tf32(tmem, ah, bh, (ch > 0 || j > 0) ? 1u : 0u);
        if (passes == 3) {
          const uint64_t al = tc_desc(smem_u32(sAl) + off, 128, 1024);
          const uint64_t bl = tc_desc(smem_u32(sBl) + off, 128, 1024);
          tc_mma_tf32(tmem, ah, bl, 1u);
          tc_mma_tf32(tmem, al, bh, 1u);
        }
      }
      tc_commit(mbar_a);
    }
    // the stage may be rewritten only after the MMAs have read it; the
    // verdict is made uniform across the block before anyone acts on it
    const bool waited = mbar_wait(mbar_a, phase);
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    ok = __syncthreads_and(waited && ok) != 0;
  }
  if (!ok) {
    // a wait gave up: give the MMAs in flight a bounded chance to finish
    // before the tensor memory they write is released
    mbar_wait(mbar_a, phase ^ 1u);
  }
  if (ok && nchunks > 0) {
    // epilogue: warp w reads rows 32w..32w+31, 32 columns at a time
    const int r = m0 + 32 * w + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < kTcN; c0 += 32) {
      // the 32 loads of C go out together, before the accumulator read
      float cv[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int c = n0 + c0 + j;
        cv[j] = (r < M && c < N) ? C[(size_t)c * ldc + r] : 0.f;
      }
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(32 * w) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
            "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
            "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
            "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (r < M) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int c = n0 + c0 + j;
          if (c < N) C[(size_t)c * ldc + r] = cv[j] - __uint_as_float(v[j]);
        }
      }
    }
  }
  if (!ok && tid == 0 && err) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (w == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTcN));
  }
}

template <bool TB, bool LO>
static cudaError_t launch_gemm_tc_t(float* C, int ldc, const float* A, int lda, const float* B, int ldb, int M,
                                    int N, int K, int passes, int* err, cudaStream_t st) {
  // always 64 KB: at most 3 CTAs per SM, i.e. at most 384 of the 512
  // tensor-memory columns, so an allocation never waits on another CTA
  const int smem = 4 * kTileBytes;
  static bool attr = false;
  if (!attr) {
    cudaError_t e =
        cudaFuncSetAttribute(k_gemm_tc<TB, LO>, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * kTileBytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid((M + kTcM - 1) / kTcM, (N + kTcN - 1) / kTcN);
  k_gemm_tc<TB, LO><<<grid, kTcThreads, smem, st>>>(C, ldc, A, lda, B, ldb, M, N, K, passes, err);
  return cudaGetLastError();
}

cudaError_t launch_gemm_tc(float* C, int ldc, const float* A, int lda, const float* B, int ldb, int M, int N,
                           int K, int passes, int* err, cudaStream_t st, bool trans_b, bool lower) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (trans_b && lower) return launch_gemm_tc_t<true, true>(C, ldc, A, lda, B, ldb, M, N, K, passes, err, st);
  if (trans_b) return launch_gemm_tc_t<true, false>(C, ldc, A, lda, B, ldb, M, N, K, passes, err, st);
  if (lower) return launch_gemm_tc_t<false, true>(C, ldc, A, lda, B, ldb, M, N, K, passes, err, st);
  return launch_gemm_tc_t<false, false>(C, ldc, A, lda, B, ldb, M, N, K, passes, err, st);
}

}  // namespace asv
