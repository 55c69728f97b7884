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
// With 16-bit operands (kind::f16, BF16 or FP16) every operand is rounded
// once to the 16-bit type and one product is accumulated in FP32: the
// low-precision trailing update of mixed-precision factorisations, whose
// accuracy iterative refinement recovers.  FP16 operand tiles are scaled by
// powers of two chosen from each tile's largest magnitude (per-tile
// scaling, undone exactly in the epilogue), so no entry leaves FP16 range.
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
#include <stdlib.h>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

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

// Instruction descriptors of kind::f16: D = F32, A = B = BF16 (type 1) or
// FP16 (type 0), both K-major, N = 128, M = 128.
constexpr uint32_t kIdescBf16 =
    (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
constexpr uint32_t kIdescFp16 = (1u << 4) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);

template <uint32_t IDESC>
__device__ __forceinline__ void tc_mma_f16(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t accum) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(ad), "l"(bd), "r"(IDESC), "r"(accum));
}

// Instruction descriptor of kind::f8f6f4: D = F32, A = B = E4M3 (type 0),
// both K-major, N = 128, M = 128.
constexpr uint32_t kIdescE4m3 = (1u << 4) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);

__device__ __forceinline__ void tc_mma_f8(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t accum) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(ad), "l"(bd), "r"(kIdescE4m3), "r"(accum));
}

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

// A reduced limit (tests of the timeout path) polls with the non-blocking
// test_wait: try_wait may itself wait for a while before it returns.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, long long limit = kSpinLimit) {
  uint32_t done = 0;
  if (limit < kSpinLimit) {
    for (long long it = 0; it < limit; ++it) {
      asm volatile(
          "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done)
          : "r"(mbar), "r"(parity)
          : "memory");
      if (done) return true;
    }
    return false;
  }
  for (long long it = 0; it < limit; ++it) {
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

// byte offset of element (row r, k) of a 128 x 64 K-major tile of 16-bit
// elements: the same core-matrix geometry (8 rows x 16 bytes) as above
__device__ __forceinline__ uint32_t tc_off16(int r, int k) {
  return (uint32_t)((((r >> 3) * 8 + (k >> 3)) * 128) + ((r & 7) * 16) + ((k & 7) * 2));
}

// two consecutive-K elements, scaled, rounded to the 16-bit type and packed
// (element k in the low half)
template <int OP>
__device__ __forceinline__ uint32_t pack16(float lo, float hi, float s) {
  if (OP == kGemmBf16) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo * s, hi * s);
    return *reinterpret_cast<const uint32_t*>(&v);
  } else {
    const __half2 v = __floats2half2_rn(lo * s, hi * s);
    return *reinterpret_cast<const uint32_t*>(&v);
  }
}

// exponent of the power-of-two scale that brings a tile's largest magnitude
// m into [2^14, 2^15) (FP16 range; FP8 E4M3, whose largest value is 448:
// [2^7, 2^8)), clamped to +-60 so that both scales and the product that
// undoes them stay normal FP32 numbers; 0 for a zero or non-finite tile
template <int OP = kGemmFp16>
__device__ __forceinline__ int tile_shift(float m) {
  if (!(m > 0.f) || !(m <= 3.0e38f)) return 0;
  return max(-60, min(60, (OP == kGemmFp8 ? 7 : 14) - ilogbf(m)));
}

// four consecutive-K elements, scaled, rounded to E4M3 (saturating) and
// packed, element k in the lowest byte
__device__ __forceinline__ uint32_t pack8(float v0, float v1, float v2, float v3, float s) {
  const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(v0 * s, v1 * s), __NV_SATFINITE, __NV_E4M3);
  const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(v2 * s, v3 * s), __NV_SATFINITE, __NV_E4M3);
  return (lo & 0xffffu) | (hi << 16);
}

// byte offset of element (row r, k) of a 128 x 128 K-major tile of 8-bit
// elements: the core-matrix geometry of the 16-bit tiles (8 rows x 16 bytes)
__device__ __forceinline__ uint32_t tc_off8(int r, int k) {
  return (uint32_t)((((r >> 3) * 8 + (k >> 4)) * 128) + ((r & 7) * 16) + (k & 15));
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
__global__ void __launch_bounds__(kTcThreads, 3)
    k_gemm_tc(float* __restrict__ C, int ldc, const float* __restrict__ A, int lda, const float* __restrict__ B,
              int ldb, int M, int N, int K, int passes, int* err, long long wait_limit) {
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
  // Each thread's 32 elements of A and of B for one K chunk are loaded into
  // registers together (all loads in flight at once); the next chunk's
  // loads are issued while the tensor core works on the current one.
  //   A: thread t holds row t, k = 0..31 (coalesced over rows)
  //   B: (n, k) with lanes over k (or over n when B is transposed)
  constexpr int kPer = kTcM * kTcK / kTcThreads;  // 32
  float va[kPer], vb[kPer];
  auto load_chunk = [&](int k0) {
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int r = tid, k = i;
      va[i] = (m0 + r < M && k0 + k < K) ? __ldg(A + (size_t)(k0 + k) * lda + m0 + r) : 0.f;
    }
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int e = tid + i * kTcThreads;
      const int k = TRANS_B ? (e >> 7) : (e & (kTcK - 1)), n = TRANS_B ? (e & (kTcN - 1)) : (e >> 5);
      float v = 0.f;
      if (n0 + n < N && k0 + k < K)
        v = TRANS_B ? __ldg(B + (size_t)(k0 + k) * ldb + n0 + n) : __ldg(B + (size_t)(n0 + n) * ldb + k0 + k);
      vb[i] = v;
    }
  };
  if (nchunks > 0) load_chunk(0);
  for (int ch = 0; ch < nchunks && ok; ++ch) {
    // stage the registers: A element (r, k), B element (n, k)
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      float hi, lo;
      tf32_split(va[i], hi, lo);
      *reinterpret_cast<float*>(sAh + tc_off(tid, i)) = (passes == 3) ? hi : va[i];
      if (passes == 3) *reinterpret_cast<float*>(sAl + tc_off(tid, i)) = lo;
    }
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int e = tid + i * kTcThreads;
      const int k = TRANS_B ? (e >> 7) : (e & (kTcK - 1)), n = TRANS_B ? (e & (kTcN - 1)) : (e >> 5);
      float hi, lo;
      tf32_split(vb[i], hi, lo);
      *reinterpret_cast<float*>(sBh + tc_off(n, k)) = (passes == 3) ? hi : vb[i];
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
    if (ch + 1 < nchunks) load_chunk((ch + 1) * kTcK);  // in flight during the MMAs
    // the stage may be rewritten only after the MMAs have read it; the
    // verdict is made uniform across the block before anyone acts on it
    const bool waited = mbar_wait(mbar_a, phase, wait_limit);
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

// 16-bit operands (OP = kGemmBf16 or kGemmFp16): K chunks of 64, four
// K = 16 MMAs per chunk; FP8 E4M3 (OP = kGemmFp8): K chunks of 128, four
// K = 32 MMAs of kind::f8f6f4 (the same bytes per chunk and core-matrix
// geometry); otherwise the structure of k_gemm_tc.
template <bool TRANS_B, bool LOWER, int OP>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_gemm_tc16(float* __restrict__ C, int ldc, const float* __restrict__ A, int lda, const float* __restrict__ B,
                int ldb, int M, int N, int K, int* err, long long wait_limit) {
  constexpr bool kF8 = OP == kGemmFp8;
  constexpr int kK = kF8 ? 128 : 64;
  constexpr uint32_t kIdesc = OP == kGemmBf16 ? kIdescBf16 : kIdescFp16;
  if (LOWER && blockIdx.y > blockIdx.x) return;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ float s_max[2][kTcThreads / 32];
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kTcM, n0 = blockIdx.y * kTcN;
  unsigned char* sA = smem;
  unsigned char* sB = smem + kTileBytes;
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
  // FP16: scales from the largest magnitudes of this tile's A rows and B
  // columns over all of K
  int sha = 0, shb = 0;
  if (OP == kGemmFp16 || kF8) {
    float am = 0.f, bm = 0.f;
    for (int k = w; k < K; k += kTcThreads / 32)
      for (int r = lane; r < kTcM; r += 32)
        if (m0 + r < M) am = fmaxf(am, fabsf(__ldg(A + (size_t)k * lda + m0 + r)));
    if (TRANS_B) {
      for (int k = w; k < K; k += kTcThreads / 32)
        for (int c = lane; c < kTcN; c += 32)
          if (n0 + c < N) bm = fmaxf(bm, fabsf(__ldg(B + (size_t)k * ldb + n0 + c)));
    } else {
      for (int c = w; c < kTcN; c += kTcThreads / 32)
        if (n0 + c < N)
          for (int k = lane; k < K; k += 32) bm = fmaxf(bm, fabsf(__ldg(B + (size_t)(n0 + c) * ldb + k)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, o));
      bm = fmaxf(bm, __shfl_xor_sync(0xffffffffu, bm, o));
    }
    if (lane == 0) {
      s_max[0][w] = am;
      s_max[1][w] = bm;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (OP == kGemmFp16 || kF8) {
    float am = 0.f, bm = 0.f;
#pragma unroll
    for (int q = 0; q < kTcThreads / 32; ++q) {
      am = fmaxf(am, s_max[0][q]);
      bm = fmaxf(bm, s_max[1][q]);
    }
    sha = tile_shift<OP>(am);
    shb = tile_shift<OP>(bm);
  }
  const float sa = ldexpf(1.f, sha), sb = ldexpf(1.f, shb);
  const uint32_t tmem = tmem_base;
  bool ok = true;
  uint32_t phase = 0;
  const int nchunks = (K + kK - 1) / kK;
  for (int ch = 0; ch < nchunks && ok; ++ch) {
    const int k0 = ch * kK;
    if constexpr (kF8) {
      // FP8: quadruples (r, k..k+3), lanes over r; (n, k..k+3), lanes over k
      // (over n when B is given transposed)
      for (int e = tid; e < kTcM * kK / 4; e += kTcThreads) {
        const int r = e & (kTcM - 1), k = 4 * (e >> 7);
        float v[4] = {0.f, 0.f, 0.f, 0.f};
        if (m0 + r < M)
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (k0 + k + q < K) v[q] = __ldg(A + (size_t)(k0 + k + q) * lda + m0 + r);
        *reinterpret_cast<uint32_t*>(sA + tc_off8(r, k)) = pack8(v[0], v[1], v[2], v[3], sa);
      }
      for (int e = tid; e < kTcN * kK / 4; e += kTcThreads) {
        const int n = TRANS_B ? (e & (kTcN - 1)) : (e >> 5);
        const int k = TRANS_B ? 4 * (e >> 7) : 4 * (e & 31);
        float v[4] = {0.f, 0.f, 0.f, 0.f};
        if (n0 + n < N)
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (k0 + k + q < K)
              v[q] = TRANS_B ? __ldg(B + (size_t)(k0 + k + q) * ldb + n0 + n)
                             : __ldg(B + (size_t)(n0 + n) * ldb + k0 + k + q);
        *reinterpret_cast<uint32_t*>(sB + tc_off8(n, k)) = pack8(v[0], v[1], v[2], v[3], sb);
      }
    } else {
    // A: element pairs (r, k), (r, k + 1); lanes over r
    for (int e = tid; e < kTcM * kK / 2; e += kTcThreads) {
      const int r = e & (kTcM - 1), k = 2 * (e >> 7);
      float v0 = 0.f, v1 = 0.f;
      if (m0 + r < M) {
        if (k0 + k < K) v0 = __ldg(A + (size_t)(k0 + k) * lda + m0 + r);
        if (k0 + k + 1 < K) v1 = __ldg(A + (size_t)(k0 + k + 1) * lda + m0 + r);
      }
      *reinterpret_cast<uint32_t*>(sA + tc_off16(r, k)) = pack16<OP>(v0, v1, sa);
    }
    // B: element pairs (n, k), (n, k + 1); lanes over k, or over n when
    // B is given transposed
    for (int e = tid; e < kTcN * kK / 2; e += kTcThreads) {
      const int n = TRANS_B ? (e & (kTcN - 1)) : (e >> 5);
      const int k = TRANS_B ? 2 * (e >> 7) : 2 * (e & 31);
      float v0 = 0.f, v1 = 0.f;
      if (n0 + n < N) {
        if (TRANS_B) {
          if (k0 + k < K) v0 = __ldg(B + (size_t)(k0 + k) * ldb + n0 + n);
          if (k0 + k + 1 < K) v1 = __ldg(B + (size_t)(k0 + k + 1) * ldb + n0 + n);
        } else {
          if (k0 + k < K) v0 = __ldg(B + (size_t)(n0 + n) * ldb + k0 + k);
          if (k0 + k + 1 < K) v1 = __ldg(B + (size_t)(n0 + n) * ldb + k0 + k + 1);
        }
      }
      *reinterpret_cast<uint32_t*>(sB + tc_off16(n, k)) = pack16<OP>(v0, v1, sb);
    }
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
      for (int j = 0; j < 4; ++j) {  // K = 16 (FP8: 32) per MMA: two core matrices
        const uint32_t off = (uint32_t)j * 256;
        if constexpr (kF8)
          tc_mma_f8(tmem, tc_desc(smem_u32(sA) + off, 128, 1024), tc_desc(smem_u32(sB) + off, 128, 1024),
                    (ch > 0 || j > 0) ? 1u : 0u);
        else
          tc_mma_f16<kIdesc>(tmem, tc_desc(smem_u32(sA) + off, 128, 1024), tc_desc(smem_u32(sB) + off, 128, 1024),
                             (ch > 0 || j > 0) ? 1u : 0u);
      }
      tc_commit(mbar_a);
    }
    const bool waited = mbar_wait(mbar_a, phase, wait_limit);
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    ok = __syncthreads_and(waited && ok) != 0;
  }
  if (!ok) mbar_wait(mbar_a, phase ^ 1u);
  if (ok && nchunks > 0) {
    const float inv = ldexpf(1.f, -(sha + shb));  // undoes the operand scales exactly
    const int r = m0 + 32 * w + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < kTcN; c0 += 32) {
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
          if (c < N) C[(size_t)c * ldc + r] = cv[j] - __uint_as_float(v[j]) * inv;
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

// Poll limit of the stage waits: kSpinLimit, or, for tests of the timeout
// path, the value of the environment variable ASOLVE_WAIT_LIMIT (read at
// every launch).  A wait that runs out raises the error flag; the kernel
// then drains its MMAs with the full limit before it frees tensor memory.
static long long wait_limit() {
  const char* e = getenv("ASOLVE_WAIT_LIMIT");
  if (!e || !*e) return kSpinLimit;
  const long long v = atoll(e);
  return v > 0 ? v : kSpinLimit;
}

template <bool TB, bool LO, int OP>
static cudaError_t launch_gemm_tc16_t(float* C, int ldc, const float* A, int lda, const float* B, int ldb, int M,
                                      int N, int K, int* err, cudaStream_t st) {
  const int smem = 4 * kTileBytes;  // as k_gemm_tc: at most 3 CTAs (384 TMEM columns) per SM
  cudaError_t e = ASV_SMEM_LIMIT_ONCE((k_gemm_tc16<TB, LO, OP>), smem);
  if (e != cudaSuccess) return e;
  dim3 grid((M + kTcM - 1) / kTcM, (N + kTcN - 1) / kTcN);
  k_gemm_tc16<TB, LO, OP><<<grid, kTcThreads, smem, st>>>(C, ldc, A, lda, B, ldb, M, N, K, err, wait_limit());
  return cudaGetLastError();
}

template <int OP>
static cudaError_t launch_gemm_tc16(float* C, int ldc, const float* A, int lda, const float* B, int ldb, int M,
                                    int N, int K, int* err, cudaStream_t st, bool trans_b, bool lower) {
  if (trans_b && lower) return launch_gemm_tc16_t<true, true, OP>(C, ldc, A, lda, B, ldb, M, N, K, err, st);
  if (trans_b) return launch_gemm_tc16_t<true, false, OP>(C, ldc, A, lda, B, ldb, M, N, K, err, st);
  if (lower) return launch_gemm_tc16_t<false, true, OP>(C, ldc, A, lda, B, ldb, M, N, K, err, st);
  return launch_gemm_tc16_t<false, false, OP>(C, ldc, A, lda, B, ldb, M, N, K, err, st);
}

template <bool TB, bool LO>
static cudaError_t launch_gemm_tc_t(float* C, int ldc, const float* A, int lda, const float* B, int ldb, int M,
                                    int N, int K, int passes, int* err, cudaStream_t st) {
  // always 64 KB: at most 3 CTAs per SM, i.e. at most 384 of the 512
  // tensor-memory columns, so an allocation never waits on another CTA
  const int smem = 4 * kTileBytes;
  cudaError_t e = ASV_SMEM_LIMIT_ONCE((k_gemm_tc<TB, LO>), smem);
  if (e != cudaSuccess) return e;
  dim3 grid((M + kTcM - 1) / kTcM, (N + kTcN - 1) / kTcN);
  k_gemm_tc<TB, LO><<<grid, kTcThreads, smem, st>>>(C, ldc, A, lda, B, ldb, M, N, K, passes, err, wait_limit());
  return cudaGetLastError();
}

cudaError_t launch_gemm_tc(float* C, int ldc, const float* A, int lda, const float* B, int ldb, int M, int N,
                           int K, int passes, int* err, cudaStream_t st, bool trans_b, bool lower) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (passes == kGemmBf16)
    return launch_gemm_tc16<kGemmBf16>(C, ldc, A, lda, B, ldb, M, N, K, err, st, trans_b, lower);
  if (passes == kGemmFp16)
    return launch_gemm_tc16<kGemmFp16>(C, ldc, A, lda, B, ldb, M, N, K, err, st, trans_b, lower);
  if (passes == kGemmFp8)
    return launch_gemm_tc16<kGemmFp8>(C, ldc, A, lda, B, ldb, M, N, K, err, st, trans_b, lower);
  if (trans_b && lower) return launch_gemm_tc_t<true, true>(C, ldc, A, lda, B, ldb, M, N, K, passes, err, st);
  if (trans_b) return launch_gemm_tc_t<true, false>(C, ldc, A, lda, B, ldb, M, N, K, passes, err, st);
  if (lower) return launch_gemm_tc_t<false, true>(C, ldc, A, lda, B, ldb, M, N, K, passes, err, st);
  return launch_gemm_tc_t<false, false>(C, ldc, A, lda, B, ldb, M, N, K, passes, err, st);
}

}  // namespace asv
