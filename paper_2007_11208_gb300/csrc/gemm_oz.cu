// gemm_oz.cu -- FP64-accurate matrix products on the BF16 tensor cores by
// the Ozaki splitting (Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of
// matrix multiplication", Numer. Algorithms 59, 2012).
//
//   C (M x N) -= A (M x K) * op(B),   all FP64, column-major;
//   op(B) = B (K x N), or with transb B given as an N x K matrix.
//
// On this GPU FP64 issues at two lanes per clock per SM, so the FP64
// factorisations' trailing updates, the blocked triangular solves' updates
// and the residuals with many right-hand sides are bound by that pipe.
// Here every FP64 operand becomes a sum of kOzS exact BF16 slices and the
// product becomes slice products on the tensor cores, accumulated exactly:
//
// * Scales.  For each row i of A and each K chunk of kOzKc columns, E_i is
//   the largest biased exponent in the chunk and sigma_i = 2^(E_i - 1021),
//   so |a_ik| < sigma_i / 2.  Likewise F_j, tau_j per column of op(B).
// * Slices.  T = round(|a| 2^56 / sigma) (an integer below 2^55, from the
//   bits of a with integer shifts) is written in balanced base 2^8:
//   T = sum_s d_s 2^(8 (6 - s)), |d_s| <= 128, so a = sigma sum_s d_s
//   2^(-8 (s + 1)) up to 2^-57 sigma.  Each d_s is exact in BF16.
// * Products.  For s + t = g the products d_s e_t (|.| <= 2^14) over a K
//   chunk of 128 sum to an integer below (g + 1) 128 2^14 < 2^24 for
//   g <= 6, so a tensor-memory FP32 accumulator D_g sums every pair of the
//   diagonal g exactly whatever the order of the additions.  The 28 pairs
//   s + t <= 6 are kept; the dropped ones and the slicing contribute an
//   error of about 2^-48 sigma tau per chunk, the size of an FP64 GEMM's.
// * Epilogue.  V = sum_g D_g 2^(8 (6 - g) - 12) is formed in 64-bit
//   integers (the last two shifts rounded), converted once to FP64 and
//   C -= V 2^(E + F - 2094) is one FMA: one FP64 operation per element and
//   K chunk, against kOzKc for an FP64 GEMM.
//
// Splitting is a separate pass (k_oz_split_a / k_oz_split_b) that writes
// each operand tile's kOzS slices contiguously in the tensor cores'
// K-major core-matrix layout, so the GEMM stages a whole tile with two
// bulk copies (cp.async.bulk, completion counted on an mbarrier).  One CTA
// (4 warps) computes a 128 x 64 tile of C; one elected thread issues the
// MMAs; the epilogue reads the seven accumulators with tcgen05.ld.  Every
// wait is bounded: on timeout the kernel raises the error flag, waits for
// its copies and MMAs with the full limit, frees its tensor memory and
// returns.
#include <stdint.h>
#include <stdlib.h>

#include <cuda_bf16.h>

#include "asolve_internal.cuh"

namespace asv {
namespace {

constexpr int kOzS = 7;                          // slices per operand
constexpr int kOzM = 128, kOzN = 64;             // C tile
constexpr int kOzKs = 64;                        // K per staged tile
constexpr int kOzKc = 128;                       // K per exact accumulation
constexpr int kOzThreads = 128;
constexpr int kOzABytes = kOzM * kOzKs * 2;      // one A slice tile: 16 KB
constexpr int kOzBBytes = kOzN * kOzKs * 2;      // one B slice tile: 8 KB
constexpr int kOzSmem = kOzS * (kOzABytes + kOzBBytes);  // 168 KB
constexpr int kOzTmemCols = 512;                 // 7 accumulators of 64 columns
constexpr long long kOzSpin = 20000000;
constexpr int kOzNonFinite = 0x7ff;

__device__ __forceinline__ uint32_t oz_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (row r, k) of a K-major tile of 16-bit elements
// with 64 K per row: core matrices of 8 rows x 16 bytes, K-adjacent ones
// 128 B apart, 8-row groups 1024 B apart
__device__ __forceinline__ uint32_t oz_off(int r, int k) {
  return (uint32_t)((((r >> 3) * 8 + (k >> 3)) * 128) + ((r & 7) * 16) + ((k & 7) * 2));
}

__device__ __forceinline__ uint64_t oz_desc(uint32_t saddr) {  // K-major, no swizzle, LBO 128, SBO 1024
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((1024u >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// kind::f16: D = F32, A = B = BF16, both K-major, N = 64, M = 128
constexpr uint32_t kOzIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kOzN >> 3) << 17) |
                              ((uint32_t)(kOzM >> 4) << 24);

__device__ __forceinline__ void oz_mma(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t accum) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(ad), "l"(bd), "r"(kOzIdesc), "r"(accum));
}

__device__ __forceinline__ bool oz_wait(uint32_t mbar, uint32_t parity, long long limit) {
  uint32_t done = 0;
  if (limit < kOzSpin) {  // tests of the timeout path: non-blocking polls
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

// Biased exponent of a for the scale (subnormals and zero count as 1 and
// 0, non-finite values as kOzNonFinite).
__device__ __forceinline__ int oz_expo(double a) {
  const uint64_t b = (uint64_t)__double_as_longlong(a);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e == 0) return (b << 1) != 0 ? 1 : 0;
  return e;
}

// The kOzS balanced base-2^8 digits of a relative to the scale exponent E
// (E >= the exponent of a; 0 < E < kOzNonFinite), most significant first.
__device__ __forceinline__ void oz_digits(double a, int E, int* d) {
  const uint64_t b = (uint64_t)__double_as_longlong(a);
  int e = (int)((b >> 52) & 0x7ff);
  uint64_t m = b & 0xFFFFFFFFFFFFFull;
  if (e == 0) e = 1;
  else m |= 1ull << 52;
  const int sh = E - e - 2;  // T = m 2^-sh, rounded
  int64_t T;
  if (sh <= 0) T = (int64_t)(m << (-sh));
  else if (sh > 54) T = 0;
  else T = (int64_t)((m + (1ull << (sh - 1))) >> sh);
  if (b >> 63) T = -T;
#pragma unroll
  for (int s = kOzS - 1; s >= 1; --s) {
    int v = (int)(T & 0xff);
    if (v >= 128) v -= 256;
    d[s] = v;
    T = (T - v) >> 8;
  }
  d[0] = (int)T;
}

__device__ __forceinline__ uint32_t oz_pack(int lo, int hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn((float)lo, (float)hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// A (M x K, lda) -> slices: tile (mt, ks) of 128 rows x 64 K holds its kOzS
// slice tiles contiguously at As + ((mt * nks + ks) * kOzS + s) * kOzABytes;
// eA[kc * Mp + i]: the scale exponent of row i in K chunk kc.
// Grid (ceil(M / 128), ceil(K / 128)), 256 threads.
__global__ void __launch_bounds__(256) k_oz_split_a(const double* __restrict__ A, int lda, int M, int K,
                                                    unsigned char* __restrict__ As, int* __restrict__ eA, int Mp) {
  __shared__ int s_e[2][kOzM];
  const int mt = blockIdx.x, kc = blockIdx.y, tid = threadIdx.x;
  const int m0 = mt * kOzM, k0 = kc * kOzKc;
  const int nks = (K + kOzKs - 1) / kOzKs;
  {  // row exponents over the chunk: two threads per row, 64 K each
    const int r = tid & (kOzM - 1), h = tid >> 7;
    int em = 0;
    if (m0 + r < M)
      for (int k = k0 + h * 64; k < min(K, k0 + h * 64 + 64); ++k)
        em = max(em, oz_expo(__ldg(A + (size_t)k * lda + m0 + r)));
    s_e[h][r] = em;
  }
  __syncthreads();
  if (tid < kOzM && m0 + tid < M) eA[(size_t)kc * Mp + m0 + tid] = max(s_e[0][tid], s_e[1][tid]);
  // element pairs (r, k), (r, k + 1): lanes over r
  for (int e = tid; e < kOzM * kOzKc / 2; e += 256) {
    const int r = e & (kOzM - 1), k = 2 * (e >> 7);
    const int E = max(s_e[0][r], s_e[1][r]);
    int d0[kOzS], d1[kOzS];
#pragma unroll
    for (int s = 0; s < kOzS; ++s) d0[s] = d1[s] = 0;
    if (m0 + r < M && E > 0 && E < kOzNonFinite) {
      if (k0 + k < K) oz_digits(__ldg(A + (size_t)(k0 + k) * lda + m0 + r), E, d0);
      if (k0 + k + 1 < K) oz_digits(__ldg(A + (size_t)(k0 + k + 1) * lda + m0 + r), E, d1);
    }
    const int ks = (k0 + k) / kOzKs;
    if (ks >= nks) continue;
    unsigned char* base = As + ((size_t)mt * nks + ks) * kOzS * kOzABytes;
    const uint32_t off = oz_off(r, (k0 + k) % kOzKs);
#pragma unroll
    for (int s = 0; s < kOzS; ++s)
      *reinterpret_cast<uint32_t*>(base + (size_t)s * kOzABytes + off) = oz_pack(d0[s], d1[s]);
  }
}

// op(B) (K x N) -> slices: tile (nt, ks) of 64 columns x 64 K at
// Bs + ((nt * nks + ks) * kOzS + s) * kOzBBytes; eB[kc * Np + j].
// TB: B given as an N x K matrix (element (k, j) at B[k * ldb + j]).
// Grid (ceil(N / 64), ceil(K / 128)), 256 threads.
template <bool TB>
__global__ void __launch_bounds__(256) k_oz_split_b(const double* __restrict__ B, int ldb, int N, int K,
                                                    unsigned char* __restrict__ Bs, int* __restrict__ eB, int Np) {
  __shared__ int s_e[4][kOzN];
  const int nt = blockIdx.x, kc = blockIdx.y, tid = threadIdx.x;
  const int n0 = nt * kOzN, k0 = kc * kOzKc;
  const int nks = (K + kOzKs - 1) / kOzKs;
  {  // column exponents: four threads per column, 32 K each
    const int c = tid & (kOzN - 1), q = tid >> 6;
    int em = 0;
    if (n0 + c < N)
      for (int k = k0 + q * 32; k < min(K, k0 + q * 32 + 32); ++k)
        em = max(em, oz_expo(TB ? __ldg(B + (size_t)k * ldb + n0 + c) : __ldg(B + (size_t)(n0 + c) * ldb + k)));
    s_e[q][c] = em;
  }
  __syncthreads();
  if (tid < kOzN && n0 + tid < N)
    eB[(size_t)kc * Np + n0 + tid] = max(max(s_e[0][tid], s_e[1][tid]), max(s_e[2][tid], s_e[3][tid]));
  for (int e = tid; e < kOzN * kOzKc / 2; e += 256) {
    // pairs (c, k), (c, k + 1): lanes over k (B) or over c (TB)
    const int c = TB ? (e & (kOzN - 1)) : (e >> 6);
    const int k = TB ? 2 * (e >> 6) : 2 * (e & 63);
    const int E = max(max(s_e[0][c], s_e[1][c]), max(s_e[2][c], s_e[3][c]));
    int d0[kOzS], d1[kOzS];
#pragma unroll
    for (int s = 0; s < kOzS; ++s) d0[s] = d1[s] = 0;
    if (n0 + c < N && E > 0 && E < kOzNonFinite) {
      if (k0 + k < K)
        oz_digits(TB ? __ldg(B + (size_t)(k0 + k) * ldb + n0 + c) : __ldg(B + (size_t)(n0 + c) * ldb + k0 + k), E,
                  d0);
      if (k0 + k + 1 < K)
        oz_digits(TB ? __ldg(B + (size_t)(k0 + k + 1) * ldb + n0 + c)
                     : __ldg(B + (size_t)(n0 + c) * ldb + k0 + k + 1),
                  E, d1);
    }
    const int ks = (k0 + k) / kOzKs;
    if (ks >= nks) continue;
    unsigned char* base = Bs + ((size_t)nt * nks + ks) * kOzS * kOzBBytes;
    const uint32_t off = oz_off(c, (k0 + k) % kOzKs);
#pragma unroll
    for (int s = 0; s < kOzS; ++s)
      *reinterpret_cast<uint32_t*>(base + (size_t)s * kOzBBytes + off) = oz_pack(d0[s], d1[s]);
  }
}

// D_g (FP32, an exact integer below 2^24) as an int
__device__ __forceinline__ int64_t oz_int(uint32_t bits) { return (int64_t)__float2int_rn(__uint_as_float(bits)); }

// LOWER: C is square and only its lower triangle is needed.
template <bool LOWER>
__global__ void __launch_bounds__(kOzThreads, 1)
    k_gemm_oz(double* __restrict__ C, int ldc, const unsigned char* __restrict__ As, const int* __restrict__ eA,
              int Mp, const unsigned char* __restrict__ Bs, const int* __restrict__ eB, int Np, int M, int N, int K,
              int* err, long long wait_limit) {
  const int m0 = blockIdx.x * kOzM, n0 = blockIdx.y * kOzN;
  if (LOWER && n0 >= m0 + kOzM) return;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar[2];  // [0] copies landed, [1] MMAs done
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  unsigned char* sA = smem;
  unsigned char* sB = smem + kOzS * kOzABytes;
  const uint32_t mb_ld = oz_smem(&mbar[0]), mb_mma = oz_smem(&mbar[1]);
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(oz_smem(&tmem_base)),
                 "r"(kOzTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb_ld));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb_mma));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_base;
  const int nks = (K + kOzKs - 1) / kOzKs, nkc = (K + kOzKc - 1) / kOzKc;
  const int mt = blockIdx.x, nt = blockIdx.y;
  bool ok = true;
  uint32_t ph_ld = 0, ph_mma = 0;
  bool ld_pending = false, mma_pending = false;
  for (int kc = 0; kc < nkc && ok; ++kc) {
    const int nsub = min(kOzKc / kOzKs, nks - kc * (kOzKc / kOzKs));
    for (int sub = 0; sub < nsub && ok; ++sub) {
      const int ks = kc * (kOzKc / kOzKs) + sub;
      if (tid == 0) {
        const unsigned char* ga = As + ((size_t)mt * nks + ks) * kOzS * kOzABytes;
        const unsigned char* gb = Bs + ((size_t)nt * nks + ks) * kOzS * kOzBBytes;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mb_ld), "r"(kOzSmem)
                     : "memory");
        for (int s = 0; s < kOzS; ++s) {
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                  oz_smem(sA + s * kOzABytes)),
              "l"(ga + (size_t)s * kOzABytes), "r"(kOzABytes), "r"(mb_ld)
              : "memory");
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                  oz_smem(sB + s * kOzBBytes)),
              "l"(gb + (size_t)s * kOzBBytes), "r"(kOzBBytes), "r"(mb_ld)
              : "memory");
        }
      }
      ld_pending = true;
      const bool landed = oz_wait(mb_ld, ph_ld, wait_limit);
      ok = __syncthreads_and(landed) != 0;
      if (!ok) break;
      ph_ld ^= 1u;
      ld_pending = false;
      if (w == 0) {  // lane 0 issues; the other lanes wait at the warp barrier, not on the mbarrier
        if (lane == 0) {
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
          const uint64_t da = oz_desc(oz_smem(sA)), db = oz_desc(oz_smem(sB));
          for (int s = 0; s < kOzS; ++s)
            for (int t = 0; s + t < kOzS; ++t) {
              const uint32_t acc_col = tmem + (uint32_t)((s + t) * kOzN);
#pragma unroll
              for (int j = 0; j < kOzKs / 16; ++j)  // K = 16 per MMA: two core matrices (16-byte units)
                oz_mma(acc_col, da + (uint64_t)((s * kOzABytes + j * 256) >> 4),
                       db + (uint64_t)((t * kOzBBytes + j * 256) >> 4), (sub > 0 || s > 0 || j > 0) ? 1u : 0u);
            }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mb_mma)
                       : "memory");
        }
        __syncwarp();
      }
      mma_pending = true;
      const bool done = oz_wait(mb_mma, ph_mma, wait_limit);
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      ok = __syncthreads_and(done) != 0;
      if (!ok) break;
      ph_mma ^= 1u;
      mma_pending = false;
    }
    if (!ok) break;
    // drain: warp w owns rows 32w..32w+31, 16 columns at a time; the
    // group's loads of C and of the column scales go out together, before
    // the accumulator reads, and its stores after all of them
    const int r = m0 + 32 * w + lane;
    const int E = r < M ? __ldg(eA + (size_t)kc * Mp + r) : 0;
#pragma unroll 1
    for (int c0 = 0; c0 < kOzN; c0 += 16) {
      double cv[16];
      int F[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int c = n0 + c0 + j;
        const bool in = r < M && c < N;
        F[j] = c < N ? __ldg(eB + (size_t)kc * Np + c) : 0;
        cv[j] = in ? C[(size_t)c * ldc + r] : 0.0;
      }
      uint32_t v[kOzS][16];
#pragma unroll
      for (int g = 0; g < kOzS; ++g) {
        const uint32_t taddr = tmem + ((uint32_t)(32 * w) << 16) + (uint32_t)(g * kOzN + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
            "[%16];\n"
            : "=r"(v[g][0]), "=r"(v[g][1]), "=r"(v[g][2]), "=r"(v[g][3]), "=r"(v[g][4]), "=r"(v[g][5]),
              "=r"(v[g][6]), "=r"(v[g][7]), "=r"(v[g][8]), "=r"(v[g][9]), "=r"(v[g][10]), "=r"(v[g][11]),
              "=r"(v[g][12]), "=r"(v[g][13]), "=r"(v[g][14]), "=r"(v[g][15])
            : "r"(taddr));
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (r < M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int c = n0 + c0 + j;
          if (c >= N || E == 0 || F[j] == 0) continue;  // a zero row or column of this chunk
          if (E == kOzNonFinite || F[j] == kOzNonFinite) {
            cv[j] = __longlong_as_double(0x7ff8000000000000ll);
          } else {
            const int64_t V = (oz_int(v[0][j]) << 36) + (oz_int(v[1][j]) << 28) + (oz_int(v[2][j]) << 20) +
                              (oz_int(v[3][j]) << 12) + (oz_int(v[4][j]) << 4) + ((oz_int(v[5][j]) + 8) >> 4) +
                              ((oz_int(v[6][j]) + 2048) >> 12);
            // C -= V 2^(E + F - 2094): the power of two built from its
            // bits when it is a normal double, else scalbn
            const int x = E + F[j] - 2094;
            if (x >= -1022 && x <= 1023) cv[j] = fma(-(double)V, __longlong_as_double((long long)(x + 1023) << 52), cv[j]);
            else cv[j] = cv[j] - scalbn((double)V, x);
          }
          C[(size_t)c * ldc + r] = cv[j];
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();  // the accumulators are read before the next chunk overwrites them
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  }
  if (!ok) {
    // a wait gave up: let the copies and MMAs in flight finish (bounded)
    // before the shared and tensor memory they write are released
    if (ld_pending) oz_wait(mb_ld, ph_ld, kOzSpin);
    if (mma_pending) oz_wait(mb_mma, ph_mma, kOzSpin);
    if (tid == 0 && err) atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (w == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kOzTmemCols));
  }
}

long long oz_wait_limit() {
  const char* e = getenv("ASOLVE_WAIT_LIMIT");
  if (!e || !*e) return kOzSpin;
  const long long v = atoll(e);
  return v > 0 ? v : kOzSpin;
}

}  // namespace

size_t gemm_oz_ws_bytes(int M, int N, int K) {
  if (M <= 0 || N <= 0 || K <= 0) return 0;
  const size_t mt = (size_t)(M + kOzM - 1) / kOzM, nt = (size_t)(N + kOzN - 1) / kOzN;
  const size_t nks = (size_t)(K + kOzKs - 1) / kOzKs, nkc = (size_t)(K + kOzKc - 1) / kOzKc;
  const size_t Mp = mt * kOzM, Np = nt * kOzN;
  auto r256 = [](size_t b) { return (b + 255) & ~(size_t)255; };
  return r256(mt * nks * kOzS * kOzABytes) + r256(nt * nks * kOzS * kOzBBytes) + r256(nkc * Mp * sizeof(int)) +
         r256(nkc * Np * sizeof(int));
}

// C -= A op(B) by the Ozaki splitting; ws: gemm_oz_ws_bytes(M, N, K) bytes
// (256-byte aligned).  tb: B given as an N x K matrix; lower: only the
// lower triangle of the square C is needed.
cudaError_t gemm_oz(double* C, int ldc, const double* A, int lda, const double* B, int ldb, int M, int N, int K,
                    bool tb, bool lower, void* ws, int* err, cudaStream_t st) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  static PerDeviceOnce once;
  cudaError_t e = once.run([] {
    cudaError_t r = cudaFuncSetAttribute(k_gemm_oz<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kOzSmem);
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(k_gemm_oz<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kOzSmem);
    return r;
  });
  if (e != cudaSuccess) return e;
  const int mt = (M + kOzM - 1) / kOzM, nt = (N + kOzN - 1) / kOzN;
  const int nks = (K + kOzKs - 1) / kOzKs, nkc = (K + kOzKc - 1) / kOzKc;
  const int Mp = mt * kOzM, Np = nt * kOzN;
  auto r256 = [](size_t b) { return (b + 255) & ~(size_t)255; };
  unsigned char* p = static_cast<unsigned char*>(ws);
  unsigned char* As = p;
  p += r256((size_t)mt * nks * kOzS * kOzABytes);
  unsigned char* Bs = p;
  p += r256((size_t)nt * nks * kOzS * kOzBBytes);
  int* eA = reinterpret_cast<int*>(p);
  p += r256((size_t)nkc * Mp * sizeof(int));
  int* eB = reinterpret_cast<int*>(p);
  k_oz_split_a<<<dim3(mt, nkc), 256, 0, st>>>(A, lda, M, K, As, eA, Mp);
  if (tb) k_oz_split_b<true><<<dim3(nt, nkc), 256, 0, st>>>(B, ldb, N, K, Bs, eB, Np);
  else k_oz_split_b<false><<<dim3(nt, nkc), 256, 0, st>>>(B, ldb, N, K, Bs, eB, Np);
  const long long lim = oz_wait_limit();
  if (lower) k_gemm_oz<true><<<dim3(mt, nt), kOzThreads, kOzSmem, st>>>(C, ldc, As, eA, Mp, Bs, eB, Np, M, N, K, err, lim);
  else k_gemm_oz<false><<<dim3(mt, nt), kOzThreads, kOzSmem, st>>>(C, ldc, As, eA, Mp, Bs, eB, Np, M, N, K, err, lim);
  return cudaGetLastError();
}

}  // namespace asv
