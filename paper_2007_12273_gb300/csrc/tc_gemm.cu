// tc_gemm.cu -- BF16 GEMM on the 5th-generation tensor cores (tcgen05) for
// the learned-initialisation network.
//
//   C[M,N] = A[M,K] . B[N,K]^T   (+ bias[N]) (ReLU) (* (mask > 0))
//
// A and B are BF16, "K-major" (row-major with K contiguous); accumulation is
// FP32 in tensor memory (TMEM).  One CTA (4 warps) computes a 128 x BN tile:
// the K dimension is walked in chunks of 64; each chunk of A (128 x 64) and
// B (BN x 64) is staged in shared memory in the canonical no-swizzle
// core-matrix layout (8 rows x 16 bytes per core matrix), one thread issues
// four tcgen05.mma (K = 16 each) and commits them to an mbarrier; the
// epilogue reads the accumulator with tcgen05.ld (warp w owns TMEM lanes
// 32w..32w+31 = tile rows) and applies bias / ReLU / mask.
//
// Every wait on the mbarrier is bounded; on time-out the kernel records an
// error flag, releases its TMEM and returns.
#include "gm_kernels.cuh"

#include <cuda_bf16.h>

namespace gmcr {

namespace {

constexpr int kBM = 128;   // tile rows (MMA M)
constexpr int kBK = 64;    // K chunk staged per round (4 MMAs of K = 16)
constexpr uint32_t kWaitLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor, no swizzle: start address, leading-
// dimension byte offset (between core matrices adjacent along K) and stride
// byte offset (between core matrices adjacent along M/N), all >> 4;
// descriptor version 1 (bits 46-47)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  uint32_t done = 0;
  for (uint32_t it = 0; it < kWaitLimit; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

template <int N>
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[N]) {
  static_assert(N == 16, "16 columns per load");
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace

// BN: tile columns (16..256, multiple of 16); TMEM columns = BN rounded up
// to a power of two >= 32.
template <int BN>
__global__ void __launch_bounds__(128) tc_gemm_kernel(const __nv_bfloat16* __restrict__ A,
                                                      const __nv_bfloat16* __restrict__ B, int M,
                                                      int N, int K, int lda, int ldb,
                                                      const float* __restrict__ bias, int relu,
                                                      const __nv_bfloat16* __restrict__ mask,
                                                      int ldm, float* __restrict__ Cf,
                                                      __nv_bfloat16* __restrict__ Cb, int ldc,
                                                      int accumulate, unsigned int* err) {
  constexpr int TCOLS = BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
  constexpr uint32_t IDESC = idesc_bf16(kBM, BN);
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;                    // 128 x 64 bf16 = 16 KB
  unsigned char* sB = smem + kBM * kBK * 2;    // BN x 64 bf16
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ int failed;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
  const uint32_t mbar_a = smem_u32(&mbar);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar_a));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    failed = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;

  uint32_t phase = 0;
  const int nk = (K + kBK - 1) / kBK;
  for (int kc = 0; kc < nk; ++kc) {
    const int k0 = kc * kBK;
    // stage A (128 x 64) and B (BN x 64): 16-byte chunks; core matrix (i, j)
    // (rows 8i.., K columns 8j..) at byte (i * 8 + j) * 128, row r % 8 at +16
    for (int c = tid; c < (kBM + BN) * 8; c += 128) {
      const bool isA = c < kBM * 8;
      const int cc = isA ? c : c - kBM * 8;
      const int r = cc >> 3, j = cc & 7;
      const int gr = (isA ? m0 : n0) + r, gk = k0 + 8 * j;
      uint4 val = make_uint4(0u, 0u, 0u, 0u);
      const int rows = isA ? M : N;
      if (gr < rows && gk + 8 <= K) {
        const __nv_bfloat16* src = isA ? A + (size_t)gr * lda + gk : B + (size_t)gr * ldb + gk;
        val = *reinterpret_cast<const uint4*>(src);
      } else if (gr < rows && gk < K) {
        __nv_bfloat16 t[8];
        const __nv_bfloat16* src = isA ? A + (size_t)gr * lda : B + (size_t)gr * ldb;
        for (int e = 0; e < 8; ++e) t[e] = (gk + e < K) ? src[gk + e] : __float2bfloat16(0.0f);
        val = *reinterpret_cast<uint4*>(t);
      }
      unsigned char* dst = (isA ? sA : sB) + ((r >> 3) * 8 + j) * 128 + (r & 7) * 16;
      *reinterpret_cast<uint4*>(dst) = val;
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
      for (int s = 0; s < kBK / 16; ++s) {
        const uint64_t ad = smem_desc(a0 + s * 256, 128, 1024);
        const uint64_t bd = smem_desc(b0 + s * 256, 128, 1024);
        const uint32_t acc = (kc > 0 || s > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(IDESC), "r"(acc));
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              mbar_a)
          : "memory");
    }
    // the MMAs of this chunk must finish before its tiles are overwritten
    if (!mbar_wait(mbar_a, phase)) {
      failed = 1;
      if (err) atomicOr(err, 1u);
    }
    phase ^= 1u;
    __syncthreads();
    if (failed) break;
  }
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");

  if (!failed) {
    // epilogue: thread (warp w, lane l) owns tile row 32 w + l
    const int row = m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < BN; c0 += 16) {
      float v[16];
      tmem_ld16<16>(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (row < M) {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int col = n0 + c0 + e;
          if (col >= N) continue;
          float x = v[e];
          if (bias) x += bias[col];
          if (relu) x = fmaxf(x, 0.0f);
          if (mask && !(__bfloat162float(mask[(size_t)row * ldm + col]) > 0.0f)) x = 0.0f;
          if (Cf) {
            float* cp = Cf + (size_t)row * ldc + col;
            *cp = accumulate ? *cp + x : x;
          }
          if (Cb) Cb[(size_t)row * ldc + col] = __float2bfloat16(x);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TCOLS));
}

size_t tc_gemm_smem(int bn) { return (size_t)(kBM + bn) * kBK * 2 + 1024; }

cudaError_t launch_tc_gemm(const void* A, const void* B, int M, int N, int K, int lda, int ldb,
                           const float* bias, int relu, const void* mask, int ldm, float* Cf,
                           void* Cb, int ldc, unsigned int* err, cudaStream_t s, int accumulate) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  int bn = N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : 256));
  // at least 80 KB of shared memory per CTA keeps two CTAs (2 x 256 TMEM
  // columns) per SM at most, so a TMEM allocation never waits
  size_t smem = tc_gemm_smem(bn);
  if (smem < 80 * 1024) smem = 80 * 1024;
  dim3 grid((M + kBM - 1) / kBM, (N + bn - 1) / bn);
#define GM_TC_LAUNCH(BNV)                                                                        \
  {                                                                                              \
    auto k = tc_gemm_kernel<BNV>;                                                                \
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,        \
                                         (int)smem);                                             \
    if (e != cudaSuccess) return e;                                                              \
    k<<<grid, 128, smem, s>>>((const __nv_bfloat16*)A, (const __nv_bfloat16*)B, M, N, K, lda,    \
                              ldb, bias, relu, (const __nv_bfloat16*)mask, ldm, Cf,              \
                              (__nv_bfloat16*)Cb, ldc, accumulate, err);                         \
  }
  if (bn == 32) GM_TC_LAUNCH(32)
  else if (bn == 64) GM_TC_LAUNCH(64)
  else if (bn == 128) GM_TC_LAUNCH(128)
  else GM_TC_LAUNCH(256)
#undef GM_TC_LAUNCH
  return cudaGetLastError();
}

}  // namespace gmcr
