// tc_gemm.cu -- BF16 GEMM on the 5th-generation tensor cores (tcgen05) for
// the learned-initialisation network.
//
//   C[M,N] = A[M,K] . B[N,K]^T   (+ bias[N]) (ReLU) (* (mask > 0))
//
// A and B are BF16, "K-major" (row-major with K contiguous); accumulation is
// FP32 in tensor memory (TMEM).  One CTA (4 warps) computes a 128 x BN tile,
// walking K in chunks of 64 through an S-stage shared-memory ring:
//   * thread 0 (warp 0) is the producer: per chunk one TMA tiled load
//     (cp.async.bulk.tensor) of A (64 x 128) and one of B (64 x BN) with the
//     128-byte swizzle, completing on the stage's "full" mbarrier;
//   * thread 32 (warp 1) issues the four tcgen05.mma (K = 16 each) of a
//     chunk once it has landed and commits them to the stage's "empty"
//     mbarrier, which the producer waits on before refilling the stage;
//   * the epilogue (all 4 warps) reads the accumulator with tcgen05.ld (warp
//     w owns TMEM lanes 32w..32w+31 = tile rows) and applies bias / ReLU /
//     mask.
// Loads of later chunks overlap the MMAs of earlier ones.  The TMA fills
// rows and K columns outside the matrices with zeros.
//
// Every wait on an mbarrier is bounded; on time-out the kernel records an
// error flag, waits (bounded) for its copies in flight, releases its TMEM
// and returns.
#include "gm_kernels.cuh"

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <mutex>

namespace gmcr {

namespace {

constexpr int kBM = 128;   // tile rows (MMA M)
constexpr int kBK = 64;    // K chunk staged per round (4 MMAs of K = 16)
constexpr uint32_t kWaitLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor of a K-major operand in the 128-byte
// swizzled layout the TMA writes (rows of 64 BF16 = 128 bytes, 8-row groups
// of 1024 bytes): start address >> 4 (bits 0-13), leading-dimension offset
// field 1 (unused by this layout), stride byte offset 1024 >> 4 between
// 8-row groups (bits 32-45), descriptor version 1 (bit 46), layout type
// "128-byte swizzle" (2, bits 61-63).  The K = 16 slice s of a chunk starts
// 32 s bytes into each row; the stage buffers are 1024-byte aligned.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
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

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes)
               : "memory");
}

// 2D tiled TMA load of the box at (x, y) (x the K coordinate: a multiple of
// 64 elements, so 128-byte aligned) into shared memory, completing on mbar
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
      : "memory");
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

// BN: tile columns (32..256, a power of two); TMEM columns = BN rounded up
// to a power of two >= 32; S: pipeline stages
template <int BN, int S>
__global__ void __launch_bounds__(128) tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA,
                                                      const __grid_constant__ CUtensorMap mapB,
                                                      int M, int N, int K,
                                                      const float* __restrict__ bias, int relu,
                                                      const __nv_bfloat16* __restrict__ mask,
                                                      int ldm, float* __restrict__ Cf,
                                                      __nv_bfloat16* __restrict__ Cb, int ldc,
                                                      int accumulate, unsigned int* err) {
  constexpr int TCOLS = BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
  constexpr uint32_t IDESC = idesc_bf16(kBM, BN);
  constexpr uint32_t A_BYTES = kBM * kBK * 2, B_BYTES = BN * kBK * 2;
  constexpr uint32_t STAGE = A_BYTES + B_BYTES;  // a multiple of 1024
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // the stages start at the first 1024-byte boundary of the dynamic buffer
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  __shared__ __align__(8) uint64_t full[S], empty[S], done;
  __shared__ uint32_t tmem_slot;
  __shared__ int failed;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
  const int nk = (K + kBK - 1) / kBK;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    for (int q = 0; q < S; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&full[q])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&empty[q])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&done)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    failed = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (tid == 0) {
    // producer: chunk kc into stage kc % S, once the MMAs of chunk kc - S
    // (the stage's previous content) have completed
    int issued = 0;
    for (int kc = 0; kc < nk; ++kc) {
      const int st = kc % S;
      if (kc >= S && !mbar_wait(smem_u32(&empty[st]), (uint32_t)((kc / S - 1) & 1))) {
        failed = 1;
        if (err) atomicOr(err, 1u);
        break;
      }
      const uint32_t fb = smem_u32(&full[st]);
      const uint32_t sa = smem_u32(smem + (size_t)st * STAGE);
      mbar_expect_tx(fb, STAGE);
      tma_load_2d(sa, &mapA, kc * kBK, m0, fb);
      tma_load_2d(sa + A_BYTES, &mapB, kc * kBK, n0, fb);
      issued = kc + 1;
    }
    // on a time-out, wait (bounded) for the copies still in flight
    if (failed)
      for (int kc = (issued > S ? issued - S : 0); kc < issued; ++kc)
        mbar_wait(smem_u32(&full[kc % S]), (uint32_t)((kc / S) & 1));
  } else if (tid == 32) {
    // MMA issuer: the four K = 16 MMAs of each landed chunk, committed to the
    // stage's empty barrier; the last commit also signals the epilogue
    for (int kc = 0; kc < nk; ++kc) {
      const int st = kc % S;
      if (!mbar_wait(smem_u32(&full[st]), (uint32_t)((kc / S) & 1))) {
        failed = 1;
        if (err) atomicOr(err, 1u);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t a0 = smem_u32(smem + (size_t)st * STAGE), b0 = a0 + A_BYTES;
#pragma unroll
      for (int s = 0; s < kBK / 16; ++s) {
        const uint64_t ad = smem_desc_sw128(a0 + 32 * s);
        const uint64_t bd = smem_desc_sw128(b0 + 32 * s);
        const uint32_t acc = (kc > 0 || s > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(IDESC), "r"(acc));
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              smem_u32(&empty[st]))
          : "memory");
    }
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
            smem_u32(&done))
        : "memory");
  }
  // the accumulator is complete once the last commit arrives (the commit
  // tracks every earlier MMA of this thread)
  if (!mbar_wait(smem_u32(&done), 0u)) {
    failed = 1;
    if (err) atomicOr(err, 1u);
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");

  if (!failed) {
    // epilogue: thread (warp w, lane l) owns tile row 32 w + l and handles
    // 16 columns at a time; a full 16-column chunk of an aligned matrix is
    // moved with 16-byte vector accesses (32 B of BF16, 64 B of FP32 per
    // row), a ragged or unaligned one element by element
    const int row = m0 + warp * 32 + lane;
    const bool vf = !Cf || (((ldc & 3) == 0) && (((uintptr_t)Cf & 15) == 0));
    const bool vb = !Cb || (((ldc & 7) == 0) && (((uintptr_t)Cb & 15) == 0));
    const bool vm = !mask || (((ldm & 7) == 0) && (((uintptr_t)mask & 15) == 0));
    for (int c0 = 0; c0 < BN; c0 += 16) {
      float v[16];
      tmem_ld16<16>(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (row >= M || n0 + c0 >= N) continue;
      const int cb = n0 + c0;
      if (cb + 16 <= N && vf && vb && vm) {
        float x[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          x[e] = v[e];
          if (bias) x[e] += bias[cb + e];
          if (relu) x[e] = fmaxf(x[e], 0.0f);
        }
        if (mask) {
          const uint4* mp = reinterpret_cast<const uint4*>(mask + (size_t)row * ldm + cb);
          const uint4 q0 = mp[0], q1 = mp[1];
          const uint32_t mw[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const float mv = __uint_as_float((e & 1) ? (mw[e >> 1] & 0xFFFF0000u) : (mw[e >> 1] << 16));
            if (!(mv > 0.0f)) x[e] = 0.0f;
          }
        }
        if (Cf) {
          float4* cp = reinterpret_cast<float4*>(Cf + (size_t)row * ldc + cb);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float4 o = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
            if (accumulate) {
              const float4 a = cp[q];
              o.x += a.x; o.y += a.y; o.z += a.z; o.w += a.w;
            }
            cp[q] = o;
          }
        }
        if (Cb) {
          uint32_t pk[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(x[2 * q], x[2 * q + 1]);
            pk[q] = *reinterpret_cast<const uint32_t*>(&h);
          }
          uint4* bp = reinterpret_cast<uint4*>(Cb + (size_t)row * ldc + cb);
          bp[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
          bp[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
        }
        continue;
      }
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int col = cb + e;
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
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TCOLS));
}

// ring depth: two stages (48 KB each for 128 x 256 tiles), so that two CTAs
// share an SM (2 x 97 KB of shared memory, at most 2 x 256 TMEM columns)
// and one's ring fill and epilogue overlap the other's MMAs
template <int BN>
constexpr int gemm_stages() { return 2; }

size_t tc_gemm_smem(int bn) { return (size_t)(kBM + bn) * kBK * 2 * 2 + 1024; }

namespace {
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

// tensor map of a K-major BF16 matrix [rows][ld] (K valid columns): boxes
// of 64 K x box_rows, 128-byte swizzle, zero fill outside
bool make_map(CUtensorMap* map, const void* base, int rows, int K, int ld, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace

cudaError_t launch_tc_gemm(const void* A, const void* B, int M, int N, int K, int lda, int ldb,
                           const float* bias, int relu, const void* mask, int ldm, float* Cf,
                           void* Cb, int ldc, unsigned int* err, cudaStream_t s, int accumulate) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  int bn = N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : 256));
  CUtensorMap mapA, mapB;
  if (!make_map(&mapA, A, M, K, lda, kBM) || !make_map(&mapB, B, N, K, ldb, bn))
    return cudaErrorInvalidValue;
  // at least 80 KB of shared memory per CTA keeps two CTAs (2 x 256 TMEM
  // columns) per SM at most, so a TMEM allocation never waits
  size_t smem = tc_gemm_smem(bn);
  if (smem < 80 * 1024) smem = 80 * 1024;
  dim3 grid((M + kBM - 1) / kBM, (N + bn - 1) / bn);
#define GM_TC_LAUNCH(BNV)                                                                        \
  {                                                                                              \
    auto k = tc_gemm_kernel<BNV, gemm_stages<BNV>()>;                                             \
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,        \
                                         (int)smem);                                             \
    if (e != cudaSuccess) return e;                                                              \
    k<<<grid, 128, smem, s>>>(mapA, mapB, M, N, K, bias, relu, (const __nv_bfloat16*)mask, ldm, \
                              Cf, (__nv_bfloat16*)Cb, ldc, accumulate, err);                     \
  }
  if (bn == 32) GM_TC_LAUNCH(32)
  else if (bn == 64) GM_TC_LAUNCH(64)
  else if (bn == 128) GM_TC_LAUNCH(128)
  else GM_TC_LAUNCH(256)
#undef GM_TC_LAUNCH
  return cudaGetLastError();
}

}  // namespace gmcr
