// gm_mlp.cu -- C ABI of the learned-initialisation network: the BF16
// tensor-core GEMM and the network's forward / backward / update steps.
#include <string>

#include "gm_kernels.cuh"

extern "C" {

int gm_gemm_bf16(int32_t M, int32_t N, int32_t K, const void* A, int32_t lda, const void* B,
                 int32_t ldb, const float* bias, int32_t relu, const void* mask, int32_t ldm,
                 float* C_f32, void* C_bf16, int32_t ldc, uint32_t* err, void* stream) {
  gmcr::record_error(GM_OK, "");
  if (M < 0 || N < 0 || K < 0) return gmcr::record_error(GM_ERR_ARG, "negative GEMM size");
  if (M == 0 || N == 0 || K == 0) return GM_OK;
  if (!A || !B || (!C_f32 && !C_bf16)) return gmcr::record_error(GM_ERR_ARG, "a GEMM pointer is NULL");
  if (lda < K || ldb < K || (lda & 7) || (ldb & 7) || ldc < N)
    return gmcr::record_error(GM_ERR_ARG, "GEMM leading dimensions: lda, ldb >= K and multiples of 8; ldc >= N");
  if ((((uintptr_t)A) & 15) || (((uintptr_t)B) & 15))
    return gmcr::record_error(GM_ERR_ARG, "GEMM operands must be 16-byte aligned");
  int dev = 0, major = 0, minor = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (major != 10 || minor != 3)
    return gmcr::record_error(GM_ERR_UNSUPPORTED, "this library is built for sm_103a");
  cudaError_t e = gmcr::launch_tc_gemm(A, B, M, N, K, lda, ldb, bias, relu, mask, ldm, C_f32,
                                       C_bf16, ldc, err, (cudaStream_t)stream);
  if (e != cudaSuccess)
    return gmcr::record_error(GM_ERR_CUDA, (std::string("GEMM launch: ") + cudaGetErrorString(e)).c_str());
  return GM_OK;
}

}  // extern "C"
