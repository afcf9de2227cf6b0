// gm_em1.cu -- instantiations of the persistent EM kernel for D = 1.
#include "gm_kernels.cuh"

namespace gmcr {

template <int NT, typename VT, typename R>
static cudaError_t go(const EmParams& p, size_t smem, int grid, cudaStream_t s) {
  auto k = em_kernel<1, NT, VT, R>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, NT, smem, s>>>(p);
  return cudaGetLastError();
}

template <int NT, typename VT, typename R>
static int occ(size_t smem) {
  auto k = em_kernel<1, NT, VT, R>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, NT, smem) != cudaSuccess) return 0;
  return nb;
}

#define GM_EM_DISPATCH(FN, ...)                                                     \
  if (nt == 128) {                                                                  \
    if (v_f64) return fp64_mstep ? FN<128, double, double>(__VA_ARGS__)             \
                                 : FN<128, double, float>(__VA_ARGS__);             \
    return fp64_mstep ? FN<128, float, double>(__VA_ARGS__)                         \
                      : FN<128, float, float>(__VA_ARGS__);                         \
  }                                                                                 \
  if (v_f64) return fp64_mstep ? FN<256, double, double>(__VA_ARGS__)               \
                               : FN<256, double, float>(__VA_ARGS__);               \
  return fp64_mstep ? FN<256, float, double>(__VA_ARGS__) : FN<256, float, float>(__VA_ARGS__);

cudaError_t launch_em1(const EmParams& p, int nt, int fp64_mstep, int v_f64, size_t smem, int grid,
                       cudaStream_t s) {
  GM_EM_DISPATCH(go, p, smem, grid, s)
}

int em_blocks_per_sm_d1(int nt, int fp64_mstep, int v_f64, size_t smem) {
  GM_EM_DISPATCH(occ, smem)
}

}  // namespace gmcr
