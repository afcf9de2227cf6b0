// em_launch.cuh -- launch and occupancy of one EM kernel instantiation
// (em_kernel<D, NT, VT, R>).  Each (D, NT) pair is compiled in a
// translation unit of its own (gm_em<D>_<NT>.cu) so that the library's
// heaviest kernels build in parallel; gm_em1.cu / gm_em3.cu dispatch.
#pragma once

#include "gm_kernels.cuh"

namespace gmcr {

template <int D, int NT, typename VT, typename R>
static cudaError_t em_go(const EmParams& p, size_t smem, int grid, cudaStream_t s) {
  auto k = em_kernel<D, NT, VT, R>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, NT, smem, s>>>(p);
  return cudaGetLastError();
}

template <int D, int NT, typename VT, typename R>
static int em_occ(size_t smem) {
  auto k = em_kernel<D, NT, VT, R>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, NT, smem) != cudaSuccess) return 0;
  return nb;
}

// one (D, NT): the four (velocity type, M-step precision) variants
template <int D, int NT>
struct EmNT {
  static cudaError_t launch(const EmParams& p, int fp64_mstep, int v_f64, size_t smem, int grid,
                            cudaStream_t s);
  static int occupancy(int fp64_mstep, int v_f64, size_t smem);
};

// the specialisations below are defined in gm_em<D>_<NT>.cu
#define GM_EM_NT_DECLARE(D, NT)                                                                   \
  template <>                                                                                   \
  cudaError_t EmNT<D, NT>::launch(const EmParams& p, int fp64_mstep, int v_f64, size_t smem,    \
                                  int grid, cudaStream_t s);                                    \
  template <>                                                                                   \
  int EmNT<D, NT>::occupancy(int fp64_mstep, int v_f64, size_t smem);
GM_EM_NT_DECLARE(1, 64)
GM_EM_NT_DECLARE(1, 128)
GM_EM_NT_DECLARE(1, 256)
GM_EM_NT_DECLARE(3, 64)
GM_EM_NT_DECLARE(3, 128)
GM_EM_NT_DECLARE(3, 256)

#define GM_EM_NT_DEFINE(D, NT)                                                                  \
  template <>                                                                                   \
  cudaError_t EmNT<D, NT>::launch(const EmParams& p, int fp64_mstep, int v_f64, size_t smem,    \
                                  int grid, cudaStream_t s) {                                   \
    if (v_f64)                                                                                  \
      return fp64_mstep ? em_go<D, NT, double, double>(p, smem, grid, s)                        \
                        : em_go<D, NT, double, float>(p, smem, grid, s);                        \
    return fp64_mstep ? em_go<D, NT, float, double>(p, smem, grid, s)                           \
                      : em_go<D, NT, float, float>(p, smem, grid, s);                           \
  }                                                                                             \
  template <>                                                                                   \
  int EmNT<D, NT>::occupancy(int fp64_mstep, int v_f64, size_t smem) {                          \
    if (v_f64) return fp64_mstep ? em_occ<D, NT, double, double>(smem) : em_occ<D, NT, double, float>(smem); \
    return fp64_mstep ? em_occ<D, NT, float, double>(smem) : em_occ<D, NT, float, float>(smem);  \
  }

}  // namespace gmcr
