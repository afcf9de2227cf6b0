// gm_em1.cu -- dispatch of the persistent EM kernel for D = 1 over the
// CTA sizes (each compiled in gm_em1_<NT>.cu).
#include "em_launch.cuh"

namespace gmcr {

cudaError_t launch_em1(const EmParams& p, int nt, int fp64_mstep, int v_f64, size_t smem, int grid,
                       cudaStream_t s) {
  if (nt == 64) return EmNT<1, 64>::launch(p, fp64_mstep, v_f64, smem, grid, s);
  if (nt == 128) return EmNT<1, 128>::launch(p, fp64_mstep, v_f64, smem, grid, s);
  return EmNT<1, 256>::launch(p, fp64_mstep, v_f64, smem, grid, s);
}

int em_blocks_per_sm_d1(int nt, int fp64_mstep, int v_f64, size_t smem) {
  if (nt == 64) return EmNT<1, 64>::occupancy(fp64_mstep, v_f64, smem);
  if (nt == 128) return EmNT<1, 128>::occupancy(fp64_mstep, v_f64, smem);
  return EmNT<1, 256>::occupancy(fp64_mstep, v_f64, smem);
}

}  // namespace gmcr
