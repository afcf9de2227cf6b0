// gm_em1_256.cu -- the EM kernel for D = 1, 256 threads per cell.
#include "em_launch.cuh"

namespace gmcr {
GM_EM_NT_DEFINE(1, 256)
}  // namespace gmcr
