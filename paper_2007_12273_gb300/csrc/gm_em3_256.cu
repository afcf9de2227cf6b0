// gm_em3_256.cu -- the EM kernel for D = 3, 256 threads per cell.
#include "em_launch.cuh"

namespace gmcr {
GM_EM_NT_DEFINE(3, 256)
}  // namespace gmcr
