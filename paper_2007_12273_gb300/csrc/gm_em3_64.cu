// gm_em3_64.cu -- the EM kernel for D = 3, 64 threads per cell.
#include "em_launch.cuh"

namespace gmcr {
GM_EM_NT_DEFINE(3, 64)
}  // namespace gmcr
