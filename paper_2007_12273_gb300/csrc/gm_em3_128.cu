// gm_em3_128.cu -- the EM kernel for D = 3, 128 threads per cell.
#include "em_launch.cuh"

namespace gmcr {
GM_EM_NT_DEFINE(3, 128)
}  // namespace gmcr
