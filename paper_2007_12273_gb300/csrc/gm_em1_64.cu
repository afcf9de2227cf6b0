// gm_em1_64.cu -- the EM kernel for D = 1, 64 threads per cell.
#include "em_launch.cuh"

namespace gmcr {
GM_EM_NT_DEFINE(1, 64)
}  // namespace gmcr
