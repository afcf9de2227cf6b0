// gm_em1_128.cu -- the EM kernel for D = 1, 128 threads per cell.
#include "em_launch.cuh"

namespace gmcr {
GM_EM_NT_DEFINE(1, 128)
}  // namespace gmcr
