// gm_convert.cu -- gm_convert: the library's FP32 <-> FP64 conversions on
// the integer pipe (f2d_exact, d2f_trunc of gm_common.cuh) applied to an
// array, so that they can be checked against the hardware conversions.
#include <string>

#include "gm_kernels.cuh"

namespace {

__global__ void convert_f2d_kernel(int64_t n, const float* in, double* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = gmcr::f2d_exact(in[i]);
}
__global__ void convert_d2f_kernel(int64_t n, const double* in, float* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = gmcr::d2f_trunc(in[i]);
}

}  // namespace

extern "C" int gm_convert(int32_t dir, int64_t n, const void* in, void* out, void* stream) {
  gmcr::record_error(GM_OK, "");
  if (n < 0 || (dir != 0 && dir != 1) || (n > 0 && (!in || !out)))
    return gmcr::record_error(GM_ERR_ARG, "gm_convert: dir must be 0 or 1, n >= 0, arrays non-null");
  if (n == 0) return GM_OK;
  int rc = gmcr::api_check_device();
  if (rc) return rc;
  const int64_t nb = (n + 255) / 256;
  const int g = (int)(nb < 4096 ? nb : 4096);
  if (dir == 0)
    convert_f2d_kernel<<<g, 256, 0, (cudaStream_t)stream>>>(n, (const float*)in, (double*)out);
  else
    convert_d2f_kernel<<<g, 256, 0, (cudaStream_t)stream>>>(n, (const double*)in, (float*)out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return gmcr::record_error(GM_ERR_CUDA, (std::string("gm_convert launch: ") + cudaGetErrorString(e)).c_str());
  return GM_OK;
}
