// gm_std.cu -- launcher of the standard-EM kernel (std_kernel.cuh): one
// persistent CTA of 256 threads per SM slot, cells pulled from a ticket.
#include "gm_kernels.cuh"
#include "std_kernel.cuh"

namespace gmcr {

template <int D, typename VT>
static cudaError_t std_go(const StdParams& p, size_t smem, int sms, cudaStream_t s) {
  auto k = std_kernel<D, 256, VT>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int64_t grid = (int64_t)per_sm * sms;
  if (grid > p.C) grid = p.C;
  k<<<(int)grid, 256, smem, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_std(int D, const StdParams& p, int v_f64, size_t smem, int sms, cudaStream_t s) {
  if (D == 1) return v_f64 ? std_go<1, double>(p, smem, sms, s) : std_go<1, float>(p, smem, sms, s);
  return v_f64 ? std_go<3, double>(p, smem, sms, s) : std_go<3, float>(p, smem, sms, s);
}

// Anderson iteration on the affine map G(x) = A x + b by one warp, with
// the same step as the standard EM kernel (a check of the extrapolation's
// arithmetic apart from the EM map)
constexpr int kAAMaxN = kMaxK * 10;
__global__ void __launch_bounds__(32) aa_affine_kernel(int n, const double* A, const double* b,
                                                       const double* x0, int m, int iters,
                                                       double* x_out, double* res_out) {
  __shared__ AAState<kAAMaxN> s;
  __shared__ double x[kAAMaxN];
  const int lane = threadIdx.x;
  if (lane == 0) {
    s.h = 0;
    s.have = 0;
  }
  for (int i = lane; i < n; i += 32) x[i] = x0[i];
  __syncwarp();
  for (int it = 0; it < iters; ++it) {
    double r = 0.0;
    for (int i = lane; i < n; i += 32) {
      double t = b[i];
      for (int j2 = 0; j2 < n; ++j2) t = __dadd_rn(t, __dmul_rn(A[(size_t)i * n + j2], x[j2]));
      s.th[i] = x[i];
      s.tg[i] = t;
      r += (t - x[i]) * (t - x[i]);
    }
    r = warp_sum(r);
    if (lane == 0) res_out[it] = sqrt(r);
    __syncwarp();
    const bool applied = aa_warp_step<kAAMaxN>(s, n, m);
    for (int i = lane; i < n; i += 32) x[i] = applied ? s.tn[i] : s.tg[i];
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) x_out[i] = x[i];
}

cudaError_t launch_aa_affine(int n, const double* A, const double* b, const double* x0, int m,
                             int iters, double* x_out, double* res_out, cudaStream_t s) {
  aa_affine_kernel<<<1, 32, 0, s>>>(n, A, b, x0, m, iters, x_out, res_out);
  return cudaGetLastError();
}

}  // namespace gmcr
