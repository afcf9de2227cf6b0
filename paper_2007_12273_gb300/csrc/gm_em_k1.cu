// gm_em_k1.cu -- launch of the closed-form pre-pass (em_k1.cuh: the sums
// kernel, then the finishing kernel) that fits the one-component, empty and
// degenerate cells of gm_compress_from before the EM kernel takes the rest.
#include "em_k1.cuh"
#include "gm_kernels.cuh"

namespace gmcr {

size_t em_k1_raw_bytes(int D, int64_t C) {
  return (size_t)C * (D == 1 ? sizeof(K1Raw<1>) : sizeof(K1Raw<3>));
}

cudaError_t launch_em_k1(int D, int v_f64, const K1Params& p, int sms, cudaStream_t s) {
  constexpr int NW = 4;  // cells (warps) per CTA
  const int64_t ncta = (p.C + NW - 1) / NW;
  const int g = (int)(ncta < (int64_t)sms * 16 ? ncta : (int64_t)sms * 16);
  if (g == 0) return cudaSuccess;
  const int64_t nf = (p.C + 255) / 256;
  const int gf = (int)(nf < 4096 ? nf : 4096);
  if (D == 1) {
    if (v_f64) em_k1_kernel<1, double, NW><<<g, NW * 32, 0, s>>>(p);
    else em_k1_kernel<1, float, NW><<<g, NW * 32, 0, s>>>(p);
    trace_mark("em_k1_kernel", s);
    if (v_f64) em_k1_finish_kernel<1, double><<<gf, 256, 0, s>>>(p);
    else em_k1_finish_kernel<1, float><<<gf, 256, 0, s>>>(p);
  } else {
    if (v_f64) em_k1_kernel<3, double, NW><<<g, NW * 32, 0, s>>>(p);
    else em_k1_kernel<3, float, NW><<<g, NW * 32, 0, s>>>(p);
    trace_mark("em_k1_kernel", s);
    if (v_f64) em_k1_finish_kernel<3, double><<<gf, 256, 0, s>>>(p);
    else em_k1_finish_kernel<3, float><<<gf, 256, 0, s>>>(p);
  }
  trace_mark("em_k1_finish_kernel", s);
  return cudaGetLastError();
}

}  // namespace gmcr
