// em_k1.cuh -- one warp per cell for the cells whose fit is known in closed
// form before any EM sweep: empty and degenerate cells, and cells started
// from a supplied mixture (gm_compress_from) with exactly one valid
// component.  With K = 1 every responsibility is the particle's weight, so
// one EM step from any start gives the weighted sample mean and covariance
// and the final unpenalised step (Sec. 2.3.1) returns them unchanged; eq.
// (lnL-GM) is then -(N/2)(D ln 2 pi + ln|Sigma| + D) - (T/2) ln N.
//
// Every other cell is appended to a work list that the persistent EM kernel
// takes its cells from.  The decisions and outputs are those of the EM
// kernel's own prologue for the same cell (moments in FP64 about the cell's
// first particle, the 1e-13 covariance floor, the validity test of the
// supplied component), so a cell's result does not depend on which kernel
// fitted it beyond the summation order of its FP64 moments.
//
// A warp per cell instead of a CTA: no CTA barriers, and the per-cell FP64
// work (GB300 runs FP64 at 1/64 of the FP32 rate) spread over the lanes --
// the particle sums lane-parallel, the moments reduced by recursive halving
// (one FP64 add per shuffle), the three coordinate scales on three lanes.
#pragma once

#include "em_kernel.cuh"

namespace gmcr {

// first lane holding the total of value q after warp_rs_d<NP>
template <int NP>
__device__ __forceinline__ int warp_rs_lane(int q) {
  int l = 0;
#pragma unroll
  for (int lv = 0; (NP >> lv) > 1; ++lv)
    if (q & (NP >> (lv + 1))) l |= 16 >> lv;
  return l;
}

struct K1Params {
  int64_t C, n;
  const int64_t* cell_off;
  const void* v;
  const double* alpha;
  const int32_t* init_K;
  const double* init_prm;
  int32_t* K_out;
  double* params_out;
  double* W_out;
  double* lnL_out;
  int32_t* sweeps_out;
  int32_t* kwork_out;
  uint32_t* status_out;
  unsigned int* list;        // cells left to the EM kernel
  unsigned int* list_count;  // their number (zeroed before the launch)
  int Kmax;
};

template <int D, typename VT, int NW>
__global__ void __launch_bounds__(NW * 32) em_k1_kernel(K1Params a) {
  constexpr int NM = D * (D + 1) / 2;
  constexpr int NS = 1 + D + NM;
  constexpr int NP = NS <= 4 ? 4 : 16;
  constexpr int P = 1 + D + NM;
  constexpr int T = D * (D + 3) / 2;
  const int lane = threadIdx.x & 31;
  const VT* __restrict__ vin = static_cast<const VT*>(a.v);
  for (int64_t j = ((int64_t)blockIdx.x * NW + (threadIdx.x >> 5)); j < a.C;
       j += (int64_t)gridDim.x * NW) {
    const int64_t off = a.cell_off[j];
    const int N = (int)(a.cell_off[j + 1] - off);
    const int K0 = a.init_K[j] < a.Kmax ? a.init_K[j] : a.Kmax;
    if (K0 != 1 && N > 0) {  // several (or no) supplied components: EM
      if (lane == 0) a.list[atomicAdd(a.list_count, 1u)] = (unsigned int)j;
      continue;
    }
    // ---- moments about the first particle (FP64) -------------------------
    double sh[D];
#pragma unroll
    for (int d = 0; d < D; ++d) sh[d] = N > 0 ? to_f64(vin[(int64_t)d * a.n + off]) : 0.0;
    double acc[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) acc[i] = 0.0;
    for (int p = lane; p < N; p += 32) {
      const double al = a.alpha[off + p];
      double dv[D];
#pragma unroll
      for (int d = 0; d < D; ++d) dv[d] = to_f64(vin[(int64_t)d * a.n + off + p]) - sh[d];
      acc[0] += al;
      int t = 1 + D;
#pragma unroll
      for (int x = 0; x < D; ++x) {
        const double ad = al * dv[x];
        acc[1 + x] += ad;
#pragma unroll
        for (int y = x; y < D; ++y, ++t) acc[t] = fma(ad, dv[y], acc[t]);
      }
    }
    warp_rs_d<NP>(acc, lane);
    double res[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) res[q] = __shfl_sync(0xffffffffu, acc[0], warp_rs_lane<NP>(q));
    const double W = res[0];
    double* prm_out = a.params_out + (size_t)j * a.Kmax * P;
    const unsigned int too_few = (N <= 10) ? GM_ST_TOO_FEW : 0u;
    if (N == 0 || !(W > 0.0)) {  // empty cell
      for (int i = lane; i < a.Kmax * P; i += 32) prm_out[i] = 0.0;
      if (lane == 0) {
        a.K_out[j] = 0;
        a.W_out[j] = N == 0 ? 0.0 : W;
        a.lnL_out[j] = 0.0;
        if (a.sweeps_out) a.sweeps_out[j] = 0;
        if (a.kwork_out) a.kwork_out[j] = 0;
        a.status_out[j] = N == 0 ? GM_ST_EMPTY : (GM_ST_EMPTY | GM_ST_DEGENERATE);
      }
      continue;
    }
    // mean and covariance (every lane: the values are warp-uniform)
    const double rW = 1.0 / W;
    double mean[D], dm[D], cov[NM];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      dm[d] = res[1 + d] * rW;
      mean[d] = sh[d] + dm[d];
    }
    {
      int t = 0;
#pragma unroll
      for (int x = 0; x < D; ++x)
#pragma unroll
        for (int y = x; y < D; ++y, ++t) cov[t] = fma(-dm[x], dm[y], res[1 + D + t] * rW);
    }
    // the covariance floor 1e-13 sum_d (cov_dd + mean_d^2) (degenerate cell)
    // and, on success, ln|Sigma| = sum of the pivots' logs
    int ok = 1;
    double logdet = 0.0;
    if (lane == 0) {
      double scale2 = 0.0;
      for (int d = 0; d < D; ++d) scale2 += cov[tri<D>(d, d)] + mean[d] * mean[d];
      const double fl = 1e-13 * scale2;
      double L2[3][3] = {{0}};
      double piv = 1.0;
      for (int x = 0; x < D && ok; ++x)
        for (int y = 0; y <= x && ok; ++y) {
          double sv = cov[tri<D>(y, x)];
          for (int m = 0; m < y; ++m) sv -= L2[x][m] * L2[y][m];
          if (x == y) {
            if (!(sv > fl) || !(sv < 1e300)) {
              ok = 0;
            } else {
              L2[x][x] = sqrt(sv);
              piv *= sv;
            }
          } else {
            L2[x][y] = sv / L2[y][y];
          }
        }
      if (ok) logdet = log(piv);
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) {  // degenerate: the cell's moments, flagged
      for (int i = lane; i < a.Kmax * P; i += 32) {
        double val = 0.0;
        if (i == 0) val = 1.0;
        else if (i < 1 + D) val = mean[i - 1];
        else if (i < P) val = cov[i - 1 - D];
        prm_out[i] = val;
      }
      if (lane == 0) {
        a.K_out[j] = 1;
        a.W_out[j] = W;
        a.lnL_out[j] = 0.0;
        if (a.sweeps_out) a.sweeps_out[j] = 0;
        if (a.kwork_out) a.kwork_out[j] = 0;
        a.status_out[j] = too_few | GM_ST_DEGENERATE | GM_ST_COV_NOT_PD;
      }
      continue;
    }
    // ---- the supplied component: valid (weight > 0, Cholesky floor in
    // whitened coordinates) and not capped away by N - T K / 2 > 0 --------
    double sc[D], isc[D];
    {
      // lane d < D takes coordinate d's scale (one sqrt and one division
      // for all D)
      double cdd = cov[0];
      if (D == 3) cdd = lane == 1 ? cov[tri<D>(1, 1)] : (lane == 2 ? cov[tri<D>(2, 2)] : cov[0]);
      const double s1 = sqrt(cdd), i1 = 1.0 / s1;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        sc[d] = __shfl_sync(0xffffffffu, s1, d);
        isc[d] = __shfl_sync(0xffffffffu, i1, d);
      }
    }
    int valid = 0;
    if (lane == 0) {
      const double* r = a.init_prm + (size_t)j * a.Kmax * P;
      double mw[D], Sw[NM], Lw[3][3], rw[3];
      for (int d = 0; d < D; ++d) mw[d] = (r[1 + d] - mean[d]) * isc[d];
      int q = 0;
      for (int x = 0; x < D; ++x)
        for (int yy = x; yy < D; ++yy, ++q) Sw[q] = r[1 + D + q] * isc[x] * isc[yy];
      valid = (r[0] > 0.0) && chol_whitened<D, double, double>(Sw, mw, mean, sc, Lw, rw);
    }
    valid = __shfl_sync(0xffffffffu, valid, 0);
    if (!valid) {  // no component left: the paper's initialisation, by EM
      if (lane == 0) a.list[atomicAdd(a.list_count, 1u)] = (unsigned int)j;
      continue;
    }
    // ---- closed form ---------------------------------------------------------
    for (int i = lane; i < a.Kmax * P; i += 32) {
      double val = 0.0;
      if (i == 0) val = 1.0;
      else if (i < 1 + D) val = mean[i - 1];
      else if (i < P) val = cov[i - 1 - D];
      prm_out[i] = val;
    }
    if (lane == 0) {
      const double Nd = (double)N;
      a.K_out[j] = 1;
      a.W_out[j] = W;
      a.lnL_out[j] = -0.5 * Nd * ((double)D * 1.8378770664093454836 + logdet + (double)D) -
                     0.5 * (double)T * log(Nd);
      if (a.sweeps_out) a.sweeps_out[j] = 1;
      if (a.kwork_out) a.kwork_out[j] = 0;
      a.status_out[j] = too_few;
    }
  }
}

}  // namespace gmcr
