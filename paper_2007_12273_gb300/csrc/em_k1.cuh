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

// The Cholesky floor test of a symmetric D x D matrix (upper triangle S),
// by its L~ diag(p) L~^T pivots p_i (the squared Cholesky diagonal, FP64,
// two reciprocals and no square root): every p_i sc2_i > fl and p_i <
// 1e300; on success det = prod p_i.  (sc2 = 1 for a matrix in original
// coordinates; the coordinate scales squared for a whitened one, as in
// chol_whitened.)
template <int D>
__device__ __forceinline__ bool ldl_floor(const double* S, const double* sc2, double fl, double& det) {
  const double p0 = S[0];
  if (!(p0 * sc2[0] > fl) || !(p0 < 1e300)) return false;
  if (D == 1) {
    det = p0;
    return true;
  }
  const double r0 = rcp_nr(p0);
  const double l10 = S[1] * r0, l20 = S[2] * r0;
  const double p1 = fma(-l10, S[1], S[3]);
  if (!(p1 * sc2[1] > fl) || !(p1 < 1e300)) return false;
  const double r1 = rcp_nr(p1);
  const double e12 = fma(-l20, S[1], S[4]);
  const double p2 = fma(-(e12 * r1), e12, fma(-l20, S[2], S[5]));
  if (!(p2 * sc2[D - 1] > fl) || !(p2 < 1e300)) return false;
  det = p0 * p1 * p2;
  return true;
}

// ---------------------------------------------------------------------------
// Moments of an equal-weight cell on the integer pipe (fixq and the 128-bit
// helpers are in gm_common.cuh).  With every weight
// equal to alpha_0 the sums are alpha_0 times sums of d = v - s (s the
// first particle), and the FP32 velocities are integers times a power of
// two: each is taken as v / 2^eq rounded to an integer with eq = (the
// cell's largest exponent in that dimension) + 1 - 54, which is exact for
// every velocity within 2^-30 of the largest and within 2^-55 of it
// otherwise.  The sums of d and of d_x d_y are then exact 128-bit integer
// sums (|d| < 2^55, d^2 < 2^110, at most 2^14 particles), converted to FP64
// once per cell -- no FP64 arithmetic per particle, where GB300's FP64 pipe
// (1/64 of the FP32 rate) bounds the FP64 sums.
// ---------------------------------------------------------------------------
// the FP64 sums [sum alpha, sum alpha d (D), sum alpha d d^T (upper, NM)] of
// an equal-weight cell (weight a0, n particles, velocities v[d * ldv + p],
// shift sh = v[., 0]) on the integer pipe, lane-parallel over particles;
// every lane returns them.  Returns false (nothing written) when a velocity
// is not finite.
template <int D>
__device__ bool fixed_moments(const float* __restrict__ v, int64_t ldv, int n, double a0, int lane,
                              double* res) {
  constexpr int NM = D * (D + 1) / 2;
  // the largest biased exponent per dimension
  int emax[D];
#pragma unroll
  for (int d = 0; d < D; ++d) emax[d] = 0;
  for (int p = lane; p < n; p += 32)
#pragma unroll
    for (int d = 0; d < D; ++d) emax[d] = max(emax[d], (int)((__float_as_uint(v[d * ldv + p]) >> 23) & 0xFFu));
  int eq[D];
  bool ok = true;
#pragma unroll
  for (int d = 0; d < D; ++d) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) emax[d] = max(emax[d], __shfl_xor_sync(0xffffffffu, emax[d], o));
    ok = ok && emax[d] < 255;
    eq[d] = (emax[d] ? emax[d] - 127 : -126) + 1 - kFixBits;
  }
  if (!ok) return false;
  long long s0[D];
#pragma unroll
  for (int d = 0; d < D; ++d) s0[d] = fixq(v[d * ldv], eq[d]);
  __int128 s1[D], s2[NM];
#pragma unroll
  for (int d = 0; d < D; ++d) s1[d] = 0;
#pragma unroll
  for (int t = 0; t < NM; ++t) s2[t] = 0;
  for (int p = lane; p < n; p += 32) {
    long long dq[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      dq[d] = fixq(v[d * ldv + p], eq[d]) - s0[d];
      s1[d] += (__int128)dq[d];
    }
    int t = 0;
#pragma unroll
    for (int x = 0; x < D; ++x)
#pragma unroll
      for (int y = x; y < D; ++y, ++t) s2[t] += (__int128)dq[x] * (__int128)dq[y];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int d = 0; d < D; ++d) s1[d] += shfl_xor_i128(s1[d], o);
#pragma unroll
    for (int t = 0; t < NM; ++t) s2[t] += shfl_xor_i128(s2[t], o);
  }
  res[0] = (double)n * a0;
#pragma unroll
  for (int d = 0; d < D; ++d) res[1 + d] = a0 * i128_to_f64(s1[d], eq[d]);
  int t = 0;
#pragma unroll
  for (int x = 0; x < D; ++x)
#pragma unroll
    for (int y = x; y < D; ++y, ++t) res[1 + D + t] = a0 * i128_to_f64(s2[t], eq[x] + eq[y]);
  return true;
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
    // ---- moments about the first particle ------------------------------
    double sh[D];
#pragma unroll
    for (int d = 0; d < D; ++d) sh[d] = N > 0 ? to_f64(vin[(int64_t)d * a.n + off]) : 0.0;
    double res[NS];
    bool fixed = false;
    if constexpr (sizeof(VT) == 4) {
      // equal weights (bit for bit) and at most 2^14 particles: exact sums
      // on the integer pipe
      if (N > 0 && N <= kFixMaxN) {
        const long long a0b = __double_as_longlong(a.alpha[off]);
        bool same = true;
        for (int p = lane; p < N; p += 32) same = same && (__double_as_longlong(a.alpha[off + p]) == a0b);
        if (__all_sync(0xffffffffu, same) && __longlong_as_double(a0b) > 0.0)
          fixed = fixed_moments<D>(reinterpret_cast<const float*>(vin) + off, a.n, N,
                                   __longlong_as_double(a0b), lane, res);
      }
    }
    if (!fixed) {  // FP64 sums
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
#pragma unroll
      for (int q = 0; q < NS; ++q) res[q] = __shfl_sync(0xffffffffu, acc[0], warp_rs_lane<NP>(q));
    }
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
    const double rW = rcp_nr(W);
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
    // and, on success, |Sigma| = the product of the pivots
    int ok = 1;
    double det = 1.0;
    if (lane == 0) {
      double scale2 = 0.0;
      for (int d = 0; d < D; ++d) scale2 += cov[tri<D>(d, d)] + mean[d] * mean[d];
      const double one[3] = {1.0, 1.0, 1.0};
      ok = ldl_floor<D>(cov, one, 1e-13 * scale2, det);
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    det = __shfl_sync(0xffffffffu, det, 0);
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
    // whitened coordinates, as chol_whitened) and not capped away by
    // N - T K / 2 > 0 ------------------------------------------------------
    double sc[D], isc[D];
    {
      // lane d < D takes coordinate d's scale (one sqrt and one reciprocal
      // for all D)
      double cdd = cov[0];
      if (D == 3) cdd = lane == 1 ? cov[tri<D>(1, 1)] : (lane == 2 ? cov[tri<D>(2, 2)] : cov[0]);
      const double s1 = sqrt(cdd), i1 = rcp_nr(s1);
#pragma unroll
      for (int d = 0; d < D; ++d) {
        sc[d] = __shfl_sync(0xffffffffu, s1, d);
        isc[d] = __shfl_sync(0xffffffffu, i1, d);
      }
    }
    int valid = 0;
    if (lane == 0) {
      const double* r = a.init_prm + (size_t)j * a.Kmax * P;
      double Sw[NM], sc2[3], scale2 = 0.0, dw;
      for (int d = 0; d < D; ++d) {
        const double m = mean[d] + sc[d] * ((r[1 + d] - mean[d]) * isc[d]);
        sc2[d] = sc[d] * sc[d];
        scale2 += sc2[d] * (r[1 + D + tri<D>(d, d)] * isc[d] * isc[d]) + m * m;
      }
      int q = 0;
      for (int x = 0; x < D; ++x)
        for (int yy = x; yy < D; ++yy, ++q) Sw[q] = r[1 + D + q] * isc[x] * isc[yy];
      valid = (r[0] > 0.0) && ldl_floor<D>(Sw, sc2, 1e-13 * scale2, dw);
    }
    valid = __shfl_sync(0xffffffffu, valid, 0);
    if (!valid) {  // no component left: the paper's initialisation, by EM
      if (lane == 0) a.list[atomicAdd(a.list_count, 1u)] = (unsigned int)j;
      continue;
    }
    // ln|Sigma| (lane 0) and ln N (lane 1) in one logarithm
    const double lg = log(lane == 1 ? (double)N : det);
    const double logdet = __shfl_sync(0xffffffffu, lg, 0), logN = __shfl_sync(0xffffffffu, lg, 1);
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
                     0.5 * (double)T * logN;
      if (a.sweeps_out) a.sweeps_out[j] = 1;
      if (a.kwork_out) a.kwork_out[j] = 0;
      a.status_out[j] = too_few;
    }
  }
}

}  // namespace gmcr
