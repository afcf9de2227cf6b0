// em_k1.cuh -- the cells whose fit is known in closed form before any EM
// sweep: empty and degenerate cells, and cells started from a supplied
// mixture (gm_compress_from) with exactly one valid component.  With K = 1
// every responsibility is the particle's weight, so one EM step from any
// start gives the weighted sample mean and covariance and the final
// unpenalised step (Sec. 2.3.1) returns them unchanged; eq. (lnL-GM) is then
// -(N/2)(D ln 2 pi + ln|Sigma| + D) - (T/2) ln N.
//
// Every other cell is appended to a work list that the persistent EM kernel
// takes its cells from.  The decisions and outputs are those of the EM
// kernel's own prologue for the same cell (moments in FP64 about the cell's
// first particle, the 1e-13 covariance floor, the validity test of the
// supplied component), so a cell's result does not depend on which kernel
// fitted it beyond the summation order of its FP64 moments.
//
// Two kernels.  em_k1_kernel, one warp per cell, reads the particles and
// writes the cell's moment sums to a per-cell record (exact 128-bit integer
// sums for an equal-weight cell, FP64 sums otherwise); em_k1_finish_kernel,
// one thread per cell, turns them into the mean, the covariance, the floor
// and validity tests and eq. (lnL-GM).  The per-cell FP64 work (a square
// root, reciprocals, logarithms, the pivots) thus runs 32 cells to a warp
// instruction: GB300 runs FP64 at 1/64 of the FP32 rate, and a warp-uniform
// FP64 instruction costs the pipe as much as a full one.
#pragma once

#include "deposit_cell.cuh"
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
// the 128-bit sums [sum d (D), sum d d^T (upper, NM)] of an equal-weight
// cell (n particles, velocities v[d * ldv + p], shift = the first particle)
// in units of 2^eq_d (2^(eq_x + eq_y) for the products), on the integer
// pipe, lane-parallel over particles; every lane returns them.  Returns
// false (nothing written) when a velocity is not finite.
template <int D>
__device__ bool fixed_sums(const float* __restrict__ v, int64_t ldv, int n, int lane,
                           __int128 (&s1)[D], __int128 (&s2)[D * (D + 1) / 2], int (&eq)[D]) {
  constexpr int NM = D * (D + 1) / 2;
  // the largest biased exponent per dimension
  int emax[D];
#pragma unroll
  for (int d = 0; d < D; ++d) emax[d] = 0;
#pragma unroll 4
  for (int p = lane; p < n; p += 32)
#pragma unroll
    for (int d = 0; d < D; ++d) emax[d] = max(emax[d], (int)((__float_as_uint(v[d * ldv + p]) >> 23) & 0xFFu));
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
#pragma unroll
  for (int d = 0; d < D; ++d) s1[d] = 0;
#pragma unroll
  for (int t = 0; t < NM; ++t) s2[t] = 0;
#pragma unroll 2
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
  return true;
}

// Per-cell record between the two kernels.  fixed = 1: the integer sums
// (sum t as (low, high) halves in words 2t, 2t+1; t < D the first moments,
// then the NM second moments), their exponents eq and the common weight a0;
// fixed = 0: the FP64 sums [sum alpha, sum alpha d (D), sum alpha d d^T] in
// words 0 .. NS-1.
template <int D>
struct alignas(16) K1Raw {
  double w[2 * (D + D * (D + 1) / 2)];
  double a0;
  int eq[D];
  int fixed;
};

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
  void* raw;                 // K1Raw<D> [C]
  // the charge deposit fused in (dep_rec = NULL: not done here): positions,
  // 1 / dx, shape order, per-cell records (deposit_cell.cuh)
  const double* x;
  double inv_dx;
  int order;
  long long* dep_rec;
  int Kmax;
};

// Pass 1, one warp per cell: cells with several (or no) supplied components
// go to the EM kernel's list; for the others the moment sums about the first
// particle go to the cell's K1Raw record, and the parameter slots past the
// first are cleared.
template <int D, typename VT, int NW>
__global__ void __launch_bounds__(NW * 32) em_k1_kernel(K1Params a) {
  constexpr int NM = D * (D + 1) / 2;
  constexpr int NS = 1 + D + NM;
  constexpr int NP = NS <= 4 ? 4 : 16;
  constexpr int P = 1 + D + NM;
  const int lane = threadIdx.x & 31;
  const VT* __restrict__ vin = static_cast<const VT*>(a.v);
  K1Raw<D>* raw = static_cast<K1Raw<D>*>(a.raw);
  for (int64_t j = ((int64_t)blockIdx.x * NW + (threadIdx.x >> 5)); j < a.C;
       j += (int64_t)gridDim.x * NW) {
    const int64_t off = a.cell_off[j];
    const int N = (int)(a.cell_off[j + 1] - off);
    const int K0 = a.init_K[j] < a.Kmax ? a.init_K[j] : a.Kmax;
    // the weights' bit-for-bit equality, shared by the deposit and the sums
    const bool same = N > 0 && N <= kFixMaxN && equal_weights(a.alpha, off, N, lane);
    if (a.dep_rec) deposit_cell(j, off, N, a.x, a.alpha, a.inv_dx, a.order, a.dep_rec + (size_t)j * kDepWords,
                                lane, same);
    if (K0 != 1 && N > 0) {  // several (or no) supplied components: EM
      if (lane == 0) a.list[atomicAdd(a.list_count, 1u)] = (unsigned int)j;
      continue;
    }
    // slots 1 .. Kmax-1 are zero in every closed-form result (a cell that
    // the finishing pass hands to EM is rewritten whole by the EM kernel)
    double* prm_out = a.params_out + (size_t)j * a.Kmax * P;
    for (int i = P + lane; i < a.Kmax * P; i += 32) prm_out[i] = 0.0;
    if (N == 0) continue;
    K1Raw<D>& r = raw[j];
    bool fixed = false;
    if constexpr (sizeof(VT) == 4) {
      // equal weights (bit for bit, positive) and at most 2^14 particles:
      // exact sums on the integer pipe
      if (same) {
        const long long a0b = __double_as_longlong(a.alpha[off]);
        // a0 > 0 on the bits: positive sign, not a NaN
        if (a0b > 0 && a0b <= 0x7FF0000000000000ll) {
          __int128 s1[D], s2[NM];
          int eq[D];
          fixed = fixed_sums<D>(reinterpret_cast<const float*>(vin) + off, a.n, N, lane, s1, s2, eq);
          if (fixed) {
            __int128 mine = 0;
#pragma unroll
            for (int t = 0; t < D; ++t)
              if (lane == t) mine = s1[t];
#pragma unroll
            for (int t = 0; t < NM; ++t)
              if (lane == D + t) mine = s2[t];
            if (lane < D + NM)
              *reinterpret_cast<longlong2*>(&r.w[2 * lane]) =
                  make_longlong2((long long)(unsigned long long)mine, (long long)(mine >> 64));
            if (lane == 0) {
              r.a0 = __longlong_as_double(a0b);
#pragma unroll
              for (int d = 0; d < D; ++d) r.eq[d] = eq[d];
              r.fixed = 1;
            }
          }
        }
      }
    }
    if (!fixed) {  // FP64 sums
      double sh[D];
#pragma unroll
      for (int d = 0; d < D; ++d) sh[d] = to_f64(vin[(int64_t)d * a.n + off]);
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
      double mine = 0.0;
#pragma unroll
      for (int q = 0; q < NS; ++q) {
        const double t = __shfl_sync(0xffffffffu, acc[0], warp_rs_lane<NP>(q));
        if (lane == q) mine = t;
      }
      if (lane < NS) r.w[lane] = mine;
      if (lane == 0) r.fixed = 0;
    }
  }
}

// Pass 2, one thread per cell: the closed-form result of every cell that
// pass 1 did not list, or its hand-over to the EM kernel's list.
template <int D, typename VT>
__global__ void em_k1_finish_kernel(K1Params a) {
  constexpr int NM = D * (D + 1) / 2;
  constexpr int NS = 1 + D + NM;
  constexpr int P = 1 + D + NM;
  constexpr int T = D * (D + 3) / 2;
  const VT* __restrict__ vin = static_cast<const VT*>(a.v);
  const K1Raw<D>* raw = static_cast<const K1Raw<D>*>(a.raw);
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < a.C;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t off = a.cell_off[j];
    const int N = (int)(a.cell_off[j + 1] - off);
    const int K0 = a.init_K[j] < a.Kmax ? a.init_K[j] : a.Kmax;
    if (K0 != 1 && N > 0) continue;  // listed by pass 1
    // ---- moments about the first particle ------------------------------
    double sh[D], res[NS];
#pragma unroll
    for (int d = 0; d < D; ++d) sh[d] = N > 0 ? to_f64(vin[(int64_t)d * a.n + off]) : 0.0;
#pragma unroll
    for (int q = 0; q < NS; ++q) res[q] = 0.0;
    if (N > 0) {
      const K1Raw<D>& r = raw[j];
      if (r.fixed) {
        const double a0 = r.a0;
        res[0] = (double)N * a0;
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const longlong2 h = *reinterpret_cast<const longlong2*>(&r.w[2 * d]);
          res[1 + d] = a0 * i128_to_f64(((__int128)h.y << 64) | (__int128)(unsigned long long)h.x, r.eq[d]);
        }
        int t = 0;
#pragma unroll
        for (int x = 0; x < D; ++x)
#pragma unroll
          for (int y = x; y < D; ++y, ++t) {
            const longlong2 h = *reinterpret_cast<const longlong2*>(&r.w[2 * (D + t)]);
            res[1 + D + t] =
                a0 * i128_to_f64(((__int128)h.y << 64) | (__int128)(unsigned long long)h.x, r.eq[x] + r.eq[y]);
          }
      } else {
#pragma unroll
        for (int q = 0; q < NS; ++q) res[q] = r.w[q];
      }
    }
    const double W = res[0];
    double* prm_out = a.params_out + (size_t)j * a.Kmax * P;
    const unsigned int too_few = (N <= 10) ? GM_ST_TOO_FEW : 0u;
    if (N == 0 || !(W > 0.0)) {  // empty cell
      for (int i = 0; i < P; ++i) prm_out[i] = 0.0;
      a.K_out[j] = 0;
      a.W_out[j] = N == 0 ? 0.0 : W;
      a.lnL_out[j] = 0.0;
      if (a.sweeps_out) a.sweeps_out[j] = 0;
      if (a.kwork_out) a.kwork_out[j] = 0;
      a.status_out[j] = N == 0 ? GM_ST_EMPTY : (GM_ST_EMPTY | GM_ST_DEGENERATE);
      continue;
    }
    // mean and covariance
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
    double det = 1.0;
    bool ok;
    {
      double scale2 = 0.0;
      for (int d = 0; d < D; ++d) scale2 += cov[tri<D>(d, d)] + mean[d] * mean[d];
      const double one[3] = {1.0, 1.0, 1.0};
      ok = ldl_floor<D>(cov, one, 1e-13 * scale2, det);
    }
    if (!ok) {  // degenerate: the cell's moments, flagged
      prm_out[0] = 1.0;
      for (int d = 0; d < D; ++d) prm_out[1 + d] = mean[d];
      for (int t = 0; t < NM; ++t) prm_out[1 + D + t] = cov[t];
      a.K_out[j] = 1;
      a.W_out[j] = W;
      a.lnL_out[j] = 0.0;
      if (a.sweeps_out) a.sweeps_out[j] = 0;
      if (a.kwork_out) a.kwork_out[j] = 0;
      a.status_out[j] = too_few | GM_ST_DEGENERATE | GM_ST_COV_NOT_PD;
      continue;
    }
    // ---- the supplied component: valid (weight > 0, Cholesky floor in
    // whitened coordinates, as chol_whitened) and not capped away by
    // N - T K / 2 > 0 ------------------------------------------------------
    double sc[D], isc[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      sc[d] = sqrt(cov[tri<D>(d, d)]);
      isc[d] = rcp_nr(sc[d]);
    }
    bool valid;
    {
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
    if (!valid) {  // no component left: the paper's initialisation, by EM
      a.list[atomicAdd(a.list_count, 1u)] = (unsigned int)j;
      continue;
    }
    // ---- closed form ---------------------------------------------------------
    const double logdet = log(det), logN = log((double)N);
    prm_out[0] = 1.0;
    for (int d = 0; d < D; ++d) prm_out[1 + d] = mean[d];
    for (int t = 0; t < NM; ++t) prm_out[1 + D + t] = cov[t];
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

}  // namespace gmcr
