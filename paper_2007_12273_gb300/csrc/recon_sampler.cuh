// recon_sampler.cuh -- the counter-based particle sampler of the
// reconstruction (Sec. 2.4, eq. mix-dist-1) and the Lemons projection
// coefficients (Sec. 2.4.2, eqs. alpha, beta), shared by the 1D and 2D
// meshes.  A particle is regenerated bit-identically from (seed, cell,
// index); FP64 is kept for the position and for the velocity's offset from
// the mixture mean, the categorical choice is decided on integers and the
// Gaussian draw is FP32.
#pragma once

#include "gm_kernels.cuh"

namespace gmcr {

// Cell j's output range [o, o + n) of the caller's particle arrays (n_out
// particles).  A range that does not lie inside [0, n_out) -- a negative
// count, or a start or an end outside the arrays -- is replaced by the empty
// range, and the function returns false: the cell is then treated as a cell
// without resampled particles and flagged GM_ST_BAD_RANGE, so that no kernel
// writes outside the caller's buffers.
__device__ __forceinline__ bool out_range(const int64_t* out_off, int64_t j, int64_t n_out,
                                          int64_t& o, int64_t& n) {
  o = out_off[j];
  n = out_off[j + 1] - o;
  if (o < 0 || n < 0 || o > n_out - n) {
    o = 0;
    n = 0;
    return false;
  }
  return true;
}
__device__ __forceinline__ int64_t out_count(const int64_t* out_off, int64_t j, int64_t n_out) {
  int64_t o, n;
  out_range(out_off, j, n_out, o, n);
  return n;
}

template <int D>
struct RecCell {
  static constexpr int NM = D * (D + 1) / 2;
  // categorical thresholds: u < cw_k  <=>  2 m + 1 < thr_k, where
  // u = (m + 1/2) 2^-52 and thr_k = ceil(cw_k 2^53) (cw_k the cumulative
  // weights summed in component order): the FP64 comparison, decided on
  // integers
  long long thr[kMaxK];
  double dz[kMaxK][D];      // mu_k - u
  float Lf[kMaxK][NM];      // lower-triangular Cholesky factor (FP32), row-major
  double u[D];              // mixture mean sum_k w_k mu_k
  double theta;             // sum_k w_k (tr Sigma_k + |mu_k - u|^2)
  double a, beta[D], alpha_new;
  int K;
  int skip;
  unsigned int status;
};

// FP32 lower-triangular Cholesky factor (row-major) of a component's
// covariance r[1 + D ..] (upper triangle), factored in FP64 with no floor: a
// non-positive pivot gives a zero column, as for a degenerate stored
// covariance
template <int D>
__device__ __forceinline__ void chol_f(const double* r, float* Lf) {
  if (D == 1) {
    const double s = r[2];
    Lf[0] = (float)(s > 0.0 ? sqrt(s) : 0.0);
  } else {
    // S upper: [s00 s01 s02 s11 s12 s22]
    const double s00 = r[4], s01 = r[5], s02 = r[6], s11 = r[7], s12 = r[8], s22 = r[9];
    const double l00 = s00 > 0.0 ? sqrt(s00) : 0.0;
    const double l10 = l00 > 0.0 ? s01 / l00 : 0.0;
    const double l20 = l00 > 0.0 ? s02 / l00 : 0.0;
    const double t11 = s11 - l10 * l10;
    const double l11 = t11 > 0.0 ? sqrt(t11) : 0.0;
    const double l21 = l11 > 0.0 ? (s12 - l20 * l10) / l11 : 0.0;
    const double t22 = s22 - l20 * l20 - l21 * l21;
    const double l22 = t22 > 0.0 ? sqrt(t22) : 0.0;
    Lf[0] = (float)l00; Lf[1] = (float)l10; Lf[2] = (float)l11;
    Lf[3] = (float)l20; Lf[4] = (float)l21; Lf[5] = (float)l22;
  }
}

// the mixture-wide quantities of a cell's Kj components rj (records of P
// values): the categorical thresholds (put_thr(k, t)), dz_k = mu_k - u
// (put_dz(k, d, value)), the mean u and the spread theta
template <int D, class PutThr, class PutDz>
__device__ __forceinline__ void mix_head(const double* rj, int Kj, PutThr put_thr, PutDz put_dz,
                                         double* u_out, double& theta) {
  constexpr int P = 1 + D + D * (D + 1) / 2;
  double cum = 0.0, u[D], th = 0.0;
  for (int d = 0; d < D; ++d) u[d] = 0.0;
  for (int q = 0; q < Kj; ++q) {
    const double* r = rj + (size_t)q * P;
    cum += r[0];
    const double t = ceil(cum * 9007199254740992.0);  // 2^53
    put_thr(q, t < 4.0e18 ? (long long)t : 4000000000000000000ll);
    for (int d = 0; d < D; ++d) u[d] += r[0] * r[1 + d];
  }
  for (int q = 0; q < Kj; ++q) {
    const double* r = rj + (size_t)q * P;
    double tr = 0.0, dd = 0.0;
    int t = 1 + D;
    for (int x = 0; x < D; ++x)
      for (int y = x; y < D; ++y, ++t) {
        if (x == y) tr += r[t];
      }
    for (int d = 0; d < D; ++d) {
      put_dz(q, d, r[1 + d] - u[d]);
      dd += (r[1 + d] - u[d]) * (r[1 + d] - u[d]);
    }
    th += r[0] * (tr + dd);
  }
  for (int d = 0; d < D; ++d) u_out[d] = u[d];
  theta = th;
}

// load cell j's mixture into the warp's RecCell: Cholesky factors on lanes
// k < K, the rest on lane 0
template <int D>
__device__ void load_cell(RecCell<D>& rc, int64_t j, int Kmax, const int32_t* K,
                          const double* prm, int lane) {
  constexpr int P = 1 + D + D * (D + 1) / 2;
  const int Kj = K[j];
  const double* rj = prm + (size_t)j * Kmax * P;
  if (lane < Kj) chol_f<D>(rj + (size_t)lane * P, rc.Lf[lane]);
  if (lane == 0) {
    rc.K = Kj;
    mix_head<D>(
        rj, Kj, [&](int q, long long t) { rc.thr[q] = t; },
        [&](int q, int d, double x) { rc.dz[q][d] = x; }, rc.u, rc.theta);
  }
}

// The same mixture data computed once per cell, by one thread per cell (the
// FP64 square roots and divisions then run 32 cells to a warp instruction),
// and kept in the workspace for the two particle passes: per cell a head
// (u, theta, K) and Kmax component records (threshold, dz, FP32 factor).
template <int D>
struct RecHead {
  double u[D];
  double theta;
  int K;
  int pad;
};
template <int D>
struct RecComp {
  long long thr;
  double dz[D];
  float Lf[D * (D + 1) / 2];
};
template <int D>
__device__ __forceinline__ void prep_cell(int64_t j, int Kmax, const int32_t* K, const double* prm,
                                          RecHead<D>* head, RecComp<D>* comp) {
  constexpr int P = 1 + D + D * (D + 1) / 2;
  const int Kj = K[j];
  const double* rj = prm + (size_t)j * Kmax * P;
  RecComp<D>* cj = comp + (size_t)j * Kmax;
  RecHead<D> h;
  mix_head<D>(
      rj, Kj, [&](int q, long long t) { cj[q].thr = t; },
      [&](int q, int d, double x) { cj[q].dz[d] = x; }, h.u, h.theta);
  h.K = Kj;
  h.pad = 0;
  head[j] = h;
  for (int q = 0; q < Kj; ++q) {
    float Lf[D * (D + 1) / 2];
    chol_f<D>(rj + (size_t)q * P, Lf);
    for (int m = 0; m < D * (D + 1) / 2; ++m) cj[q].Lf[m] = Lf[m];
  }
}
// copy cell j's prepared mixture into the warp's RecCell (lanes k < K copy
// component k, lane 0 the head)
template <int D>
__device__ __forceinline__ void load_prepped(RecCell<D>& rc, int64_t j, int Kmax,
                                             const RecHead<D>* head, const RecComp<D>* comp,
                                             int lane) {
  constexpr int NM = D * (D + 1) / 2;
  const int Kj = head[j].K;
  if (lane < Kj) {
    const RecComp<D>& c = comp[(size_t)j * Kmax + lane];
    rc.thr[lane] = c.thr;
#pragma unroll
    for (int d = 0; d < D; ++d) rc.dz[lane][d] = c.dz[d];
#pragma unroll
    for (int m = 0; m < NM; ++m) rc.Lf[lane][m] = c.Lf[m];
  }
  if (lane == 0) {
    const RecHead<D>& h = head[j];
    rc.K = Kj;
#pragma unroll
    for (int d = 0; d < D; ++d) rc.u[d] = h.u[d];
    rc.theta = h.theta;
  }
}

// the 52 leading bits of (hi, lo), as uniform52 uses them
__device__ __forceinline__ uint64_t bits52(uint32_t hi, uint32_t lo) {
  return ((uint64_t)hi << 20) | (uint64_t)(lo >> 12);
}
// (t + 1/2) 2^-52 in FP32 (relative error ~2^-24) for a 52-bit t, without
// FP64 arithmetic: t = hi26 2^26 + lo26
__device__ __forceinline__ float half_ulp52_f(uint64_t t) {
  const float hi = (float)(uint32_t)(t >> 26), lo = (float)(uint32_t)(t & 0x3FFFFFFull);
  return fmaf(hi, 1.4901161193847656e-08f /* 2^-26 */, (lo + 0.5f) * 2.220446049250313e-16f);
}
// Box-Muller radius sqrt(-2 ln u) for u = (m + 1/2) 2^-52, in FP32 from the
// integer: below 1/2, ln u; above, log1p(-(1 - u)) with 1 - u =
// (2^52 - 1 - m + 1/2) 2^-52 formed exactly on integers, so the radius
// keeps FP32 relative accuracy where its derivative is unbounded
__device__ __forceinline__ float bm_radius(uint64_t m) {
  const float lnu = m < (1ull << 51) ? logf(half_ulp52_f(m))
                                     : log1pf(-half_ulp52_f((1ull << 52) - 1ull - m));
  return sqrtf(-2.0f * lnu);
}

// (w + 1/2) 2^-32 in FP32 (relative error ~2^-24) for a 32-bit w
__device__ __forceinline__ float half_ulp32_f(uint32_t w) {
  return fmaf((float)w, 2.3283064365386963e-10f /* 2^-32 */, 1.1641532182693481e-10f /* 2^-33 */);
}
// the same radius for a 32-bit uniform (w + 1/2) 2^-32
__device__ __forceinline__ float bm_radius32(uint32_t w) {
  const float lnu = w < 0x80000000u ? logf(half_ulp32_f(w)) : log1pf(-half_ulp32_f(0xFFFFFFFFu - w));
  return sqrtf(-2.0f * lnu);
}

// particle i of cell j (Sec. 2.4, eq. mix-dist-1): the 52-bit integer m0
// of its position's uniform u0 = (m0 + 1/2) 2^-52 (x = (j + u0) dx), its
// component z (the categorical draw) and f = L_z xi (FP32), so that
// w = v - u = (mu_z - u) + f
template <int D>
__device__ __forceinline__ void sample_f(const RecCell<D>& rc, int64_t j, int64_t i, uint64_t seed,
                                         uint64_t& m0, int& z, float (&f)[D]) {
  const u32x4 r0 = philox_draw(seed, (uint32_t)i, kTagSample | 0u, j);
  m0 = bits52(r0.x, r0.y);
  const int K = rc.K;
  z = K - 1;  // the only choice when K <= 1
  if (K > 1) {
    const long long m1x2 = 2 * (long long)bits52(r0.z, r0.w) + 1;
    for (int k = 0; k < K; ++k)
      if (m1x2 < rc.thr[k]) { z = k; break; }
  }
  // Box-Muller (Box & Muller 1958) on block 1: for D = 1 one (radius,
  // angle) pair of 52-bit uniforms, for D = 3 two pairs of 32-bit uniforms
  // (words x, y and z, w), so that a 3V particle takes two Philox blocks
  float xi[3];
  const u32x4 r1 = philox_draw(seed, (uint32_t)i, kTagSample | 1u, j);
  if (D == 1) {
    const float rr = bm_radius(bits52(r1.x, r1.y));
    xi[0] = rr * cospif(2.0f * half_ulp52_f(bits52(r1.z, r1.w)));
  } else {
    const float rr = bm_radius32(r1.x);
    float sn, cs;
    sincospif(2.0f * half_ulp32_f(r1.y), &sn, &cs);
    xi[0] = rr * cs;
    xi[1] = rr * sn;
    xi[2] = bm_radius32(r1.z) * cospif(2.0f * half_ulp32_f(r1.w));
  }
  if (K == 0) {
    for (int d = 0; d < D; ++d) f[d] = 0.0f;
    return;
  }
  const float* L = rc.Lf[z];
  if (D == 1) {
    f[0] = L[0] * xi[0];
  } else {
    f[0] = L[0] * xi[0];
    f[1] = fmaf(L[2], xi[1], L[1] * xi[0]);
    f[2] = fmaf(L[5], xi[2], fmaf(L[4], xi[1], L[3] * xi[0]));
  }
}

// the particle's w = v - u in FP64 from its draw (z, f): (mu_z - u) + f
// (w = -u for a cell without a mixture)
template <int D>
__device__ __forceinline__ void draw_offset(const RecCell<D>& rc, int z, const float (&f)[D],
                                            double (&w)[D]) {
  if (rc.K == 0) {
    for (int d = 0; d < D; ++d) w[d] = -rc.u[d];
    return;
  }
#pragma unroll
  for (int d = 0; d < D; ++d) w[d] = rc.dz[z][d] + f2d_exact(f[d]);
}
// the same, drawing the particle
template <int D>
__device__ __forceinline__ void sample_particle(const RecCell<D>& rc, int64_t j, int64_t i,
                                                uint64_t seed, uint64_t& m0, double (&w)[D]) {
  int z;
  float f[D];
  sample_f<D>(rc, j, i, seed, m0, z, f);
  draw_offset<D>(rc, z, f, w);
}

// the 52 leading bits of the y uniform of particle i of cell j on a 2D mesh
// (Philox block 3, words 0-1)
__device__ __forceinline__ uint64_t sample_y_bits(int64_t j, int64_t i, uint64_t seed) {
  const u32x4 r3 = philox_draw(seed, (uint32_t)i, kTagSample | 3u, j);
  return bits52(r3.x, r3.y);
}

// (m + 1/2) 2^-52 - 1/2, the in-cell offset of a position from the cell
// centre in cell units (exact in FP64)
__device__ __forceinline__ double centred52(uint64_t m) {
  // ((m - 2^51) + 1/2) 2^-52 = (2 m - 2^52 + 1) 2^-53, built on the integer pipe
  return m >= (1ull << 51) ? odd_2m53(2ull * m - (1ull << 52) + 1ull, false)
                           : odd_2m53((1ull << 52) - 2ull * m - 1ull, true);
}
// the position uniform u0 = (m + 1/2) 2^-52 = (2 m + 1) 2^-53 of a 52-bit m
__device__ __forceinline__ double uniform_pos52(uint64_t m) { return odd_2m53(2ull * m + 1ull, false); }
// j + u0 rounded to the nearest double (ties to even), as the FP64 addition
// (double)j + u0 gives it, on the integer pipe, for 0 <= j < 2^52: with L
// the leading bit of j the sum's 53-bit significand in units of 2^(L - 52)
// is j 2^(52 - L) + t / 2^(L + 1), t = 2 m + 1; the fraction t mod 2^(L+1)
// decides the rounding, and a carry to 2^53 moves the exponent up by one
__device__ __forceinline__ double cell_plus_u0(uint64_t j, uint64_t m) {
  const unsigned long long t = 2ull * m + 1ull;
  if (j == 0) return odd_2m53(t, false);
  const int L = 63 - __clzll((long long)j);
  unsigned long long M = (j << (52 - L)) + (t >> (L + 1));
  const unsigned long long rem = t & ((2ull << L) - 1ull), half = 1ull << L;
  M += (rem > half || (rem == half && (M & 1ull))) ? 1ull : 0ull;
  const int e = M >> 53 ? L + 1 : L;
  M = M >> 53 ? (1ull << 52) : M;
  return __longlong_as_double((long long)(((unsigned long long)(1023 + e) << 52) | (M & ((1ull << 52) - 1ull))));
}

// Lemons projection of a cell with n resampled particles: the corrected
// weight alpha' = W_j / n + dA_j and, from the sums sw[d] = sum_p w_d and
// sw[D] = sum_p |w|^2 (w = v - u), the scale a and shift beta of eqs.
// (alpha), (beta) in the frame of the mixture mean u:
// 2 E N' - p^2 = W (N' theta + (N' - W) |u|^2),
// 2 E' N' - p'^2 = alpha'^2 (n sum|w|^2 - |sum w|^2).
template <int D>
struct ProjCoef {
  double a, beta[D], alpha_new;
  int skip;
  unsigned int status;
};
template <int D>
__device__ __forceinline__ ProjCoef<D> proj_coeffs(int K, const double* u, double theta, int64_t n,
                                                   double Wj, double dAj, const double* sw) {
  ProjCoef<D> pc;
  unsigned int st = 0;
  if (n == 0) st |= GM_ST_MM_EMPTY_COL;
  const double an = (n > 0 ? Wj / (double)n : 0.0) + dAj;
  pc.alpha_new = an;
  if (n > 0 && !(an > 0.0)) st |= GM_ST_NEG_WEIGHT;
  pc.skip = 1;
  pc.a = 1.0;
  for (int d = 0; d < D; ++d) pc.beta[d] = 0.0;
  if (n > 0 && K == 0) st |= GM_ST_NO_MIXTURE;
  if (n > 0 && K > 0) {
    const double Np = (double)n * an;
    double u2 = 0.0, sw2 = 0.0;
    for (int d = 0; d < D; ++d) {
      u2 += u[d] * u[d];
      sw2 += sw[d] * sw[d];
    }
    const double num = Wj * (Np * theta + (Np - Wj) * u2);
    const double den = an * an * ((double)n * sw[D] - sw2);
    if (num > 0.0 && den > 0.0 && Np > 0.0) {
      const double aa = sqrt(num / den);
      pc.a = aa;
      for (int d = 0; d < D; ++d) pc.beta[d] = ((Wj - Np) * u[d] - aa * an * sw[d]) / (aa * Np);
      pc.skip = 0;
    } else {
      st |= GM_ST_PROJ_SKIPPED;
    }
  }
  pc.status = st;
  return pc;
}
// the same on the warp's RecCell (lane 0); returns the status
template <int D>
__device__ unsigned int projection_coeffs(RecCell<D>& rc, int64_t n, double Wj, double dAj,
                                          const double* sw) {
  const ProjCoef<D> pc = proj_coeffs<D>(rc.K, rc.u, rc.theta, n, Wj, dAj, sw);
  rc.alpha_new = pc.alpha_new;
  rc.a = pc.a;
  for (int d = 0; d < D; ++d) rc.beta[d] = pc.beta[d];
  rc.skip = pc.skip;
  rc.status = pc.status;
  return pc.status;
}

}  // namespace gmcr
