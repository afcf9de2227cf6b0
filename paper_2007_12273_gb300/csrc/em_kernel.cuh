// em_kernel.cuh -- persistent per-cell adaptive EM (compression, Sec. 2.2-2.3)
//
// One CTA fits one cell at a time and pulls the next cell from an atomic
// ticket.  A cell's particles are staged once (whitened FP32 velocities and
// normalised weights) in shared memory -- or, when the cell is larger than
// the shared tile, in an L2-resident global scratch with the same layout --
// and reused by every sweep.  Each thread works on pairs of particles with
// Blackwell's packed FP32 (f32x2) arithmetic.
//
// Component-wise EM (Sec. 2.3, Celeux et al.): the E-step of component k
// needs the normaliser s_p = sum_j omega_j f_j(v_p) with the *current*
// parameters of every component.  s_p is kept per particle (FP32, relative
// to a per-particle log2 shift m_p): a pass for component k first replaces
// the previous component's old term by its updated one, then evaluates
// f_k, the responsibility gamma_pk = alpha_p omega_k f_k / s_p and the
// per-thread FP32 sufficient statistics of component k about its old mean.
// Once per sweep an exact pass recomputes s_p and m_p and yields eq.
// (lnL-GM).  Weights are kept unnormalised (omega_j = u_j / Z), which makes
// the renormalisation after each component (step 3) implicit.
//
// The exact pass is fused with the E-step of the next sweep's first
// component, so a sweep of K components costs K passes over the particles.
//
// Precision: E-step densities / responsibilities FP32; statistics FP32 per
// thread and per warp, summed across warps in R; the M-step in R (FP32:
// precision 0, FP64: precision 1) with the component means accumulated to
// about 48 bits either way (FP64, or an unevaluated FP32 sum hi + lo when R
// is FP32, which keeps FP64 arithmetic off the M-step's critical path); the
// final unpenalised step (Sec. 2.3.1) entirely in FP64 with FP64-normalised
// responsibilities, which is what makes the moments exact.
#pragma once

#include "gm_common.cuh"

namespace gmcr {

struct EmParams {
  int64_t C, n;
  const int64_t* cell_off;
  const void* v;
  const double* alpha;
  int32_t* K_out;
  double* params_out;
  double* W_out;
  double* lnL_out;
  int32_t* sweeps_out;
  int32_t* kwork_out;
  uint32_t* status_out;
  const int32_t* init_K;   // optional initial mixtures (original coordinates)
  const double* init_prm;  // [C][Kmax][P]
  float* scratch;          // global tile for cells larger than the shared one
  int64_t scratch_stride;  // floats per array of the global tile (even)
  unsigned int* queue;
  // optional work list: the queue then runs over list[0 .. *list_count)
  // (the cells that a closed-form pre-pass left to EM)
  const unsigned int* list;
  const unsigned int* list_count;
  int Kmax, max_sweeps, cap;
  double tol;
  uint64_t seed;
};

// float offset o of cell j's global tile: even, and disjoint from its
// neighbours' tiles of N_j rounded up to even length.  Its velocity arrays
// start at o (stride: scratch_stride floats), its two pair records at
// D * stride + 2 o and (D + 2) * stride + 2 o.
__host__ __device__ inline int64_t scratch_offset(int64_t off, int64_t j) {
  return off + 2 * j + (off & 1);
}
// floats per array of the global tile; a multiple of 4, so that the pair
// records are 16-byte aligned
__host__ inline int64_t scratch_stride(int64_t n, int64_t C) { return (n + 2 * C + 2 + 3) & ~(int64_t)3; }

constexpr double kLn2 = 0.69314718055994530942;

template <int D>
struct NConst {  // packed E constants of one component
  static constexpr int NM = D * (D + 1) / 2;
  static constexpr int N = D + NM + 1;  // -mu (D), A (D = 3) or -A^2 (D = 1), b
};

// smallest power of two >= n (n <= 32)
constexpr int pow2_at_least(int n) { return n <= 1 ? 1 : 2 * pow2_at_least((n + 1) / 2); }

template <int D, int NW, typename R>
struct EmCtl {
  static constexpr int NM = D * (D + 1) / 2;
  static constexpr int NS = 1 + D + NM;
  static constexpr int NRED = pow2_at_least(NS + 1);  // statistics + log-likelihood
  // master parameters in whitened coordinates y = (v - mean) / sc
  R u[kMaxK];  // unnormalised weights, omega = u / Z (precision of the M-step)
  R Z;
  double mu[kMaxK][D];
  float mulo[kMaxK][D];  // R = FP32: mean = emu + mulo (emu the high part)
  double S0[NM];  // whitened total covariance (initial covariance of every component)
  // FP32 E-step constants: log2(u f) = b - |A (y - mu)|^2
  float emu[kMaxK][D];
  float eA[kMaxK][NM];  // lower triangle of sqrt(log2e/2) L^{-1}, row-major
  float elc[kMaxK];     // -log2|L| - (D/2) log2(2 pi)
  float eb[kMaxK];      // log2(u) + elc
  // FP64 M-step only: the product of the whitened covariance's pivots
  // (|Sigma_k|), the first-order log-likelihood error (log2 units, per unit
  // responsibility mass) of the FP32 inverse-factor diagonal the E-step
  // uses, and each component's responsibility mass N_k at its last update;
  // with them the convergence test corrects the log-likelihood for the
  // rounding of the FP32 E-step constants
  double pp[kMaxK];
  float corrA[kMaxK], Nkf[kMaxK];
  // the same, packed for the pair loop; slot kMaxK holds the previous
  // component's updated constants
  f32x2 ec[kMaxK + 1][NConst<D>::N];
  double mean[D], sc[D], isc[D];
  float meanf[D], scf[D];
  double Nd, W, L, logjac, logN;
  double cov0[D * (D + 1) / 2];  // the cell's weighted covariance (original coordinates)
  // convergence test on the centred log-likelihood (natural log, up to the
  // constant Lbase that c0 removes), assembled in FP64 from FP64 warp sums
  // of the FP32 per-particle terms: at the stopping point L changes by about
  // tol |L| per sweep, and an FP32 sum of N terms (or an FP32 log of the
  // weights' normaliser times N) errs by a tenth of that
  double Ld, Ldprev, Lbase;
  double sumAH;  // sum of the staged FP32 weights
  float c0;      // centring constant of the log-likelihood sum (log2 units)
  R NdR;
  float redf[NW][NRED];
  double redL[NW];  // per-warp FP64 sums of the centred log-likelihood terms
  double redd[NW][NS + 1];
  double res[NS + 1];
  // final step (centered original coordinates)
  double fw[kMaxK], fmu[kMaxK][D], fS[kMaxK][NM];
  int64_t cell;
  int K, Kf, k, sweep, kwork, annih, done, pstate, degenerate, final_pd;
  unsigned int status;
};

// ---------------------------------------------------------------------------
// small dense helpers (one thread)
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ int tri(int i, int j) {  // upper-triangle index, i <= j
  return D == 1 ? 0 : (i == 0 ? j : (i == 1 ? 2 + j : 5));
}

// Reciprocal and reciprocal square root for the one-thread M-step: an FP32
// hardware seed refined by Newton steps (two in FP64: relative error about
// 1e-16; one in FP32).  They avoid the long division / square-root
// sequences on the M-step's critical path.
__device__ __forceinline__ double rcp_nr(double x) {
  if (!(fabs(x) > 1e-30 && fabs(x) < 1e30)) return 1.0 / x;  // outside the FP32 seed's range
  double r = (double)rcp_approx((float)x);
  r = r * (2.0 - x * r);
  return r * (2.0 - x * r);
}
__device__ __forceinline__ float rcp_nr(float x) {
  const float r = rcp_approx(x);
  return r * (2.0f - x * r);
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ double rsqrt_nr(double x) {
  if (!(x > 1e-30 && x < 1e30)) return 1.0 / sqrt(x);  // outside the FP32 seed's range
  double y = (double)rsqrt_approx((float)x);
  y = y * (1.5 - 0.5 * x * y * y);
  return y * (1.5 - 0.5 * x * y * y);
}
__device__ __forceinline__ float rsqrt_nr(float x) {
  const float y = rsqrt_approx(x);
  return y * (1.5f - 0.5f * x * y * y);
}

// Cholesky of the upper-triangle S (precision R); returns false if a pivot
// is not positive or, measured in the original coordinates (pivots scale by
// sc_i^2), falls under rel * sum_d (Sigma_dd + mu_d^2) (rel = 1e-13: the
// covariance floor).  Lc[i][i] holds the pivot's square root and ri[i] its
// reciprocal.
template <int D, typename R, typename M>
__device__ bool chol_whitened(const R* S, const R* mu, const M* mean, const M* sc,
                              R (&Lc)[3][3], R (&ri)[3], double rel = 1e-13) {
  R scale2 = 0;
  for (int d = 0; d < D; ++d) {
    const R m = (R)mean[d] + (R)sc[d] * mu[d];
    scale2 += (R)(sc[d] * sc[d]) * S[tri<D>(d, d)] + m * m;
  }
  const R fl = (R)rel * scale2;
  for (int i = 0; i < D; ++i)
    for (int j = 0; j <= i; ++j) {
      R s = S[tri<D>(j, i)];
      for (int m = 0; m < j; ++m) s -= Lc[i][m] * Lc[j][m];
      if (i == j) {
        if (!(s * (R)(sc[i] * sc[i]) > fl) || !(s < (R)(sizeof(R) == 8 ? 1e300 : 1e30))) return false;
        ri[i] = rsqrt_nr(s);
        Lc[i][i] = s * ri[i];
      } else {
        Lc[i][j] = s * ri[j];
      }
    }
  return true;
}
template <int D, typename R, typename M>
__device__ bool chol_whitened(const R* S, const R* mu, const M* mean, const M* sc,
                              R (&Lc)[3][3]) {
  R ri[3];
  return chol_whitened<D, R, M>(S, mu, mean, sc, Lc, ri);
}

// E-step constants of a component from its Cholesky factor (ri: reciprocal
// diagonal)
template <int D, typename R>
__device__ void make_econst(const R (&Lc)[3][3], const R (&ri)[3], float* eA, float& elc) {
  const float c = 0.84932180028801904272f;  // sqrt(log2(e) / 2)
  if (D == 1) {
    eA[0] = c * (float)ri[0];
    elc = -lg2((float)Lc[0][0]) - 0.5f * 2.6514961294723187f;  // log2(2 pi) / 2
  } else {
    const R i00 = ri[0], i11 = ri[1], i22 = ri[2];
    const R i10 = -Lc[1][0] * i00 * i11;
    const R i21 = -Lc[2][1] * i11 * i22;
    const R i20 = -(Lc[2][0] * i00 + Lc[2][1] * i10) * i22;
    eA[0] = c * (float)i00;
    eA[1] = c * (float)i10;
    eA[2] = c * (float)i11;
    eA[3] = c * (float)i20;
    eA[4] = c * (float)i21;
    eA[5] = c * (float)i22;
    elc = -lg2((float)Lc[0][0]) - lg2((float)Lc[1][1]) - lg2((float)Lc[2][2]) -
          1.5f * 2.6514961294723187f;
  }
}

// packed copy of scalar E constants
template <int D>
__device__ __forceinline__ void pack_econst(const float* mu, const float* A, float b, f32x2* out) {
  constexpr int NM = D * (D + 1) / 2;
  for (int x = 0; x < D; ++x) out[x] = bc2(-mu[x]);
  if (D == 1)
    out[1] = bc2(-A[0] * A[0]);
  else
    for (int q = 0; q < NM; ++q) out[D + q] = bc2(A[q]);
  out[D + NM] = bc2(b);
}

// log2(u_k f_k(y)) (scalar), with d = y - mu returned
template <int D>
__device__ __forceinline__ float lg_eval(const float* mu, const float* A, float b, const float* y,
                                         float* d) {
  if (D == 1) {
    d[0] = y[0] - mu[0];
    const float t0 = A[0] * d[0];
    return fmaf(-t0, t0, b);
  } else {
    d[0] = y[0] - mu[0];
    d[1] = y[1] - mu[1];
    d[2] = y[2] - mu[2];
    const float t0 = A[0] * d[0];
    const float t1 = fmaf(A[1], d[0], A[2] * d[1]);
    const float t2 = fmaf(A[3], d[0], fmaf(A[4], d[1], A[5] * d[2]));
    return b - fmaf(t0, t0, fmaf(t1, t1, t2 * t2));
  }
}

// the same for a pair of particles (packed constants)
template <int D>
__device__ __forceinline__ f32x2 lg_eval2(const f32x2* e, const f32x2* y, f32x2* d) {
  constexpr int NM = D * (D + 1) / 2;
  if (D == 1) {
    d[0] = add2(y[0], e[0]);
    return fma2(e[1], mul2(d[0], d[0]), e[2]);
  } else {
    d[0] = add2(y[0], e[0]);
    d[1] = add2(y[1], e[1]);
    d[2] = add2(y[2], e[2]);
    const f32x2 t0 = mul2(e[3], d[0]);
    const f32x2 t1 = fma2(e[4], d[0], mul2(e[5], d[1]));
    const f32x2 t2 = fma2(e[6], d[0], fma2(e[7], d[1], mul2(e[8], d[2])));
    const f32x2 q = fma2(t0, t0, fma2(t1, t1, mul2(t2, t2)));
    return fma2(q, bc2(-1.0f), e[D + NM]);
  }
}

// FP64 block reduction of NV values (NV <= NS + 1); result in c.res
template <int D, int NT, int NV, typename R>
__device__ __forceinline__ void block_sum_d(EmCtl<D, NT / 32, R>& c, double (&v)[NV]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) c.redd[w][i] = v[i];
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
    for (int q = 0; q < NT / 32; ++q) s += c.redd[q][threadIdx.x];
    c.res[threadIdx.x] = s;
  }
  __syncthreads();
}

// Warp sum of NP values (NP a power of two <= 32) by recursive halving: at
// each level a lane keeps half of its values, sends the other half to its
// partner and adds what it receives, so NP values cost NP - 1 + 5 - log2(NP)
// shuffles instead of 5 NP.  On return v[0] of every lane holds the warp
// total of value warp_rs_index<NP>(lane).
template <int NP>
__device__ __forceinline__ void warp_rs(float (&v)[NP], int lane) {
  constexpr int LV = NP == 1 ? 0 : (NP == 2 ? 1 : (NP == 4 ? 2 : (NP == 8 ? 3 : (NP == 16 ? 4 : 5))));
#pragma unroll
  for (int lv = 0; lv < LV; ++lv) {
    const int h = NP >> (lv + 1), b = 16 >> lv;
    const bool up = (lane & b) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const float send = up ? v[i] : v[i + h];
      const float keep = up ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, b);
    }
  }
#pragma unroll
  for (int b = 16 >> LV; b >= 1; b >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], b);
}
template <int NP>
__device__ __forceinline__ int warp_rs_index(int lane) {
  int q = 0;
#pragma unroll
  for (int lv = 0; (NP >> lv) > 1; ++lv) q += ((lane >> (4 - lv)) & 1) * (NP >> (lv + 1));
  return q;
}

// warp sums of NP doubles by recursive halving (the FP64 form of warp_rs):
// lane l ends with the total of value warp_rs_index<NP>(l) in v[0]
template <int NP>
__device__ __forceinline__ void warp_rs_d(double (&v)[NP], int lane) {
  constexpr int LV = NP == 1 ? 0 : (NP == 2 ? 1 : (NP == 4 ? 2 : (NP == 8 ? 3 : (NP == 16 ? 4 : 5))));
#pragma unroll
  for (int lv = 0; lv < LV; ++lv) {
    const int h2 = NP >> (lv + 1), b = 16 >> lv;
    const bool up = (lane & b) != 0;
#pragma unroll
    for (int i = 0; i < h2; ++i) {
      const double send = up ? v[i] : v[i + h2];
      const double keep = up ? v[i + h2] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, b);
    }
  }
#pragma unroll
  for (int b = 16 >> LV; b >= 1; b >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], b);
}

// per-warp totals of NV per-thread values into red[warp][q], then a barrier
template <int NV, int NP, int NW>
__device__ __forceinline__ void block_partials(const float (&v)[NV], float (&red)[NW][NP]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float t[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) t[q] = q < NV ? v[q] : 0.0f;
  warp_rs<NP>(t, lane);
  if ((lane & (32 / NP - 1)) == 0) {
    const int q = warp_rs_index<NP>(lane);
    if (q < NV) red[w][q] = t[0];
  }
  __syncthreads();
}

// one component (thread 0): fw, fmu, fS of the final mixture = the sample
// moments; L = eq. (lnL-GM) in closed form: -(N/2)(D ln 2 pi + ln|Sigma| +
// D) - (T/2) ln N (d = T parameters, ln omega = 0); the covariance passed
// the floor in the prologue
template <int D, int NT, typename R>
__device__ void k1_closed_form(EmCtl<D, NT / 32, R>& c) {
  constexpr int NM = D * (D + 1) / 2;
  constexpr int T = D * (D + 3) / 2;
  c.K = 1;
  c.fw[0] = 1.0;
  for (int d = 0; d < D; ++d) c.fmu[0][d] = 0.0;
  for (int i = 0; i < NM; ++i) c.fS[0][i] = c.cov0[i];
  double L2[3][3] = {{0}}, logdet = 0.0;
  for (int x = 0; x < D; ++x)
    for (int y = 0; y <= x; ++y) {
      double sv = c.cov0[tri<D>(y, x)];
      for (int m = 0; m < y; ++m) sv -= L2[x][m] * L2[y][m];
      if (x == y) {
        L2[x][x] = sqrt(sv);
        logdet += 2.0 * log(L2[x][x]);
      } else {
        L2[x][y] = sv / L2[y][y];
      }
    }
  c.L = -0.5 * c.Nd * ((double)D * 1.8378770664093454836 + logdet + (double)D) - 0.5 * (double)T * c.logN;
  c.final_pd = 1;
}

// the cell's outputs (thread 0 writes, then a barrier)
template <int D, int NT, typename R>
__device__ __forceinline__ void write_cell(const EmParams& a, EmCtl<D, NT / 32, R>& c, int64_t j,
                                           double* prm_out) {
  constexpr int NM = D * (D + 1) / 2;
  constexpr int P = 1 + D + NM;
  if (threadIdx.x == 0) {
    const int Kf = c.K;
    for (int k = 0; k < Kf; ++k) {
      double* r = prm_out + (size_t)k * P;
      r[0] = c.fw[k];
      for (int d = 0; d < D; ++d) r[1 + d] = c.mean[d] + c.fmu[k][d];
      for (int q = 0; q < NM; ++q) r[1 + D + q] = c.fS[k][q];
    }
    for (int i = Kf * P; i < a.Kmax * P; ++i) prm_out[i] = 0.0;
    a.K_out[j] = Kf;
    a.W_out[j] = c.W;
    a.lnL_out[j] = c.final_pd ? c.L : 0.0;
    if (a.sweeps_out) a.sweeps_out[j] = c.sweep;
    if (a.kwork_out) a.kwork_out[j] = c.kwork;
    a.status_out[j] = c.status;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// one cell, after its moments are known and it is not degenerate.  The
// particle tile (shared or global) holds N rounded up to even particles (a
// zero-weight pad particle) as pairs:
//   Y[d][p]  whitened velocity, array d at Y + d * ys
//   SMT[pp]  16 bytes per pair: {s_p (2), -m_p (2)}
//   GAT[pp]  16 bytes per pair: {the current component's term (2), the
//            normalised weights (2)}
// so a pair's state is read with one 16-byte load per record.
// ---------------------------------------------------------------------------
template <int D, int NT, typename VT, typename R>
__device__ __forceinline__ void em_cell_body(const EmParams& a, EmCtl<D, NT / 32, R>& c,
                                             int64_t j, int64_t off, int N, float* Y, int ys,
                                             float* SMT, float* GAT) {
  constexpr int NW = NT / 32;
  constexpr int NM = D * (D + 1) / 2;
  constexpr int NS = 1 + D + NM;
  constexpr int T = D * (D + 3) / 2;
  constexpr int P = 1 + D + NM;
  constexpr int NC = NConst<D>::N;
  const double halfT = 0.5 * T;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const VT* __restrict__ vin = static_cast<const VT*>(a.v);
  double* prm_out = a.params_out + (size_t)j * a.Kmax * P;
  const int P2 = (N + 1) >> 1;  // particle pairs
  const int ys2 = ys >> 1;

  // ---- initialisation --------------------------------------------------
  // A supplied initial mixture (learned initialisation) is used when given:
  // components failing the Cholesky floor are dropped, the count is capped
  // so that N - T K / 2 > 0, and an empty result falls back to the paper's
  // initialisation (Sec. 2.3): Kmax components at random particles.
  if (tid == 0) {
    int K = 0;
    if (a.init_K) {
      const int K0 = a.init_K[j] < a.Kmax ? a.init_K[j] : a.Kmax;
      double wsum = 0.0;
      for (int k = 0; k < K0; ++k) {
        const double* r = a.init_prm + ((size_t)j * a.Kmax + k) * P;
        double mw[D], Sw[NM], Lw[3][3], rw[3];
        for (int d = 0; d < D; ++d) mw[d] = (r[1 + d] - c.mean[d]) * c.isc[d];
        int q = 0;
        for (int x = 0; x < D; ++x)
          for (int yy = x; yy < D; ++yy, ++q) Sw[q] = r[1 + D + q] * c.isc[x] * c.isc[yy];
        if (!(r[0] > 0.0) || !chol_whitened<D, double, double>(Sw, mw, c.mean, c.sc, Lw, rw))
          continue;
        float eA[NM], elc;
        make_econst<D, double>(Lw, rw, eA, elc);
        for (int d = 0; d < D; ++d) {
          c.mu[K][d] = mw[d];
          c.emu[K][d] = (float)mw[d];
          c.mulo[K][d] = (float)(mw[d] - (double)c.emu[K][d]);
        }
        for (int i = 0; i < NM; ++i) c.eA[K][i] = eA[i];
        c.elc[K] = elc;
        c.u[K] = (R)r[0];
        wsum += r[0];
        ++K;
      }
      while (K > 1 && c.Nd - halfT * K <= 0.0) {
        --K;
        wsum -= (double)c.u[K];
      }
      for (int k = 0; k < K; ++k) {
        c.u[k] = (R)((double)c.u[k] / wsum);
        c.eb[k] = lg2((float)c.u[k]) + c.elc[k];
        c.pp[k] = 1.0;
        c.corrA[k] = c.Nkf[k] = 0.0f;
        pack_econst<D>(c.emu[k], c.eA[k], c.eb[k], c.ec[k]);
      }
      c.K = K;
      c.Z = (R)1;
    }
  }
  __syncthreads();
  if (tid == 0 && c.K == 0) {
    int K = a.Kmax < N ? a.Kmax : N;
    while (K > 1 && c.Nd - halfT * K <= 0.0) --K;
    int picks[kMaxK];
    int got = 0;
    for (uint32_t t = 0; got < K; ++t) {
      int idx;
      if (t < 100000u) {
        const u32x4 r = philox_draw(a.seed, t, kTagInit, j);
        const double uu = uniform52(r.x, r.y);
        idx = (int)floor(uu * c.Nd);
        if (idx >= N) idx = N - 1;
      } else {
        idx = 0;
        for (;;) {
          bool used = false;
          for (int m = 0; m < got; ++m) used |= (picks[m] == idx);
          if (!used) break;
          ++idx;
        }
      }
      bool dup = false;
      for (int m = 0; m < got; ++m) dup |= (picks[m] == idx);
      if (!dup) picks[got++] = idx;
    }
    c.K = K;
    c.Z = (R)1;
    R Lc[3][3], ri[3];
    R S0[NM], m0[D];
    for (int i = 0; i < NM; ++i) S0[i] = (R)c.S0[i];
    for (int d = 0; d < D; ++d) m0[d] = 0;
    chol_whitened<D, R, double>(S0, m0, c.mean, c.sc, Lc, ri);  // the total covariance passed
    float eA[NM], elc;
    make_econst<D, R>(Lc, ri, eA, elc);
    for (int k = 0; k < K; ++k) {
      c.u[k] = (R)1 / (R)K;
      for (int d = 0; d < D; ++d) {
        c.mu[k][d] = ((double)vin[(int64_t)d * a.n + off + picks[k]] - c.mean[d]) * c.isc[d];
        c.emu[k][d] = (float)c.mu[k][d];
        c.mulo[k][d] = (float)(c.mu[k][d] - (double)c.emu[k][d]);
      }
      for (int i = 0; i < NM; ++i) c.eA[k][i] = eA[i];
      c.elc[k] = elc;
      c.eb[k] = lg2((float)c.u[k]) + elc;
      c.pp[k] = 1.0;
      c.corrA[k] = c.Nkf[k] = 0.0f;
      pack_econst<D>(c.emu[k], c.eA[k], c.eb[k], c.ec[k]);
    }
  }
  __syncthreads();
  // ---- one component: the EM's fixed point in closed form ----------------
  // With K = 1 every responsibility is the particle's weight, so one EM step
  // from any start gives the weighted sample mean and covariance (Sec.
  // 2.3.1), and eq. (lnL-GM) is -(N/2)(D ln 2 pi + ln|Sigma| + D) - (T/2) ln N.
  // Reported as one sweep without component E-steps (kwork 0).
  if (c.K == 1) {
    if (tid == 0) {
      c.sweep = 1;
      c.kwork = 0;
      k1_closed_form<D, NT, R>(c);
    }
    __syncthreads();
    write_cell<D, NT, R>(a, c, j, prm_out);
    return;
  }
  // ---- stage whitened velocities and normalised weights ------------------
  {
    const double nw = c.Nd / c.W;
    double sa[1] = {0.0};
    for (int p = tid; p < 2 * P2; p += NT) {
      if (p < N) {
#pragma unroll
        for (int d = 0; d < D; ++d)
          Y[d * ys + p] = (float)(((double)vin[(int64_t)d * a.n + off + p] - c.mean[d]) * c.isc[d]);
        const float ah = (float)(a.alpha[off + p] * nw);
        GAT[4 * (p >> 1) + 2 + (p & 1)] = ah;
        sa[0] += (double)ah;
      } else {  // zero-weight pad particle
#pragma unroll
        for (int d = 0; d < D; ++d) Y[d * ys + p] = 0.0f;
        GAT[4 * (p >> 1) + 2 + (p & 1)] = 0.0f;
      }
    }
    block_sum_d<D, NT, 1, R>(c, sa);
    if (tid == 0) {
      c.sumAH = c.res[0];
      c.c0 = -2.0471975511965976f * D;  // mean log2 density of a standard normal
      c.NdR = (R)c.Nd;
    }
  }
  if (tid == 0) {
    c.sweep = 0;
    c.kwork = 0;
    c.done = 0;
    c.annih = 0;
  }
  __syncthreads();

  const f32x2* Y2 = reinterpret_cast<const f32x2*>(Y);
  ulonglong2* SM4 = reinterpret_cast<ulonglong2*>(SMT);
  ulonglong2* GA4 = reinterpret_cast<ulonglong2*>(GAT);
  f32x2* GG2 = reinterpret_cast<f32x2*>(GAT);  // term of pair pp at GG2[2 * pp]
  constexpr int NRED = EmCtl<D, NW, R>::NRED;

  // ---- annihilation of component k (one thread): compaction, eq. (omegak)'s
  // renormalisation through Z
  auto remove_comp = [&](int k) {
    const int K = c.K;
    c.Z -= c.u[k];
    for (int m = k; m < K - 1; ++m) {
      c.u[m] = c.u[m + 1];
      for (int x = 0; x < D; ++x) {
        c.mu[m][x] = c.mu[m + 1][x];
        c.emu[m][x] = c.emu[m + 1][x];
        c.mulo[m][x] = c.mulo[m + 1][x];
      }
      for (int q = 0; q < NM; ++q) c.eA[m][q] = c.eA[m + 1][q];
      for (int q = 0; q < NC; ++q) c.ec[m][q] = c.ec[m + 1][q];
      c.elc[m] = c.elc[m + 1];
      c.eb[m] = c.eb[m + 1];
      c.pp[m] = c.pp[m + 1];
      c.corrA[m] = c.corrA[m + 1];
      c.Nkf[m] = c.Nkf[m + 1];
    }
    c.K = K - 1;
    c.annih = 1;
    c.pstate = 2;
  };

  // ---- M-step for component k (eqs. muk, sigmak, omegak), one thread -----
  // sv: N_k, the first moments and the second moments about the FP32 mean
  // the E-step used.
  auto mstep = [&](int k, const R (&sv)[NS + 1]) {
    c.kwork++;
    const int K = c.K;
    const R Nk = sv[0];
    bool removed = false;
    if (K > 1 && Nk - (R)halfT <= (R)0) {
      removed = true;
    } else {
      const R rN = rcp_nr(Nk);
      R dl[D], mun[D], Sn[NM];
      // The shift of the mean is added to a ~48-bit master copy (FP64, or
      // hi + lo FP32 when R is FP32), which keeps the sub-ulp part of every
      // update: the FP32 copy then follows the FP64 trajectory instead of
      // stalling when an update is below its resolution.
      double mu64[D];
      float mlo[D];
      for (int x = 0; x < D; ++x) {
        dl[x] = sv[1 + x] * rN;
        if constexpr (sizeof(R) == 4) {
          const float hi = c.emu[k][x];
          const float sm = hi + (float)dl[x];  // two-sum of hi and the shift
          const float bb = sm - hi;
          const float er = (hi - (sm - bb)) + ((float)dl[x] - bb);
          const float lo = c.mulo[k][x] + er;
          const float h2 = sm + lo;  // renormalise
          mlo[x] = lo - (h2 - sm);
          mun[x] = (R)h2;
        } else {
          mu64[x] = c.mu[k][x] + (double)dl[x];
          mun[x] = (R)mu64[x];
        }
      }
      int t = 0;
      for (int x = 0; x < D; ++x)
        for (int yy = x; yy < D; ++yy, ++t) Sn[t] = sv[1 + D + t] * rN - dl[x] * dl[yy];
      R Lc[3][3], ri[3];
      bool pd;
      if constexpr (sizeof(R) == 4)
        pd = chol_whitened<D, R, float>(Sn, mun, c.meanf, c.scf, Lc, ri);
      else
        pd = chol_whitened<D, R, double>(Sn, mun, c.mean, c.sc, Lc, ri);
      if (!pd) {
        c.status |= GM_ST_COV_NOT_PD;
        if (K > 1) {
          removed = true;
        } else {
          c.pstate = 0;  // a lone component keeps its parameters
          c.k = k + 1;
        }
      } else {
        // eq. (omegak), then the renormalisation of step 3 through Z
        const R wn = (K == 1) ? (R)1 : (Nk - (R)halfT) * rcp_nr(c.NdR - (R)halfT * (R)K);
        const R un = wn * c.Z;
        c.Z = c.Z - c.u[k] + un;
        c.u[k] = un;
        float eA[NM], elc;
        make_econst<D, R>(Lc, ri, eA, elc);
        for (int x = 0; x < D; ++x) {
          if constexpr (sizeof(R) == 4)
            c.mulo[k][x] = mlo[x];
          else
            c.mu[k][x] = mu64[x];
          c.emu[k][x] = (float)mun[x];
        }
        for (int q = 0; q < NM; ++q) c.eA[k][q] = eA[q];
        c.elc[k] = elc;
        const float eb = lg2((float)un) + elc;
        c.eb[k] = eb;
        float emu[D];
        for (int x = 0; x < D; ++x) emu[x] = (float)mun[x];
        f32x2 ec[NC];
        pack_econst<D>(emu, eA, eb, ec);
        for (int q = 0; q < NC; ++q) {
          c.ec[k][q] = ec[q];
          c.ec[kMaxK][q] = ec[q];
        }
        c.pstate = 1;
        c.k = k + 1;
      }
    }
    if (removed) remove_comp(k);
  };

  // ---- the same M-step in FP64 by the 32 lanes of warp 0 (precision 1) ------
  // Every lane holds the cross-warp FP64 sums sv.  Independent FP64 steps run
  // on separate lanes in one instruction (the two reciprocals, the D new
  // means, the D(D+1)/2 covariance entries, the floor's D terms), which
  // keeps the FP64 instruction count -- GB300's FP64 pipe is 1/64 of its
  // FP32 rate and every warp instruction occupies it whole -- near 60.
  // The covariance about the new mean is factored as L~ diag(p) L~^T in
  // FP64 (pivots p_i = the squared Cholesky diagonal); the FP32 E-step
  // constants are then c diag(p)^-1/2 L~^-1 with c = sqrt(log2(e) / 2) and
  // eb = log2(u) - log2|L| - (D/2) log2(2 pi) (FP32 logarithms: their error
  // is what the convergence test corrects for).  The floor test is
  // chol_whitened's: p_i sc_i^2 > 1e-13 sum_d (sc_d^2 S_dd + m_d^2) and
  // p_i < 1e300.
  auto mstep64 = [&](int k, const double (&sv)[NS + 1]) {
    const int K = c.K;
    const double Nk = sv[0];
    const double Zold = (double)c.Z, uold = (double)c.u[k];
    __syncwarp();
    if (lane == 0) c.kwork++;
    if (K > 1 && Nk - halfT <= 0.0) {
      if (lane == 0) remove_comp(k);
      __syncwarp();
      return;
    }
    // 1 / N_k (lane 0) and 1 / (N - T K / 2) (lane 1)
    const double rin = rcp_nr(lane == 1 ? (double)c.NdR - halfT * K : Nk);
    const double rN = __shfl_sync(0xffffffffu, rin, 0);
    const double rD = __shfl_sync(0xffffffffu, rin, 1);
    // the mean's shift dl and the new FP64 mean, coordinate x on lane x
    double dl[D], mun[D];
    {
      double s1 = sv[1];
      if (D == 3) s1 = lane == 1 ? sv[2] : (lane == 2 ? sv[3] : sv[1]);
      const double dlv = s1 * rN;
      const double mv = c.mu[k][lane < D ? lane : 0] + dlv;
#pragma unroll
      for (int x = 0; x < D; ++x) {
        dl[x] = __shfl_sync(0xffffffffu, dlv, x);
        mun[x] = __shfl_sync(0xffffffffu, mv, x);
      }
    }
    // covariance about the new mean, entry t (upper triangle) on lane t
    double Sn[NM];
    if (D == 1) {
      Sn[0] = fma(-dl[0], dl[0], sv[2] * rN);
    } else {
      const int t = lane < NM ? lane : 0;
      const int tx = t < 3 ? 0 : (t < 5 ? 1 : 2);
      const int ty = t < 3 ? t : (t < 5 ? t - 2 : 2);
      double s2 = sv[4];
#pragma unroll
      for (int q = 1; q < NM; ++q) s2 = t == q ? sv[4 + q] : s2;
      const double dx = tx == 0 ? dl[0] : (tx == 1 ? dl[1] : dl[D - 1]);
      const double dy = ty == 0 ? dl[0] : (ty == 1 ? dl[1] : dl[D - 1]);
      const double snv = fma(-dx, dy, s2 * rN);
#pragma unroll
      for (int q = 0; q < NM; ++q) Sn[q] = __shfl_sync(0xffffffffu, snv, q);
    }
    // L~ diag(p) L~^T (FP64)
    double piv[D], l10 = 0.0, l20 = 0.0, l21 = 0.0;
    piv[0] = Sn[0];
    if (D == 3) {
      const double r0 = rcp_nr(piv[0]);
      l10 = Sn[1] * r0;
      l20 = Sn[2] * r0;
      piv[1] = fma(-l10, Sn[1], Sn[3]);
      const double r1 = rcp_nr(piv[1]);
      const double e12 = fma(-l20, Sn[1], Sn[4]);
      l21 = e12 * r1;
      piv[D - 1] = fma(-l21, e12, fma(-l20, Sn[2], Sn[5]));
    }
    // floor test, coordinate d on lane d
    int pd;
    {
      const int d = lane < D ? lane : 0;
      const double pd_ = D == 1 ? piv[0] : (d == 0 ? piv[0] : (d == 1 ? piv[1] : piv[D - 1]));
      const double sdd = D == 1 ? Sn[0] : (d == 0 ? Sn[0] : (d == 1 ? Sn[3] : Sn[NM - 1]));
      const double mud = D == 1 ? mun[0] : (d == 0 ? mun[0] : (d == 1 ? mun[1] : mun[D - 1]));
      const double scd = c.sc[d], md = fma(scd, mud, c.mean[d]);
      double term = lane < D ? fma(scd * scd, sdd, md * md) : 0.0;
      if (D == 3) {
        term += __shfl_xor_sync(0xffffffffu, term, 1);
        term += __shfl_xor_sync(0xffffffffu, term, 2);
      }
      const double scale2 = __shfl_sync(0xffffffffu, term, 0);
      const bool ok = !(lane < D) || ((pd_ * (scd * scd) > 1e-13 * scale2) && (pd_ < 1e300));
      pd = __all_sync(0xffffffffu, ok);
    }
    if (!pd) {
      if (lane == 0) {
        c.status |= GM_ST_COV_NOT_PD;
        if (K > 1) {
          remove_comp(k);
        } else {
          c.pstate = 0;  // a lone component keeps its parameters
          c.k = k + 1;
        }
      }
      __syncwarp();
      return;
    }
    // eq. (omegak), then the renormalisation of step 3 through Z
    const double wn = (K == 1) ? 1.0 : (Nk - halfT) * rD;
    const double un = wn * Zold;
    // FP32 E constants: p_i^-1/2 on lane i
    float ri[D];
    {
      const int d = lane < D ? lane : 0;
      const float pf = (float)(D == 1 ? piv[0] : (d == 0 ? piv[0] : (d == 1 ? piv[1] : piv[D - 1])));
      const float rr = rsqrt_nr(pf);
#pragma unroll
      for (int x = 0; x < D; ++x) ri[x] = __shfl_sync(0xffffffffu, rr, x);
    }
    const float cc = 0.84932180028801904272f;  // sqrt(log2(e) / 2)
    float eA[NM];
    if (D == 1) {
      eA[0] = cc * ri[0];
    } else {
      eA[0] = cc * ri[0];
      eA[1] = cc * (float)(-l10) * ri[1];
      eA[2] = cc * ri[1];
      eA[3] = cc * (float)fma(l10, l21, -l20) * ri[D - 1];
      eA[4] = cc * (float)(-l21) * ri[D - 1];
      eA[5] = cc * ri[D - 1];
    }
    // eb = log2(u) - (1/2) log2(prod p) - (D/2) log2(2 pi) (FP32), and the
    // first-order log-likelihood error of the FP32 inverse factor's diagonal:
    // the quadratic form's error summed over the component's
    // responsibilities is N_k sum_i (A_ii^2 p_i - c^2), A_ii as used
    double pp = piv[0];
#pragma unroll
    for (int x = 1; x < D; ++x) pp *= piv[x];
    const float eb = lg2((float)un) - 0.5f * lg2((float)pp) - (float)D * 1.3257480647361593f;
    double ca = 0.0;
    if (D == 1) {
      const float a2 = eA[0] * eA[0];  // the packed constant is -A^2 (one FP32 product)
      ca = fma((double)a2, piv[0], -0.72134752044448170368);
    } else {
      ca = fma((double)eA[0] * (double)eA[0], piv[0], -0.72134752044448170368) +
           fma((double)eA[2] * (double)eA[2], piv[1], -0.72134752044448170368) +
           fma((double)eA[5] * (double)eA[5], piv[D - 1], -0.72134752044448170368);
    }
    float ec[NC];
    {
      float em[D];
#pragma unroll
      for (int x = 0; x < D; ++x) em[x] = (float)mun[x];
      f32x2 e2[NC];
      pack_econst<D>(em, eA, eb, e2);
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        float lo, hi;
        upk2(e2[q], lo, hi);
        ec[q] = lo;
      }
    }
    __syncwarp();
    if (lane < D) {
      const int x = lane;
      double mx = mun[0];
#pragma unroll
      for (int q = 1; q < D; ++q) mx = x == q ? mun[q] : mx;
      c.mu[k][x] = mx;
      c.emu[k][x] = (float)mx;
    }
    if (lane < NM) {
      float ax = eA[0];
#pragma unroll
      for (int q = 1; q < NM; ++q) ax = lane == q ? eA[q] : ax;
      c.eA[k][lane] = ax;
    }
    if (lane < NC) {
      float ex = ec[0];
#pragma unroll
      for (int q = 1; q < NC; ++q) ex = lane == q ? ec[q] : ex;
      c.ec[k][lane] = bc2(ex);
      c.ec[kMaxK][lane] = bc2(ex);
    }
    if (lane == 0) {
      c.Z = (R)(Zold - uold + un);
      c.u[k] = (R)un;
      c.elc[k] = eb - lg2((float)un);
      c.eb[k] = eb;
      c.pp[k] = pp;
      c.corrA[k] = (float)ca;
      c.Nkf[k] = (float)Nk;
      c.pstate = 1;
      c.k = k + 1;
    }
    __syncwarp();
  };

  // ---- exact pass: s_p, m_p and eq. (lnL-GM) ------------------------------
  // s_p = sum_k 2^(log2(u_k f_k) - m_p).  A fresh pass (the first of a cell,
  // or a pair whose sum left [1e-30, 1e30]) takes m_p = max_k log2(u_k f_k),
  // so s_p >= 1; otherwise the pair keeps its previous shift m_p, which saves
  // the pass for the maximum.  Either way every unchanged component's term
  // stays below 1e30 until the next exact pass.  The per-particle
  // log-likelihood enters the sum minus a per-cell constant c0 close to its
  // mean, which keeps the FP32 partial sums small.  With stats0 the pass also
  // yields component 0's E-step statistics (the first step of the next
  // sweep).  Per-warp partials: c.redf[w][0 .. NS-1] statistics,
  // c.redf[w][NS] the centred sum.
  auto exact_pass = [&](bool stats0, bool fresh) {
    const int K = c.K;
    const float c0 = c.c0;
    float accl = 0.0f;
    f32x2 acc[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) acc[q] = 0ull;
    for (int pp = tid; pp < P2; pp += NT) {
      f32x2 y[D], d[D], d0[D];
#pragma unroll
      for (int q = 0; q < D; ++q) y[q] = Y2[q * ys2 + pp];
      f32x2 nm, sp, G;
      float x0, x1, s0 = 0.0f, s1 = 0.0f;
      bool slow = fresh;
      if (!fresh) {
        nm = SM4[pp].y;
        upk2(add2(lg_eval2<D>(c.ec[0], y, d0), nm), x0, x1);
        G = pk2(ex2(x0), ex2(x1));
        sp = G;
        for (int k = 1; k < K; ++k) {
          upk2(add2(lg_eval2<D>(c.ec[k], y, d), nm), x0, x1);
          sp = add2(sp, pk2(ex2(x0), ex2(x1)));
        }
        upk2(sp, s0, s1);
        slow = !(s0 > 1e-30f && s0 < 1e30f && s1 > 1e-30f && s1 < 1e30f);
      }
      if (slow) {
        float m0 = -3.0e38f, m1 = -3.0e38f;
        for (int k = 0; k < K; ++k) {
          float l0, l1;
          upk2(lg_eval2<D>(c.ec[k], y, d), l0, l1);
          m0 = fmaxf(m0, l0);
          m1 = fmaxf(m1, l1);
        }
        nm = pk2(-m0, -m1);
        upk2(add2(lg_eval2<D>(c.ec[0], y, d0), nm), x0, x1);
        G = pk2(ex2(x0), ex2(x1));
        sp = G;
        for (int k = 1; k < K; ++k) {
          upk2(add2(lg_eval2<D>(c.ec[k], y, d), nm), x0, x1);
          sp = add2(sp, pk2(ex2(x0), ex2(x1)));
        }
        upk2(sp, s0, s1);
      }
      SM4[pp] = make_ulonglong2(sp, nm);
      const f32x2 ah = GA4[pp].y;
      float a0, a1, n0, n1;
      upk2(ah, a0, a1);
      upk2(nm, n0, n1);
      accl = fmaf(a0, (-n0 - c0) + lg2(s0), accl);
      accl = fmaf(a1, (-n1 - c0) + lg2(s1), accl);
      if (stats0) {
        GG2[2 * pp] = G;
        const f32x2 gam = mul2(ah, mul2(G, pk2(rcp_approx(s0), rcp_approx(s1))));
        acc[0] = add2(acc[0], gam);
        int t = 1 + D;
#pragma unroll
        for (int x = 0; x < D; ++x) {
          const f32x2 gd = mul2(gam, d0[x]);
          acc[1 + x] = add2(acc[1 + x], gd);
#pragma unroll
          for (int yy = x; yy < D; ++yy, ++t) acc[t] = fma2(gd, d0[yy], acc[t]);
        }
      }
    }
    float v[NS + 1];
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      float lo, hi;
      upk2(acc[q], lo, hi);
      v[q] = lo + hi;
    }
    v[NS] = 0.0f;
    const double accw = warp_sum((double)accl);
    if (lane == 0) c.redL[wid] = accw;
    block_partials<NS + 1, NRED, NW>(v, c.redf);
  };

  // warp 0 after a pass that summed the log-likelihood: the cross-warp sums
  // of the statistics (returned in sv by every lane of warp 0) and eq.
  // (lnL-GM) (lane 0, FP64): the centred value c.Ld for the convergence test,
  // and with full the value c.L.  The first pass of a cell fixes c0 at the
  // mean per-particle term, so that later passes sum small deviations.  The
  // weights enter as omega_k = u_k / Z with Z = sum_k u_k summed afresh in
  // FP64 (the running Z of the M-step carries its rounding).
  auto finish_exact = [&](R (&sv)[NS + 1], bool full) {
    const int K = c.K;
    R st[NW];
#pragma unroll
    for (int q = 0; q < NW; ++q) st[q] = lane < NS ? (R)c.redf[q][lane] : (R)0;
#pragma unroll
    for (int h = NW / 2; h >= 1; h >>= 1)
#pragma unroll
      for (int q = 0; q < h; ++q) st[q] += st[q + h];
#pragma unroll
    for (int q = 0; q < NS; ++q) sv[q] = __shfl_sync(0xffffffffu, st[0], q);
    sv[NS] = (R)0;
    const double ud = lane < K ? (double)c.u[lane] : 0.0;
    const double Zd = warp_sum(ud);
    float pen = lane < K ? lg2((float)ud / (float)Zd) : 0.0f;  // log2 omega_k
    pen = warp_sum(pen) * (float)kLn2;
    // FP64 logarithms in one lane-parallel sequence: lane k < K log2 u_k,
    // lane 16 + k log2 |Sigma_k|, lane K (K < 16) log2 Z
    const int kk = lane & 15;
    double arg = 1.0;
    if (lane < K) arg = ud;
    else if (lane >= 16 && kk < K) arg = (sizeof(R) == 8) ? c.pp[kk] : 1.0;
    else if (lane == K) arg = Zd;
    const double lg = log2(arg);
    const double lz = K < 16 ? __shfl_sync(0xffffffffu, lg, K < 16 ? K : 0) : log2(Zd);
    // FP64 M-step, convergence test: the first-order correction
    // sum_k N_k corr_k (log2 units) of the log-likelihood for the rounding of
    // the FP32 E-step constants, corr_k = (eb_k exact - eb_k as used) +
    // corrA_k (see mstep64).  Not for the reported value after the final
    // step (full), whose constants the final step rebuilt.
    float cor = 0.0f;
    if (sizeof(R) == 8 && !full) {
      const double lpp = __shfl_sync(0xffffffffu, lg, (lane + 16) & 31);
      float ck = 0.0f;
      if (lane < K) {
        const double b64 = lg - 0.5 * lpp - D * 1.3257480647361593;
        ck = c.Nkf[lane] * ((float)(b64 - (double)c.eb[lane]) + c.corrA[lane]);
      }
      cor = warp_sum(ck);
    }
    if (lane == 0) {
      const int dpar = K * (T + 1) - 1;
      double lsum = (double)cor;
#pragma unroll
      for (int q = 0; q < NW; ++q) lsum += c.redL[q];
      lsum -= c.sumAH * lz;
      const double pc = -0.5 * dpar * c.logN - 0.5 * T * (double)pen;
      if (full || c.sweep == 0) {
        const double ls = lsum + (double)c.c0 * c.sumAH;
        c.L = ls * kLn2 - c.Nd * c.logjac + pc;
        if (!full) {
          const float c0n = c.sumAH > 0.0 ? (float)(ls / c.sumAH) : c.c0;
          c.c0 = c0n;
          c.Ld = (ls - (double)c0n * c.sumAH) * kLn2 + pc;
          c.Lbase = (double)c0n * c.sumAH * kLn2 - c.Nd * c.logjac;
        }
      } else {
        c.Ld = kLn2 * lsum + pc;
      }
    }
  };

  // ---- one component step's pass ----------------------------------------
  // Replaces the previous component's term in s_p (ps = 1: updated, 2:
  // removed), evaluates component k and accumulates its statistics; with
  // withL it also sums the centred log-likelihood of s_p after the
  // replacement (the first step of a sweep without an exact pass: s_p then
  // holds every component's current term).  A pair whose s_p dropped more
  // than 64-fold in the replacement (cancellation), or with withL left
  // [1e-30, 1e30], is recomputed exactly from all components with a fresh
  // shift.  Terms are clamped at 2^100 relative to the shift.
  auto comp_pass = [&](int k, int ps, bool withL) {
    const f32x2* ek = c.ec[k];
    const f32x2* ep = c.ec[kMaxK];
    const int K = c.K;
    const float c0 = c.c0;
    float accl = 0.0f;
    f32x2 acc[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) acc[q] = 0ull;
    for (int pp = tid; pp < P2; pp += NT) {
      f32x2 y[D], d[D];
#pragma unroll
      for (int q = 0; q < D; ++q) y[q] = Y2[q * ys2 + pp];
      const ulonglong2 sm = SM4[pp];
      const ulonglong2 ga = GA4[pp];
      f32x2 nm = sm.y;  // -m
      f32x2 sp = sm.x;
      bool fix = false;
      if (ps != 0) {
        float so0, so1;
        upk2(sp, so0, so1);
        float sn0, sn1;
        if (ps == 1) {  // previous component updated: replace its term
          float x0, x1;
          upk2(add2(lg_eval2<D>(ep, y, d), nm), x0, x1);
          const float gn0 = ex2(fminf(x0, 100.0f)), gn1 = ex2(fminf(x1, 100.0f));
          upk2(add2(fma2(ga.x, bc2(-1.0f), sp), pk2(gn0, gn1)), sn0, sn1);
          sn0 = fmaxf(sn0, gn0);
          sn1 = fmaxf(sn1, gn1);
        } else {  // previous component removed
          upk2(fma2(ga.x, bc2(-1.0f), sp), sn0, sn1);
        }
        fix = !(sn0 * 64.0f >= so0 && sn1 * 64.0f >= so1);
        sp = pk2(sn0, sn1);
      }
      if (withL) {
        float s0, s1;
        upk2(sp, s0, s1);
        fix |= !(s0 > 1e-30f && s0 < 1e30f && s1 > 1e-30f && s1 < 1e30f);
      }
      float x0, x1;
      upk2(add2(lg_eval2<D>(ek, y, d), nm), x0, x1);
      f32x2 G = pk2(ex2(fminf(x0, 100.0f)), ex2(fminf(x1, 100.0f)));
      if (fix) {  // exact s_p with the largest term as the shift
        f32x2 dd[D];
        float m0 = -3.0e38f, m1 = -3.0e38f;
        for (int j2 = 0; j2 < K; ++j2) {
          float l0, l1;
          upk2(lg_eval2<D>(c.ec[j2], y, dd), l0, l1);
          m0 = fmaxf(m0, l0);
          m1 = fmaxf(m1, l1);
        }
        nm = pk2(-m0, -m1);
        sp = 0ull;
        for (int j2 = 0; j2 < K; ++j2) {
          upk2(add2(lg_eval2<D>(c.ec[j2], y, dd), nm), x0, x1);
          const f32x2 t = pk2(ex2(x0), ex2(x1));
          sp = add2(sp, t);
          if (j2 == k) G = t;
        }
      }
      GG2[2 * pp] = G;
      SM4[pp] = make_ulonglong2(sp, nm);
      float s0, s1, g0, g1;
      upk2(sp, s0, s1);
      upk2(G, g0, g1);
      if (withL) {
        float a0, a1, n0, n1;
        upk2(ga.y, a0, a1);
        upk2(nm, n0, n1);
        accl = fmaf(a0, (-n0 - c0) + lg2(s0), accl);
        accl = fmaf(a1, (-n1 - c0) + lg2(s1), accl);
      }
      const f32x2 rr = pk2(rcp_approx(max3f(s0, g0, 1e-30f)), rcp_approx(max3f(s1, g1, 1e-30f)));
      const f32x2 gam = mul2(ga.y, mul2(G, rr));
      acc[0] = add2(acc[0], gam);
      int t = 1 + D;
#pragma unroll
      for (int x = 0; x < D; ++x) {
        const f32x2 gd = mul2(gam, d[x]);
        acc[1 + x] = add2(acc[1 + x], gd);
#pragma unroll
        for (int yy = x; yy < D; ++yy, ++t) acc[t] = fma2(gd, d[yy], acc[t]);
      }
    }
    float v[NS + 1];
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      float lo, hi;
      upk2(acc[q], lo, hi);
      v[q] = lo + hi;
    }
    v[NS] = 0.0f;
    if (withL) {
      const double accw = warp_sum((double)accl);
      if (lane == 0) c.redL[wid] = accw;
    }
    block_partials<NS + 1, NRED, NW>(v, c.redf);
  };

  // ---- sweeps -------------------------------------------------------------
  // Every kExactEvery-th sweep starts with the exact pass (after the weights
  // are normalised); the others start with the first component step, which
  // also yields the log-likelihood of the previous sweep's parameters.
  constexpr int kExactEvery = 8;
  for (;;) {
    if (c.sweep % kExactEvery == 0) {
      if (c.sweep > 0) {
        if (tid < c.K) {
          const R un = c.u[tid] / c.Z;
          c.u[tid] = un;
          c.eb[tid] = lg2((float)un) + c.elc[tid];
          pack_econst<D>(c.emu[tid], c.eA[tid], c.eb[tid], c.ec[tid]);
        }
        __syncthreads();
        if (tid == 0) c.Z = (R)1;
        __syncthreads();
      }
      exact_pass(true, c.sweep == 0);
    } else {
      comp_pass(0, c.pstate, true);
    }
    if (tid < 32) {
      R sv[NS + 1];
      finish_exact(sv, false);
      if (lane == 0) {
        if (c.sweep > 0 && !c.annih && fabs(c.Ld - c.Ldprev) <= a.tol * fabs(c.Ldprev + c.Lbase))
          c.done = 1;
        else if (c.sweep >= a.max_sweeps)
          c.done = 2;
        c.Ldprev = c.Ld;
        if (!c.done) {
          c.sweep = c.sweep + 1;
          c.annih = 0;
          c.k = 0;
          c.pstate = 0;
        }
      }
      __syncwarp();
      if (!c.done) {
        if constexpr (sizeof(R) == 8)
          mstep64(0, sv);
        else if (lane == 0)
          mstep(0, sv);
      }
    }
    __syncthreads();
    if (c.done) break;
    while (c.k < c.K) {
      const int k = c.k;
      comp_pass(k, c.pstate, false);
      if (tid < 32) {
        R st[NW];
#pragma unroll
        for (int q = 0; q < NW; ++q) st[q] = lane < NS ? (R)c.redf[q][lane] : (R)0;
#pragma unroll
        for (int h = NW / 2; h >= 1; h >>= 1)
#pragma unroll
          for (int q = 0; q < h; ++q) st[q] += st[q + h];
        R sv[NS + 1];
#pragma unroll
        for (int q = 0; q < NS; ++q) sv[q] = __shfl_sync(0xffffffffu, st[0], q);
        sv[NS] = (R)0;
        if constexpr (sizeof(R) == 8)
          mstep64(k, sv);
        else if (lane == 0)
          mstep(k, sv);
      }
      __syncthreads();
    }
  }
  if (tid == 0 && c.done == 2) c.status |= GM_ST_EM_MAXSWEEPS;
  if constexpr (sizeof(R) == 4) {  // FP64 means from the hi + lo pairs
    if (tid < c.K)
      for (int x = 0; x < D; ++x) c.mu[tid][x] = (double)c.emu[tid][x] + (double)c.mulo[tid][x];
    __syncthreads();
  }

  // ---- final unpenalised step (Sec. 2.3.1), FP64 ---------------------------
  if (c.K == 1) {  // the final step of one component: the sample moments
    if (tid == 0) k1_closed_form<D, NT, R>(c);
    __syncthreads();
    write_cell<D, NT, R>(a, c, j, prm_out);
    return;
  }
  if (tid == 0) c.Kf = 0;
  __syncthreads();
  {
    const int K = c.K;
    const double nw = c.Nd / c.W;
    // Normaliser pass: per particle the shift m_p = max_j log2(u_j f_j) and
    // r_p = alpha_p (N / W) / S_p with S_p = sum_j 2^(log2(u_j f_j) - m_p)
    // summed in FP64.  r_p goes to the tile's s_p / m_p records (8 bytes per
    // particle there) and m_p to the first word of each particle's term
    // record; the weights in the second word stay for the last exact pass.
    // Every thread keeps its particles p = tid + i NT in all passes below, so
    // it reads back only what it wrote.  The component passes recompute
    // 2^(log2(u_k f_k) - m_p) with the same instructions on the same operands,
    // so sum_k gamma_pk = alpha_p N / W to FP64 rounding.
    double* Rd = reinterpret_cast<double*>(SMT);
    float* Mf = GAT;  // particle p at 4 (p >> 1) + (p & 1)
    for (int p = tid; p < N; p += NT) {
      float y[D], d[D];
#pragma unroll
      for (int q = 0; q < D; ++q) y[q] = Y[q * ys + p];
      float m = -3.0e38f;
      for (int jj = 0; jj < K; ++jj) m = fmaxf(m, lg_eval<D>(c.emu[jj], c.eA[jj], c.eb[jj], y, d));
      double Ssum = 0.0;
      for (int jj = 0; jj < K; ++jj)
        Ssum += (double)ex2(lg_eval<D>(c.emu[jj], c.eA[jj], c.eb[jj], y, d) - m);
      Rd[p] = a.alpha[off + p] * nw / Ssum;
      Mf[4 * (p >> 1) + (p & 1)] = m;
    }
    for (int k = 0; k < K; ++k) {
      double ck[D];
#pragma unroll
      for (int q = 0; q < D; ++q) ck[q] = c.mu[k][q] * c.sc[q];
      double acc[NS];
#pragma unroll
      for (int q = 0; q < NS; ++q) acc[q] = 0.0;
      for (int p = tid; p < N; p += NT) {
        float y[D], d[D];
#pragma unroll
        for (int q = 0; q < D; ++q) y[q] = Y[q * ys + p];
        const float m = Mf[4 * (p >> 1) + (p & 1)];
        const double gk = (double)ex2(lg_eval<D>(c.emu[k], c.eA[k], c.eb[k], y, d) - m);
        const double gam = Rd[p] * gk;
        double dv[D];
#pragma unroll
        for (int q = 0; q < D; ++q) dv[q] = (to_f64(vin[(int64_t)q * a.n + off + p]) - c.mean[q]) - ck[q];
        acc[0] += gam;
        int t = 1 + D;
#pragma unroll
        for (int x = 0; x < D; ++x) {
          const double gd = gam * dv[x];
          acc[1 + x] += gd;
#pragma unroll
          for (int yy = x; yy < D; ++yy, ++t) acc[t] += gd * dv[yy];
        }
      }
      block_sum_d<D, NT, NS, R>(c, acc);
      if (tid == 0 && c.res[0] > 0.0) {
        const int f = c.Kf;
        const double n = c.res[0];
        double dl[D];
        for (int x = 0; x < D; ++x) {
          dl[x] = c.res[1 + x] / n;
          c.fmu[f][x] = ck[x] + dl[x];
        }
        int t = 0;
        for (int x = 0; x < D; ++x)
          for (int yy = x; yy < D; ++yy, ++t) c.fS[f][t] = c.res[1 + D + t] / n - dl[x] * dl[yy];
        c.fw[f] = n / c.Nd;
        c.Kf = f + 1;
      }
      __syncthreads();
    }
  }
  // ---- final parameters: E constants, Cholesky floor, eq. (lnL-GM) -------
  if (tid == 0) {
    const int Kf = c.Kf;
    int pd = 1;
    double one[D];
    for (int d = 0; d < D; ++d) one[d] = 1.0;
    for (int k = 0; k < Kf; ++k) {
      // floor test in the original coordinates
      double So[NM], mo[D], Lo[3][3];
      for (int q = 0; q < NM; ++q) So[q] = c.fS[k][q];
      for (int d = 0; d < D; ++d) mo[d] = 0.0;
      double meano[D];
      for (int d = 0; d < D; ++d) meano[d] = c.mean[d] + c.fmu[k][d];
      if (!chol_whitened<D, double, double>(So, mo, meano, one, Lo)) pd = 0;
      // whitened copy for the likelihood pass
      double Sw[NM], mw[D], Lw[3][3];
      for (int x = 0; x < D; ++x) {
        mw[x] = c.fmu[k][x] * c.isc[x];
        for (int yy = x; yy < D; ++yy) Sw[tri<D>(x, yy)] = c.fS[k][tri<D>(x, yy)] * c.isc[x] * c.isc[yy];
      }
      double rw[3];
      if (chol_whitened<D, double, double>(Sw, mw, c.mean, c.sc, Lw, rw)) {
        float eA[NM], elc;
        make_econst<D, double>(Lw, rw, eA, elc);
        for (int q = 0; q < NM; ++q) c.eA[k][q] = eA[q];
        c.elc[k] = elc;
      } else {
        pd = 0;
      }
      for (int x = 0; x < D; ++x) c.emu[k][x] = (float)mw[x];
      c.eb[k] = lg2((float)c.fw[k]) + c.elc[k];
      c.u[k] = (R)c.fw[k];
      pack_econst<D>(c.emu[k], c.eA[k], c.eb[k], c.ec[k]);
    }
    if (!pd) c.status |= GM_ST_COV_NOT_PD;
    c.final_pd = pd;
    c.K = Kf;
    c.Z = (R)1;
  }
  __syncthreads();
  if (c.final_pd) {
    exact_pass(false, true);
    if (tid < 32) {
      R sv[NS + 1];
      finish_exact(sv, true);
    }
    __syncthreads();
  }
  write_cell<D, NT, R>(a, c, j, prm_out);
  (void)NW;
}

// ---------------------------------------------------------------------------
// the kernel: work queue, per-cell moments, degenerate cells, dispatch of
// the cell body on the shared or the global tile
// ---------------------------------------------------------------------------
template <int D, int NT, typename VT, typename R>
__global__ void __launch_bounds__(NT, (D == 1 ? 1024 : 512) / NT) em_kernel(EmParams a) {
  constexpr int NW = NT / 32;
  constexpr int NM = D * (D + 1) / 2;
  constexpr int P = 1 + D + NM;
  __shared__ EmCtl<D, NW, R> c;
  extern __shared__ __align__(16) float tile_smem[];
  const int tid = threadIdx.x;
  const VT* __restrict__ vin = static_cast<const VT*>(a.v);

  for (;;) {
    if (tid == 0) {
      const unsigned int t = atomicAdd(a.queue, 1u);
      c.cell = a.list ? (t < *a.list_count ? (int64_t)a.list[t] : a.C) : (int64_t)t;
    }
    __syncthreads();
    const int64_t j = c.cell;
    if (j >= a.C) break;
    const int64_t off = a.cell_off[j];
    const int N = (int)(a.cell_off[j + 1] - off);
    double* prm_out = a.params_out + (size_t)j * a.Kmax * P;

    // ---- total weight, mean and covariance (FP64, one pass) ----------------
    // sums of alpha, alpha d and alpha d d^T with d = v - s, s the cell's
    // first particle (d is exact in FP64, and s lies within the cell's
    // spread, so mean = s + sum(alpha d) / W and cov = sum(alpha d d^T) / W
    // - (mean - s)(mean - s)^T lose no more than a few ulps to cancellation)
    {
      double sh[D];
#pragma unroll
      for (int d = 0; d < D; ++d) sh[d] = N > 0 ? to_f64(vin[(int64_t)d * a.n + off]) : 0.0;
      double acc[1 + D + NM];
#pragma unroll
      for (int i = 0; i < 1 + D + NM; ++i) acc[i] = 0.0;
      for (int p = tid; p < N; p += NT) {
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
      block_sum_d<D, NT, 1 + D + NM, R>(c, acc);
      if (tid == 0) {
        c.W = c.res[0];
        c.Nd = (double)N;
        c.status = (N <= 10) ? GM_ST_TOO_FEW : 0u;
        const double rW = 1.0 / c.res[0];
        double dm[D];
        for (int d = 0; d < D; ++d) {
          dm[d] = c.res[1 + d] * rW;
          c.mean[d] = sh[d] + dm[d];
        }
        double cov[NM];
        int t = 0;
        for (int x = 0; x < D; ++x)
          for (int y = x; y < D; ++y, ++t) cov[t] = fma(-dm[x], dm[y], c.res[1 + D + t] * rW);
        c.degenerate = 0;
        if (N == 0 || !(c.W > 0.0)) {
          c.degenerate = 2;  // empty: handled below
        } else {
          // degenerate cell: the total covariance fails the Cholesky floor
          // 1e-13 * sum_d (cov_dd + mean_d^2)
          double scale2 = 0.0;
          for (int d = 0; d < D; ++d) scale2 += cov[tri<D>(d, d)] + c.mean[d] * c.mean[d];
          const double fl = 1e-13 * scale2;
          bool ok = true;
          double L2[3][3] = {{0}};
          for (int x = 0; x < D && ok; ++x)
            for (int y = 0; y <= x && ok; ++y) {
              double sv = cov[tri<D>(y, x)];
              for (int m = 0; m < y; ++m) sv -= L2[x][m] * L2[y][m];
              if (x == y) {
                if (!(sv > fl) || !(sv < 1e300)) ok = false;
                else L2[x][x] = sqrt(sv);
              } else {
                L2[x][y] = sv / L2[y][y];
              }
            }
          c.degenerate = ok ? 0 : 1;
          if (c.degenerate) {
            for (int i = 0; i < NM; ++i) c.fS[0][i] = cov[i];
          } else {
            for (int i = 0; i < NM; ++i) c.cov0[i] = cov[i];
            c.logN = log(c.Nd);
            double prod = 1.0;
            for (int d = 0; d < D; ++d) {
              c.sc[d] = sqrt(cov[tri<D>(d, d)]);
              c.isc[d] = 1.0 / c.sc[d];
              prod *= c.sc[d];
              c.meanf[d] = (float)c.mean[d];
              c.scf[d] = (float)c.sc[d];
            }
            c.logjac = log(prod);
            // whitened total covariance (correlation matrix) for the init
            for (int x = 0; x < D; ++x)
              for (int y = x; y < D; ++y)
                c.S0[tri<D>(x, y)] = (x == y) ? 1.0 : cov[tri<D>(x, y)] * c.isc[x] * c.isc[y];
          }
        }
      }
      __syncthreads();
    }
    if (c.degenerate == 2) {
      for (int i = tid; i < a.Kmax * P; i += NT) prm_out[i] = 0.0;
      if (tid == 0) {
        a.K_out[j] = 0;
        a.W_out[j] = N == 0 ? 0.0 : c.W;
        a.lnL_out[j] = 0.0;
        if (a.sweeps_out) a.sweeps_out[j] = 0;
        if (a.kwork_out) a.kwork_out[j] = 0;
        a.status_out[j] = N == 0 ? GM_ST_EMPTY : (GM_ST_EMPTY | GM_ST_DEGENERATE);
      }
      __syncthreads();
      continue;
    }
    if (c.degenerate) {
      for (int i = tid; i < a.Kmax * P; i += NT) prm_out[i] = 0.0;
      __syncthreads();
      if (tid == 0) {
        prm_out[0] = 1.0;
        for (int d = 0; d < D; ++d) prm_out[1 + d] = c.mean[d];
        for (int i = 0; i < NM; ++i) prm_out[1 + D + i] = c.fS[0][i];
        a.K_out[j] = 1;
        a.W_out[j] = c.W;
        a.lnL_out[j] = 0.0;
        if (a.sweeps_out) a.sweeps_out[j] = 0;
        if (a.kwork_out) a.kwork_out[j] = 0;
        a.status_out[j] = c.status | GM_ST_DEGENERATE | GM_ST_COV_NOT_PD;
      }
      __syncthreads();
      continue;
    }
    if (tid == 0) c.K = 0;
    __syncthreads();
    if (N + (N & 1) <= a.cap) {
      em_cell_body<D, NT, VT, R>(a, c, j, off, N, tile_smem, a.cap, tile_smem + D * a.cap,
                                 tile_smem + (D + 2) * a.cap);
    } else {
      const int64_t o = scratch_offset(off, j), ss = a.scratch_stride;
      em_cell_body<D, NT, VT, R>(a, c, j, off, N, a.scratch + o, (int)ss,
                                 a.scratch + D * ss + 2 * o, a.scratch + (D + 2) * ss + 2 * o);
    }
  }
}

}  // namespace gmcr
