// std_kernel.cuh -- standard (non-adaptive) EM with K-means initialisation
// and Anderson acceleration: the acceleration study of Sec. 4, where the
// paper applies both to the non-adaptive EM-GM algorithm.
//
// One CTA fits one cell at a time (persistent, atomic cell ticket).  The
// cell is staged once as whitened FP32 velocities and normalised weights
// (shared tile, or an L2-resident global tile for cells over the tile).
//
//   * K-means (Lloyd) from the paper's random particles: assignment on the
//     FP32 coordinates (squared distance with fmaf in dimension order, the
//     lowest index on ties), centre sums in 64-bit fixed point (2^-40:
//     exact, so the result does not depend on the order of the sums).
//   * Standard EM iteration: an exact pass gives each particle's normaliser
//     and the log-likelihood L(theta_i); one pass per component gives its
//     E-step statistics (no barrier between components); the M-step of all
//     components runs on one lane each (eq. omegak-mle), in FP32 with the
//     mean's shift added to the FP64 iterate and the covariance floor
//     retested in FP64 near the floor: FP64 on warp 0 between barriers
//     stalls the CTA (GB300's FP64 pipe is narrow and shared by the SM).
//   * Anderson acceleration (FP64, warp 0) on theta = (omega_k, mu_k,
//     M2_k = Sigma_k + mu_k mu_k^T) in the cell's whitened coordinates,
//     started once the relative change of L is at most 1e-4, reset when an
//     extrapolation has a non-positive weight or an indefinite covariance.
//   * Penalised variant (mml): the same simultaneous iteration with the
//     weights of eq. (omegak) from every component's N_k, annihilation of
//     components with N_k - T/2 <= 0 (never the last), convergence of the
//     penalised L (eq. lnL-GM) over an iteration without annihilation.
//   * Output: one standard EM step from the last iterate, entirely in FP64
//     (FP64-normalised responsibilities), which makes the moments exact.
#pragma once

#include "em_kernel.cuh"

namespace gmcr {

struct StdParams {
  int64_t C, n;
  const int64_t* cell_off;
  const void* v;
  const double* alpha;
  int32_t* K_out;
  double* params_out;
  double* W_out;
  double* lnL_out;
  int32_t* iters_out;
  int32_t* aa_steps_out;
  int32_t* aa_resets_out;
  int32_t* km_out;
  uint32_t* status_out;
  float* scratch;
  int64_t scratch_stride;
  unsigned int* queue;
  int Kmax, max_sweeps, cap, init, aa_m, km_iters;
  int mml;  // 1: simultaneous penalised EM with annihilation (eq. omegak)
  double tol;
  uint64_t seed;
};

constexpr int kStdMaxM = 8;            // Anderson memory, at most
constexpr double kAAStart = 1e-4;      // AA starts when |dL| <= kAAStart |L|
constexpr double kFix = 1099511627776.0;  // 2^40: fixed point of the K-means sums

// Anderson state (Walker & Ni 2011, type II): the iterate x, G(x), the
// extrapolation, the previous (f, G) pair and the last h <= m differences,
// kept in a ring of m slots (the oldest at slot head) with their Gram
// matrix, which only gains the newest column's row each step
template <int MAXN>
struct AAState {
  double th[MAXN], tg[MAXN], tn[MAXN], fprev[MAXN], gprev[MAXN];
  double dF[kStdMaxM][MAXN], dG[kStdMaxM][MAXN];
  double gram[kStdMaxM][kStdMaxM], rhs[kStdMaxM], gam[kStdMaxM];
  double A[kStdMaxM][kStdMaxM + 1], z[kStdMaxM];  // the small system, logical order
  int h, have, head;
};

// 1/t for t > 0 in FP64: an FP32 estimate of the mantissa's reciprocal
// (t = m 2^e, so any t gets one) refined by two Newton steps
// y <- y (2 - t y) (each doubles the correct bits: ~2^-22 -> 2^-44 -> below
// FP64 rounding)
__device__ __forceinline__ double rcp_nr_d(double t) {
  int ex;
  const double m = frexp(t, &ex);
  double y = ldexp((double)rcp_approx((float)m), -ex);
  y = y * (2.0 - t * y);
  return y * (2.0 - t * y);
}

// One Anderson step by a whole warp (FP64): f = G(x) - x; the difference
// with the previous pair joins the history (the oldest dropped beyond m);
// gamma from (dF^T dF + 1e-12 max diag I) gamma = dF^T f; tn = G(x) - dG
// gamma.  The history is a ring of m slots (the oldest at head) whose Gram
// matrix gains the newest column's row each step; the step's dot products
// (dF^T f and the new column against every column) are summed per lane in
// one pass and reduced together; the h x h system is solved by Gaussian
// elimination without pivoting (it is symmetric positive definite), one
// row per lane, columns oldest first.  Returns true if the extrapolation
// was made (tn valid); false with no history or a pivot that is not
// positive.  Reads s.th, s.tg (n values); the caller syncs the warp before
// and after; h = 0 clears the history.
template <int MAXN>
__device__ bool aa_warp_step(AAState<MAXN>& s, int n, int m) {
  const int lane = threadIdx.x & 31;
  int h = s.h, head = h > 0 ? s.head : 0, nw = -1;
  if (m > 0 && s.have) {
    if (h == m) {  // drop the oldest: its slot takes the new column
      head = head + 1 == m ? 0 : head + 1;
      --h;
    }
    nw = head + h;
    nw = nw >= m ? nw - m : nw;
    for (int i = lane; i < n; i += 32) {
      s.dF[nw][i] = (s.tg[i] - s.th[i]) - s.fprev[i];
      s.dG[nw][i] = s.tg[i] - s.gprev[i];
    }
    ++h;
  }
  for (int i = lane; i < n; i += 32) {
    s.fprev[i] = s.tg[i] - s.th[i];
    s.gprev[i] = s.tg[i];
  }
  __syncwarp();
  if (lane == 0) {
    s.h = h;
    s.head = head;
    s.have = 1;
  }
  __syncwarp();
  if (h == 0) return false;
  auto slot = [&](int a) {
    const int q = head + a;
    return q >= m ? q - m : q;
  };
  double part[2 * kStdMaxM];
#pragma unroll
  for (int a = 0; a < 2 * kStdMaxM; ++a) part[a] = 0.0;
  for (int i = lane; i < n; i += 32) {
    const double fi = s.fprev[i], di = s.dF[nw][i];
#pragma unroll
    for (int a = 0; a < kStdMaxM; ++a)
      if (a < h) {
        const double v = s.dF[slot(a)][i];
        part[a] = fma(v, fi, part[a]);
        part[kStdMaxM + a] = fma(v, di, part[kStdMaxM + a]);
      }
  }
  warp_rs_d<2 * kStdMaxM>(part, lane);
  if ((lane & 1) == 0) {
    const int q = warp_rs_index<2 * kStdMaxM>(lane);
    const int a = q < kStdMaxM ? q : q - kStdMaxM;
    if (a < h) {
      const int sa = slot(a);
      if (q < kStdMaxM) {
        s.rhs[sa] = part[0];
      } else {
        s.gram[nw][sa] = part[0];
        s.gram[sa][nw] = part[0];
      }
    }
  }
  __syncwarp();
  double dmax = lane < h ? s.gram[slot(lane)][slot(lane)] : 0.0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
  if (!(dmax > 0.0)) return false;
  if (lane < h) {
    const int sl = slot(lane);
    for (int b = 0; b < h; ++b) s.A[lane][b] = s.gram[sl][slot(b)] + (b == lane ? 1e-12 * dmax : 0.0);
    s.A[lane][kStdMaxM] = s.rhs[sl];
  }
  __syncwarp();
  double myr = 0.0;
  for (int j = 0; j < h; ++j) {
    const double d = s.A[j][j];
    if (!(d > 0.0) || !(d < 1e300)) return false;  // the same on every lane
    const double rd = rcp_nr_d(d);
    if (lane == j) myr = rd;
    if (lane > j && lane < h) {
      const double f = s.A[lane][j] * rd;
      for (int b = j + 1; b < h; ++b) s.A[lane][b] = fma(-f, s.A[j][b], s.A[lane][b]);
      s.A[lane][kStdMaxM] = fma(-f, s.A[j][kStdMaxM], s.A[lane][kStdMaxM]);
    }
    __syncwarp();
  }
  for (int j = h - 1; j >= 0; --j) {
    if (lane == j) {
      double t = s.A[j][kStdMaxM];
      for (int b = j + 1; b < h; ++b) t = fma(-s.A[j][b], s.z[b], t);
      s.z[j] = t * myr;
    }
    __syncwarp();
  }
  if (lane < h) s.gam[slot(lane)] = s.z[lane];
  __syncwarp();
  for (int i = lane; i < n; i += 32) {
    double t = s.tg[i];
    for (int a = 0; a < h; ++a) {
      const int sa = slot(a);
      t = fma(-s.dG[sa][i], s.gam[sa], t);
    }
    s.tn[i] = t;
  }
  __syncwarp();
  return true;
}

template <int D, int NW>
struct StdCtl {
  static constexpr int NM = D * (D + 1) / 2;
  static constexpr int NS = 1 + D + NM;
  static constexpr int P = 1 + D + NM;
  static constexpr int NTH = kMaxK * P;
  static constexpr int NRED = pow2_at_least(NS);
  // the cell
  double mean[D], sc[D], isc[D], S0[NM];
  float meanf[D], scf[D], rsumAH;  // FP32 copies for the iteration's M-steps
  double W, Nd, sumAH, logjac, L, Lprev;
  float c0;
  int64_t cell;
  unsigned int status;
  int K, degenerate, it, done, aa_on, naa, nreset, kmp, Kg, ann;
  int picks[kMaxK];
  // mixture in whitened coordinates (FP64 masters) and its M-step update
  double w[kMaxK], mu[kMaxK][D], S[kMaxK][NM];
  double gw[kMaxK], gmu[kMaxK][D], gS[kMaxK][NM];
  int gok[kMaxK];
  // FP32 E-step constants: log2(omega f) = eb - |eA (y - emu)|^2
  float emu[kMaxK][D], eA[kMaxK][NM], eb[kMaxK];
  // reductions
  float redk[kMaxK][NW][NRED];
  float redl[NW];
  double redd[NW][NS + 1];
  double res[NS + 1];
  // K-means
  float kc[kMaxK][D];
  unsigned long long kacc[kMaxK][1 + D + NM];
  // Anderson
  AAState<NTH> aa;
  // final step
  double fw[kMaxK], fmu[kMaxK][D], fS[kMaxK][NM];
  int Kf;
};

// FP64 block sum of NV values (result in c.res)
template <int D, int NW, int NV>
__device__ __forceinline__ void std_bsum(StdCtl<D, NW>& c, double (&v)[NV]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) c.redd[w][i] = v[i];
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
    for (int q = 0; q < NW; ++q) s += c.redd[q][threadIdx.x];
    c.res[threadIdx.x] = s;
  }
  __syncthreads();
}

// E-step constants of component k from its FP64 whitened (w, mu, S);
// false if the covariance fails the Cholesky floor (original coordinates)
// The covariance floor test of the iteration (FP64 S, mu in whitened
// coordinates): FP32 first, accepted only if every pivot clears 1e-6 of the
// floor's scale (far above FP32 rounding); otherwise FP64 with the floor
// itself (1e-13), as the oracle has it.  Factors returned in FP32 (the
// E-step's precision).
template <int D>
__device__ bool std_chol(const double* S, const double* mu, const double* mean, const double* sc,
                         const float* meanf, const float* scf, float (&Lc)[3][3], float (&ri)[3]) {
  constexpr int NM = D * (D + 1) / 2;
  float Sf[NM], muf[D];
  for (int q = 0; q < NM; ++q) Sf[q] = (float)S[q];
  for (int d = 0; d < D; ++d) muf[d] = (float)mu[d];
  if (chol_whitened<D, float, float>(Sf, muf, meanf, scf, Lc, ri, 1e-6)) return true;
  double L64[3][3], r64[3];
  if (!chol_whitened<D, double, double>(S, mu, mean, sc, L64, r64)) return false;
  for (int i = 0; i < D; ++i) {
    ri[i] = (float)r64[i];
    for (int j = 0; j <= i; ++j) Lc[i][j] = (float)L64[i][j];
  }
  return true;
}

template <int D, int NW>
__device__ bool std_econst(StdCtl<D, NW>& c, int k) {
  constexpr int NM = D * (D + 1) / 2;
  float Lc[3][3], ri[3], muf[D];
  for (int d = 0; d < D; ++d) muf[d] = (float)c.mu[k][d];
  if (!std_chol<D>(c.S[k], c.mu[k], c.mean, c.sc, c.meanf, c.scf, Lc, ri)) return false;
  float eA[NM], elc;
  make_econst<D, float>(Lc, ri, eA, elc);
  for (int q = 0; q < NM; ++q) c.eA[k][q] = eA[q];
  for (int d = 0; d < D; ++d) c.emu[k][d] = muf[d];
  c.eb[k] = lg2((float)c.w[k]) + elc;
  return true;
}

// component k of theta (whitened) -> (w, mu, M2 upper triangle)
template <int D, int NW>
__device__ __forceinline__ void std_pack(const double* w, const double (*mu)[D],
                                         const double (*S)[D * (D + 1) / 2], int k, double* th) {
  constexpr int P = 1 + D + D * (D + 1) / 2;
  double* t = th + k * P;
  t[0] = w[k];
  for (int d = 0; d < D; ++d) t[1 + d] = mu[k][d];
  int q = 0;
  for (int x = 0; x < D; ++x)
    for (int y = x; y < D; ++y, ++q) t[1 + D + q] = S[k][q] + mu[k][x] * mu[k][y];
}

template <int D, int NT, typename VT>
__global__ void __launch_bounds__(NT, (D == 1 ? 1024 : 512) / NT) std_kernel(StdParams a) {
  constexpr int NW = NT / 32;
  using Ctl = StdCtl<D, NW>;
  constexpr int NM = Ctl::NM, NS = Ctl::NS, P = Ctl::P, NRED = Ctl::NRED;
  constexpr int T = D * (D + 3) / 2;
  __shared__ Ctl c;
  extern __shared__ __align__(16) float tile_smem[];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const VT* __restrict__ vin = static_cast<const VT*>(a.v);

  for (;;) {
    if (tid == 0) c.cell = (int64_t)atomicAdd(a.queue, 1u);
    __syncthreads();
    const int64_t j = c.cell;
    if (j >= a.C) break;
    const int64_t off = a.cell_off[j];
    const int N = (int)(a.cell_off[j + 1] - off);
    double* prm_out = a.params_out + (size_t)j * a.Kmax * P;

    // ---- total weight and weighted mean (FP64) ----------------------------
    {
      double acc[1 + D];
#pragma unroll
      for (int i = 0; i <= D; ++i) acc[i] = 0.0;
      for (int p = tid; p < N; p += NT) {
        const double al = a.alpha[off + p];
        acc[0] += al;
#pragma unroll
        for (int d = 0; d < D; ++d) acc[1 + d] += al * (double)vin[(int64_t)d * a.n + off + p];
      }
      std_bsum<D, NW, 1 + D>(c, acc);
      if (tid == 0) {
        c.W = c.res[0];
        c.Nd = (double)N;
        for (int d = 0; d < D; ++d) c.mean[d] = c.res[1 + d] / c.res[0];
      }
      __syncthreads();
    }
    if (N == 0 || !(c.W > 0.0)) {
      for (int i = tid; i < a.Kmax * P; i += NT) prm_out[i] = 0.0;
      if (tid == 0) {
        a.K_out[j] = 0;
        a.W_out[j] = N == 0 ? 0.0 : c.W;
        a.lnL_out[j] = 0.0;
        if (a.iters_out) a.iters_out[j] = 0;
        if (a.aa_steps_out) a.aa_steps_out[j] = 0;
        if (a.aa_resets_out) a.aa_resets_out[j] = 0;
        if (a.km_out) a.km_out[j] = 0;
        a.status_out[j] = N == 0 ? GM_ST_EMPTY : (GM_ST_EMPTY | GM_ST_DEGENERATE);
      }
      __syncthreads();
      continue;
    }
    // ---- total covariance (two-pass, FP64) --------------------------------
    {
      double acc[NM];
#pragma unroll
      for (int i = 0; i < NM; ++i) acc[i] = 0.0;
      for (int p = tid; p < N; p += NT) {
        const double al = a.alpha[off + p];
        double dv[D];
#pragma unroll
        for (int d = 0; d < D; ++d) dv[d] = (double)vin[(int64_t)d * a.n + off + p] - c.mean[d];
        int t = 0;
#pragma unroll
        for (int x = 0; x < D; ++x)
#pragma unroll
          for (int y = x; y < D; ++y, ++t) acc[t] += al * dv[x] * dv[y];
      }
      std_bsum<D, NW, NM>(c, acc);
      if (tid == 0) {
        double cov[NM];
        for (int i = 0; i < NM; ++i) cov[i] = c.res[i] / c.W;
        c.status = (N <= 10) ? GM_ST_TOO_FEW : 0u;
        double scale2 = 0.0;
        for (int d = 0; d < D; ++d) scale2 += cov[tri<D>(d, d)] + c.mean[d] * c.mean[d];
        const double fl = 1e-13 * scale2;
        bool ok = true;
        double L2[3][3] = {{0}};
        for (int x = 0; x < D && ok; ++x)
          for (int y = 0; y <= x && ok; ++y) {
            double s = cov[tri<D>(y, x)];
            for (int m = 0; m < y; ++m) s -= L2[x][m] * L2[y][m];
            if (x == y) {
              if (!(s > fl) || !(s < 1e300)) ok = false;
              else L2[x][x] = sqrt(s);
            } else {
              L2[x][y] = s / L2[y][y];
            }
          }
        c.degenerate = ok ? 0 : 1;
        if (c.degenerate) {
          for (int i = 0; i < NM; ++i) c.S0[i] = cov[i];
        } else {
          c.logjac = 0.0;
          for (int d = 0; d < D; ++d) {
            c.sc[d] = sqrt(cov[tri<D>(d, d)]);
            c.isc[d] = 1.0 / c.sc[d];
            c.meanf[d] = (float)c.mean[d];
            c.scf[d] = (float)c.sc[d];
            c.logjac += log(c.sc[d]);
          }
          for (int x = 0; x < D; ++x)
            for (int y = x; y < D; ++y)
              c.S0[tri<D>(x, y)] = (x == y) ? 1.0 : cov[tri<D>(x, y)] * c.isc[x] * c.isc[y];
        }
      }
      __syncthreads();
    }
    if (c.degenerate) {
      for (int i = tid; i < a.Kmax * P; i += NT) prm_out[i] = 0.0;
      __syncthreads();
      if (tid == 0) {
        prm_out[0] = 1.0;
        for (int d = 0; d < D; ++d) prm_out[1 + d] = c.mean[d];
        for (int i = 0; i < NM; ++i) prm_out[1 + D + i] = c.S0[i];
        a.K_out[j] = 1;
        a.W_out[j] = c.W;
        a.lnL_out[j] = 0.0;
        if (a.iters_out) a.iters_out[j] = 0;
        if (a.aa_steps_out) a.aa_steps_out[j] = 0;
        if (a.aa_resets_out) a.aa_resets_out[j] = 0;
        if (a.km_out) a.km_out[j] = 0;
        a.status_out[j] = c.status | GM_ST_DEGENERATE | GM_ST_COV_NOT_PD;
      }
      __syncthreads();
      continue;
    }

    // ---- staging: whitened FP32 velocities and normalised weights ---------
    float *Y, *AH, *SS, *MM;
    int ys;
    if (N <= a.cap) {
      Y = tile_smem;
      ys = a.cap;
    } else {
      Y = a.scratch + scratch_offset(off, j);
      ys = (int)a.scratch_stride;
    }
    AH = Y + D * ys;
    SS = Y + (D + 1) * ys;
    MM = Y + (D + 2) * ys;
    {
      const double nw = c.Nd / c.W;
      double sa[1] = {0.0};
      for (int p = tid; p < N; p += NT) {
#pragma unroll
        for (int d = 0; d < D; ++d)
          Y[d * ys + p] = (float)(((double)vin[(int64_t)d * a.n + off + p] - c.mean[d]) * c.isc[d]);
        const float ah = (float)(a.alpha[off + p] * nw);
        AH[p] = ah;
        sa[0] += (double)ah;
      }
      std_bsum<D, NW, 1>(c, sa);
      if (tid == 0) {
        c.sumAH = c.res[0];
        c.rsumAH = (float)(1.0 / c.res[0]);
        c.c0 = -2.0471975511965976f * D;
      }
    }
    // ---- the paper's random picks (Sec. 2.3), K = min(Kmax, N) -------------
    if (tid == 0) {
      int K = a.Kmax < N ? a.Kmax : N;
      if (a.mml)
        while (K > 1 && c.Nd - 0.5 * (double)T * K <= 0.0) --K;
      int got = 0;
      for (uint32_t t = 0; got < K; ++t) {
        int idx;
        if (t < 100000u) {
          const u32x4 r = philox_draw(a.seed, t, kTagInit, j);
          idx = (int)floor(uniform52(r.x, r.y) * c.Nd);
          if (idx >= N) idx = N - 1;
        } else {
          idx = 0;
          for (;;) {
            bool used = false;
            for (int m = 0; m < got; ++m) used |= (c.picks[m] == idx);
            if (!used) break;
            ++idx;
          }
        }
        bool dup = false;
        for (int m = 0; m < got; ++m) dup |= (c.picks[m] == idx);
        if (!dup) c.picks[got++] = idx;
      }
      c.K = K;
      c.kmp = 0;
      c.naa = 0;
      c.nreset = 0;
      c.aa_on = 0;
      c.ann = 0;
      c.aa.h = 0;
      c.aa.have = 0;
    }
    __syncthreads();

    if (a.init == 1) {
      // ---- K-means (Lloyd) on the staged coordinates ------------------------
      const int K = c.K;
      int* AS = reinterpret_cast<int*>(SS);
      if (tid < K * D) c.kc[tid / D][tid % D] = Y[(tid % D) * ys + c.picks[tid / D]];
      const int iters = a.km_iters > 0 ? a.km_iters : 100;
      int it;
      for (it = 0; it < iters; ++it) {
        for (int i = tid; i < K * (1 + D); i += NT) c.kacc[i / (1 + D)][i % (1 + D)] = 0ull;
        __syncthreads();
        int changed = 0;
        for (int p = tid; p < N; p += NT) {
          float y[D];
#pragma unroll
          for (int d = 0; d < D; ++d) y[d] = Y[d * ys + p];
          int best = 0;
          float bd = 0.0f;
          for (int k = 0; k < K; ++k) {
            const float d0 = y[0] - c.kc[k][0];
            float dist = d0 * d0;
            if (D == 3) {
              const float d1 = y[1] - c.kc[k][1], d2 = y[2] - c.kc[k][2];
              dist = fmaf(d2, d2, fmaf(d1, d1, d0 * d0));
            }
            if (k == 0 || dist < bd) {
              bd = dist;
              best = k;
            }
          }
          if (it == 0 || AS[p] != best) changed = 1;
          AS[p] = best;
          const double af = (double)AH[p];
          atomicAdd(&c.kacc[best][0], (unsigned long long)llrint(af * kFix));
#pragma unroll
          for (int d = 0; d < D; ++d)
            atomicAdd(&c.kacc[best][1 + d], (unsigned long long)llrint(af * (double)y[d] * kFix));
        }
        const int any = __syncthreads_or(changed);
        if (it > 0 && !any) break;
        if (tid < K) {
          const double A = (double)(long long)c.kacc[tid][0];
          if (A > 0.0)
            for (int d = 0; d < D; ++d)
              c.kc[tid][d] = (float)((double)(long long)c.kacc[tid][1 + d] / A);
        }
        __syncthreads();
      }
      if (tid == 0) c.kmp = it < iters ? it + 1 : iters;
      // cluster means (from the last pass's sums) and covariances
      for (int i = tid; i < K * NM; i += NT) c.kacc[i / NM][1 + D + i % NM] = 0ull;
      __syncthreads();
      if (tid < K) {
        const double A = (double)(long long)c.kacc[tid][0];
        for (int d = 0; d < D; ++d)
          c.mu[tid][d] = A > 0.0 ? (double)(long long)c.kacc[tid][1 + d] / A : 0.0;
      }
      __syncthreads();
      for (int p = tid; p < N; p += NT) {
        const int k = AS[p];
        const double af = (double)AH[p];
        double dy[D];
#pragma unroll
        for (int d = 0; d < D; ++d) dy[d] = (double)Y[d * ys + p] - c.mu[k][d];
        int q = 0;
#pragma unroll
        for (int x = 0; x < D; ++x)
#pragma unroll
          for (int y = x; y < D; ++y, ++q)
            atomicAdd(&c.kacc[k][1 + D + q], (unsigned long long)llrint(af * dy[x] * dy[y] * kFix));
      }
      __syncthreads();
      if (tid == 0) {
        int Ko = 0;
        for (int k = 0; k < K; ++k) {
          const double A = (double)(long long)c.kacc[k][0];
          if (!(A > 0.0)) continue;
          c.w[Ko] = A / kFix / c.Nd;
          for (int d = 0; d < D; ++d) c.mu[Ko][d] = c.mu[k][d];
          for (int q = 0; q < NM; ++q) c.S[Ko][q] = (double)(long long)c.kacc[k][1 + D + q] / A;
          double Lc[3][3], ri[3];
          if (!chol_whitened<D, double, double>(c.S[Ko], c.mu[Ko], c.mean, c.sc, Lc, ri))
            for (int q = 0; q < NM; ++q) c.S[Ko][q] = c.S0[q];
          ++Ko;
        }
        c.K = Ko;
      }
      __syncthreads();
    } else {
      if (tid < c.K) {
        const int k = tid;
        c.w[k] = 1.0 / (double)c.K;
        for (int d = 0; d < D; ++d)
          c.mu[k][d] = ((double)vin[(int64_t)d * a.n + off + c.picks[k]] - c.mean[d]) * c.isc[d];
        for (int q = 0; q < NM; ++q) c.S[k][q] = c.S0[q];
      }
      __syncthreads();
    }
    if (tid < c.K) std_econst<D, NW>(c, tid);
    if (tid == 0) {
      c.done = 0;
      c.it = 0;
    }
    __syncthreads();

    // ---- standard EM iterations (with Anderson acceleration) ---------------
    for (;;) {
      const int K = c.K;
      const float c0 = c.c0;
      // exact pass: m_p = max_k log2(omega_k f_k) and s_p = sum_k 2^(l_k - m_p)
      // in one evaluation per component (a new maximum rescales the running
      // sum), R_p = ah_p / s_p for the component passes, and the
      // log-likelihood
      {
        float accl = 0.0f;
        for (int p = tid; p < N; p += NT) {
          float y[D], dd[D];
#pragma unroll
          for (int d = 0; d < D; ++d) y[d] = Y[d * ys + p];
          float m = -3.0e38f, s = 0.0f;
          for (int k = 0; k < K; ++k) {
            const float l = lg_eval<D>(c.emu[k], c.eA[k], c.eb[k], y, dd);
            if (l > m) {
              s = fmaf(s, ex2(m - l), 1.0f);
              m = l;
            } else {
              s += ex2(l - m);
            }
          }
          const float ah = AH[p];
          SS[p] = ah * rcp_approx(s);
          MM[p] = m;
          accl = fmaf(ah, (m - c0) + lg2(s), accl);
        }
        accl = warp_sum(accl);
        if (lane == 0) c.redl[wid] = accl;
      }
      __syncthreads();
      // one pass per component: its E-step statistics about its FP32 mean
      for (int k = 0; k < K; ++k) {
        float acc[NRED];
#pragma unroll
        for (int q = 0; q < NRED; ++q) acc[q] = 0.0f;
        for (int p = tid; p < N; p += NT) {
          float y[D], dd[D];
#pragma unroll
          for (int d = 0; d < D; ++d) y[d] = Y[d * ys + p];
          const float gam = ex2(lg_eval<D>(c.emu[k], c.eA[k], c.eb[k], y, dd) - MM[p]) * SS[p];
          acc[0] += gam;
          int t = 1 + D;
#pragma unroll
          for (int x = 0; x < D; ++x) {
            const float gd = gam * dd[x];
            acc[1 + x] += gd;
#pragma unroll
            for (int yy = x; yy < D; ++yy, ++t) acc[t] = fmaf(gd, dd[yy], acc[t]);
          }
        }
        warp_rs<NRED>(acc, lane);
        if ((lane & (32 / NRED - 1)) == 0) {
          const int q = warp_rs_index<NRED>(lane);
          if (q < NS) c.redk[k][wid][q] = acc[0];
        }
      }
      __syncthreads();
      // M-step of every component (one lane each), L, convergence, AA start
      if (tid < 32) {
        // FP32 (the statistics are FP32 sums; FP64 here would put ~200
        // serial FP64 instructions on every iteration's critical path): the
        // shift of the mean is added to the FP64 iterate, so the mean keeps
        // its full precision
        float Nk = 0.0f;
        if (lane < K) {
          const int k = lane;
          float st[NS];
          for (int q = 0; q < NS; ++q) {
            float sq = 0.0f;
            for (int w = 0; w < NW; ++w) sq += c.redk[k][w][q];
            st[q] = sq;
          }
          Nk = st[0];
          bool ok = Nk > 0.0f;
          if (ok) {
            const float rN = rcp_nr(Nk);
            float dl[D], muf[D], Sf[NM];
            for (int x = 0; x < D; ++x) {
              dl[x] = st[1 + x] * rN;
              muf[x] = c.emu[k][x] + dl[x];
              c.gmu[k][x] = (double)c.emu[k][x] + (double)dl[x];
            }
            int t = 0;
            for (int x = 0; x < D; ++x)
              for (int yy = x; yy < D; ++yy, ++t) {
                Sf[t] = fmaf(-dl[x], dl[yy], st[1 + D + t] * rN);
                c.gS[k][t] = (double)Sf[t];
              }
            c.gw[k] = (double)(Nk * c.rsumAH);
            float Lc[3][3], ri[3];
            ok = chol_whitened<D, float, float>(Sf, muf, c.meanf, c.scf, Lc, ri, 1e-6);
            if (!ok) {  // near the floor: the covariance and its test in FP64
              const double rN64 = 1.0 / (double)Nk;
              double dl64[D], L64[3][3], r64[3];
              for (int x = 0; x < D; ++x) dl64[x] = (double)st[1 + x] * rN64;
              int t2 = 0;
              for (int x = 0; x < D; ++x)
                for (int yy = x; yy < D; ++yy, ++t2)
                  c.gS[k][t2] = (double)st[1 + D + t2] * rN64 - dl64[x] * dl64[yy];
              ok = chol_whitened<D, double, double>(c.gS[k], c.gmu[k], c.mean, c.sc, L64, r64);
            }
            if (!ok) atomicOr(&c.status, GM_ST_COV_NOT_PD);
          }
          c.gok[k] = ok ? 1 : 0;
        }
        __syncwarp();
        if (a.mml) {
          // eq. (omegak) over the survivors; annihilation of N_k - T/2 <= 0
          const float hT = 0.5f * (float)T;
          const bool okk = lane < K && c.gok[lane];
          const bool alive = okk && Nk - hT > 0.0f;
          const float den = warp_sum(alive ? Nk - hT : 0.0f);
          if (__ballot_sync(0xffffffffu, alive) == 0u) {
            // nothing survives: the component with the largest N_k stays
            // (lowest index on ties), with its old parameters if its new
            // covariance failed the floor
            float bv = lane < K ? Nk : -1.0f;
            int bi = lane;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
              const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
              if (ov > bv || (ov == bv && oi < bi)) {
                bv = ov;
                bi = oi;
              }
            }
            if (lane < K) {
              c.gok[lane] = lane == bi ? 1 : 0;
              if (lane == bi) {
                c.gw[lane] = 1.0;
                if (!okk) {
                  for (int d = 0; d < D; ++d) c.gmu[lane][d] = c.mu[lane][d];
                  for (int q = 0; q < NM; ++q) c.gS[lane][q] = c.S[lane][q];
                }
              }
            }
          } else if (lane < K) {
            c.gok[lane] = alive ? 1 : 0;
            c.gw[lane] = alive ? (double)((Nk - hT) / den) : 0.0;
          }
          __syncwarp();
        }
        double ls = lane < NW ? (double)c.redl[lane] : 0.0;
        ls = warp_sum(ls);
        __syncwarp();
        if (lane == 0) {
          double L = (ls + (double)c.c0 * c.sumAH) * kLn2 - c.Nd * c.logjac;
          if (a.mml) {  // eq. (lnL-GM) at the current parameters
            double pen = 0.0;
            for (int k = 0; k < K; ++k) pen += log(c.w[k]);
            const double dpar = (double)K * (T + 1) - 1.0;
            L -= 0.5 * dpar * log(c.Nd) + 0.5 * (double)T * pen;
          }
          const int it = c.it;
          if (it > 0 && !c.ann && fabs(L - c.Lprev) <= a.tol * fabs(c.Lprev))
            c.done = 1;
          else if (it + 1 >= a.max_sweeps)
            c.done = 2;
          if (!c.aa_on && it > 0 && fabs(L - c.Lprev) <= kAAStart * fabs(c.Lprev)) c.aa_on = 1;
          if (it == 0 && c.sumAH > 0.0) {
            // centre the FP32 log-likelihood sums on the first mean term
            c.c0 = (float)((ls + (double)c.c0 * c.sumAH) / c.sumAH);
          }
          c.Lprev = L;
          int Kg = 0;
          for (int k = 0; k < K; ++k) Kg += c.gok[k];
          c.Kg = Kg;
        }
      }
      __syncthreads();
      if (c.done) break;
      // ---- the next iterate --------------------------------------------------
      const bool plain = (c.Kg < K) || a.aa_m == 0 || !c.aa_on;
      if (plain) {
        if (tid == 0) {
          int Ko = 0;
          for (int k = 0; k < K; ++k) {
            if (!c.gok[k]) continue;
            c.w[Ko] = c.gw[k];
            for (int d = 0; d < D; ++d) c.mu[Ko][d] = c.gmu[k][d];
            for (int q = 0; q < NM; ++q) c.S[Ko][q] = c.gS[k][q];
            ++Ko;
          }
          if (Ko < K) {  // a dropped component restarts AA
            c.aa.h = 0;
            c.aa.have = 0;
          }
          c.ann = a.mml && Ko < K;
          c.K = Ko;
        }
      } else if (tid < 32) {
        // Anderson step (warp 0, FP64) on theta = (w, mu, M2) per component
        const int n = K * P;
        if (lane < K) {
          std_pack<D, NW>(c.w, c.mu, c.S, lane, c.aa.th);
          std_pack<D, NW>(c.gw, c.gmu, c.gS, lane, c.aa.tg);
        }
        __syncwarp();
        const int m = a.aa_m < kStdMaxM ? a.aa_m : kStdMaxM;
        bool applied = aa_warp_step<Ctl::NTH>(c.aa, n, m);
        const int h = c.aa.h;
        if (applied) {
          // validity of the extrapolation: positive weights, covariances
          // M2 - mu mu^T passing the floor (whitened and original)
          bool valid = true;
          if (lane < K) {
            // M2 - mu mu^T formed in FP64; the floor tested in FP32 and,
            // near it, in FP64 (whitened and original coordinates)
            const double* t = c.aa.tn + lane * P;
            double mw[D], Sw[NM];
            float Lc[3][3], ri[3];
            const double zero[3] = {0.0, 0.0, 0.0}, one[3] = {1.0, 1.0, 1.0};
            const float zf[3] = {0.0f, 0.0f, 0.0f}, of[3] = {1.0f, 1.0f, 1.0f};
            for (int d = 0; d < D; ++d) mw[d] = t[1 + d];
            int q = 0;
            for (int x = 0; x < D; ++x)
              for (int yy = x; yy < D; ++yy, ++q) Sw[q] = fma(-t[1 + x], t[1 + yy], t[1 + D + q]);
            valid = t[0] > 0.0 && std_chol<D>(Sw, mw, zero, one, zf, of, Lc, ri) &&
                    std_chol<D>(Sw, mw, c.mean, c.sc, c.meanf, c.scf, Lc, ri);
          }
          applied = __all_sync(0xffffffffu, valid);
          if (applied) {
            double ws = lane < K ? c.aa.tn[lane * P] : 0.0;
            ws = warp_sum(ws);
            if (lane < K) {
              const double* t = c.aa.tn + lane * P;
              c.w[lane] = t[0] / ws;
              for (int d = 0; d < D; ++d) c.mu[lane][d] = t[1 + d];
              int q = 0;
              for (int x = 0; x < D; ++x)
                for (int yy = x; yy < D; ++yy, ++q) c.S[lane][q] = t[1 + D + q] - t[1 + x] * t[1 + yy];
            }
          }
        }
        if (!applied) {
          if (lane < K) {
            c.w[lane] = c.gw[lane];
            for (int d = 0; d < D; ++d) c.mu[lane][d] = c.gmu[lane][d];
            for (int q = 0; q < NM; ++q) c.S[lane][q] = c.gS[lane][q];
          }
          if (lane == 0 && h > 0) {  // a failed extrapolation clears the history
            c.aa.h = 0;
            c.nreset++;
          }
        } else if (lane == 0) {
          c.naa++;
        }
      }
      __syncthreads();
      if (tid < c.K) std_econst<D, NW>(c, tid);
      if (tid == 0) c.it++;
      __syncthreads();
    }
    if (tid == 0 && c.done == 2) c.status |= GM_ST_EM_MAXSWEEPS;

    // ---- output: one standard EM step in FP64 (Sec. 4; eq. omegak-mle) ------
    if (tid == 0) c.Kf = 0;
    __syncthreads();
    {
      const int K = c.K;
      const double nw = c.Nd / c.W;
      // Normaliser pass: per particle r_p = alpha_p (N / W) / S_p with
      // S_p = sum_j 2^(log2(w_j f_j) - m_p) summed in FP64 (m_p the largest
      // term), kept exactly as its two 32-bit halves in the particle's SS
      // and MM words (free after the iterations).  Each thread keeps its
      // particles p = tid + i NT in every pass, so it reads back only what it
      // wrote; the component passes recompute m_p and the term of component k
      // with the same instructions on the same operands, so
      // sum_k gamma_pk = alpha_p N / W to FP64 rounding.
      int* Rlo = reinterpret_cast<int*>(SS);
      int* Rhi = reinterpret_cast<int*>(MM);
      for (int p = tid; p < N; p += NT) {
        float y[D], d[D];
#pragma unroll
        for (int q = 0; q < D; ++q) y[q] = Y[q * ys + p];
        float m = -3.0e38f;
        for (int jj = 0; jj < K; ++jj) m = fmaxf(m, lg_eval<D>(c.emu[jj], c.eA[jj], c.eb[jj], y, d));
        double Ssum = 0.0;
        for (int jj = 0; jj < K; ++jj)
          Ssum += (double)ex2(lg_eval<D>(c.emu[jj], c.eA[jj], c.eb[jj], y, d) - m);
        const double r = a.alpha[off + p] * nw / Ssum;
        Rlo[p] = __double2loint(r);
        Rhi[p] = __double2hiint(r);
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
          float m = -3.0e38f;
          for (int jj = 0; jj < K; ++jj) m = fmaxf(m, lg_eval<D>(c.emu[jj], c.eA[jj], c.eb[jj], y, d));
          const double gk = (double)ex2(lg_eval<D>(c.emu[k], c.eA[k], c.eb[k], y, d) - m);
          const double gam = __hiloint2double(Rhi[p], Rlo[p]) * gk;
          double dv[D];
#pragma unroll
          for (int q = 0; q < D; ++q) dv[q] = ((double)vin[(int64_t)q * a.n + off + p] - c.mean[q]) - ck[q];
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
        std_bsum<D, NW, NS>(c, acc);
        if (tid == 0 && c.res[0] > 0.0) {
          const int f = c.Kf;
          const double nn = c.res[0];
          double dl[D];
          for (int x = 0; x < D; ++x) {
            dl[x] = c.res[1 + x] / nn;
            c.fmu[f][x] = ck[x] + dl[x];
          }
          int t = 0;
          for (int x = 0; x < D; ++x)
            for (int yy = x; yy < D; ++yy, ++t) c.fS[f][t] = c.res[1 + D + t] / nn - dl[x] * dl[yy];
          c.fw[f] = nn / c.Nd;
          // a covariance failing the floor is dropped, as in every EM step
          double So[NM], mo[D], meano[D], one[D], Lo[3][3];
          for (int q = 0; q < NM; ++q) So[q] = c.fS[f][q];
          for (int d2 = 0; d2 < D; ++d2) {
            mo[d2] = 0.0;
            one[d2] = 1.0;
            meano[d2] = c.mean[d2] + c.fmu[f][d2];
          }
          if (chol_whitened<D, double, double>(So, mo, meano, one, Lo))
            c.Kf = f + 1;
          else
            c.status |= GM_ST_COV_NOT_PD;
        }
        __syncthreads();
      }
    }
    // ---- the log-likelihood of the output (unpenalised) ---------------------
    if (tid < c.Kf) {
      const int k = tid;
      c.w[k] = c.fw[k];
      for (int x = 0; x < D; ++x) c.mu[k][x] = c.fmu[k][x] * c.isc[x];
      int q = 0;
      for (int x = 0; x < D; ++x)
        for (int yy = x; yy < D; ++yy, ++q) c.S[k][q] = c.fS[k][q] * c.isc[x] * c.isc[yy];
      std_econst<D, NW>(c, k);
    }
    __syncthreads();
    {
      const int K = c.Kf;
      const float c0 = c.c0;
      float accl = 0.0f;
      for (int p = tid; p < N; p += NT) {
        float y[D], dd[D];
#pragma unroll
        for (int d = 0; d < D; ++d) y[d] = Y[d * ys + p];
        float m = -3.0e38f, s = 0.0f;
        for (int k = 0; k < K; ++k) {
          const float l = lg_eval<D>(c.emu[k], c.eA[k], c.eb[k], y, dd);
          if (l > m) {
            s = fmaf(s, ex2(m - l), 1.0f);
            m = l;
          } else {
            s += ex2(l - m);
          }
        }
        accl = fmaf(AH[p], (m - c0) + lg2(s), accl);
      }
      double v1[1] = {(double)accl};
      std_bsum<D, NW, 1>(c, v1);
    }
    if (tid == 0) {
      const int Kf = c.Kf;
      for (int k = 0; k < Kf; ++k) {
        double* r = prm_out + (size_t)k * P;
        r[0] = c.fw[k];
        for (int d = 0; d < D; ++d) r[1 + d] = c.mean[d] + c.fmu[k][d];
        for (int q = 0; q < NM; ++q) r[1 + D + q] = c.fS[k][q];
      }
      for (int i = Kf * P; i < a.Kmax * P; ++i) prm_out[i] = 0.0;
      a.K_out[j] = Kf;
      a.W_out[j] = c.W;
      a.lnL_out[j] = Kf > 0 ? (c.res[0] + (double)c.c0 * c.sumAH) * kLn2 - c.Nd * c.logjac : 0.0;
      if (a.iters_out) a.iters_out[j] = c.it + 1;
      if (a.aa_steps_out) a.aa_steps_out[j] = c.naa;
      if (a.aa_resets_out) a.aa_resets_out[j] = c.nreset;
      if (a.km_out) a.km_out[j] = c.kmp;
      a.status_out[j] = c.status;
    }
    __syncthreads();
  }
}

}  // namespace gmcr
