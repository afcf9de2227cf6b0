/*
 * gm_oracle.c -- plain, slow FP64 CPU oracle of the Gaussian-mixture
 * checkpoint-restart method of Chen, Chacon & Nguyen, "An unsupervised
 * machine-learning checkpoint-restart algorithm using Gaussian mixtures for
 * particle-in-cell simulations" (arXiv 2007.12273).
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the package smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header,
 * table or helper with the CUDA path, and the CUDA path never calls it.
 *
 * Every routine follows the paper's definitions in the paper's order, in
 * FP64, one cell at a time, with no blocking, fusion or reordering beyond
 * what the definition states.  Readings of points the paper leaves open are
 * marked "Reading:" where they are applied.
 *
 * Parameter record of one component (the checkpoint payload, Sec. 1):
 *   [ omega, mu_0..mu_{D-1}, Sigma upper triangle row-major ]
 * i.e. P = 1 + D + D(D+1)/2 numbers (3 for 1V, 10 for 3V).
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXD 3
#define OR_MAXK 16
#define OR_PI 3.14159265358979323846

/* per-cell status bits (same values as the library's documented ABI) */
#define ST_EM_MAXSWEEPS   0x01u
#define ST_COV_NOT_PD     0x02u
#define ST_TOO_FEW        0x04u
#define ST_EMPTY          0x08u
#define ST_DEGENERATE     0x10u
#define ST_PROJ_SKIPPED   0x100u
#define ST_NEG_WEIGHT     0x200u
#define ST_MM_EMPTY_COL   0x400u
#define ST_NO_MIXTURE     0x800u

/* Allocation that fails loudly: this library is test infrastructure, so an
 * allocation failure ends the process with a message (instead of a NULL
 * dereference inside a parallel loop). */
static void *or_malloc(size_t bytes) {
  void *p = malloc(bytes > 0 ? bytes : 1);
  if (!p) {
    fprintf(stderr, "gm_oracle: out of memory (%zu bytes)\n", bytes);
    abort();
  }
  return p;
}
static void *or_calloc(size_t n, size_t size) {
  void *p = calloc(n > 0 ? n : 1, size > 0 ? size : 1);
  if (!p) {
    fprintf(stderr, "gm_oracle: out of memory (%zu x %zu bytes)\n", n, size);
    abort();
  }
  return p;
}

typedef struct oracle_cfg {
  int D;            /* velocity dimensions, 1 or 3 */
  int Kmax;         /* initial number of components */
  int shape_order;  /* 1 = CIC (S1), 2 = quadratic B-spline (S2) */
  int max_sweeps;   /* cap on EM sweeps */
  double tol;       /* relative change of L that ends EM */
  uint64_t seed;    /* Philox key for the initial picks / the sampler */
  double L;         /* periodic domain length; dx = L / C */
  double q;         /* species charge */
} oracle_cfg;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator, written from its published        */
/* definition (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy */
/* as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies, the key      */
/* bumped by the two Weyl constants between rounds.                          */
/* ------------------------------------------------------------------------ */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uniform in (0,1) from two 32-bit words: 52 random bits m, u = (m + 1/2) 2^-52 */
double oracle_uniform52(uint32_t hi, uint32_t lo) {
  uint64_t m = ((uint64_t)hi << 20) | (uint64_t)(lo >> 12);
  return ((double)m + 0.5) * (1.0 / 4503599627370496.0);
}

/* uniform in (0,1) from one 32-bit word w: u = (w + 1/2) 2^-32 (exact) */
static double oracle_uniform32(uint32_t w) { return ((double)w + 0.5) * (1.0 / 4294967296.0); }

#define TAG_INIT 0x494E4954u   /* counter word 1 of the initial picks */
#define TAG_SAMPLE 0x53000000u /* counter word 1 of the sampler (| block) */

static void philox_draw(uint64_t seed, uint32_t c0, uint32_t c1, int64_t cell, uint32_t out[4]) {
  uint32_t ctr[4] = {c0, c1, (uint32_t)((uint64_t)cell & 0xffffffffu), (uint32_t)((uint64_t)cell >> 32)};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  oracle_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------------ */
/* Gaussian component: eq. (mix-dist) and the density below it.             */
/* ------------------------------------------------------------------------ */
typedef struct comp {
  double w;                    /* omega_k */
  double mu[OR_MAXD];          /* mu_k */
  double S[OR_MAXD][OR_MAXD];  /* Sigma_k (full symmetric) */
  double Lc[OR_MAXD][OR_MAXD]; /* Cholesky factor, Sigma = Lc Lc^T */
  double logdet;               /* ln |Sigma_k| */
} comp;

/* Cholesky of a symmetric DxD matrix.  Fails (returns 0) if a pivot is not
 * positive or falls under the covariance floor 1e-13 * scale2, where scale2
 * = sum_d (S_dd + mu_d^2) (Reading: the paper adds no regularisation; a
 * numerically singular covariance is treated as not positive definite). */
static int chol_floor(int D, double S[OR_MAXD][OR_MAXD], const double *mu,
                      double Lc[OR_MAXD][OR_MAXD], double *logdet) {
  double scale2 = 0.0;
  for (int d = 0; d < D; ++d) scale2 += S[d][d] + mu[d] * mu[d];
  double floor_ = 1e-13 * scale2;
  double ld = 0.0;
  memset(Lc, 0, sizeof(double) * OR_MAXD * OR_MAXD);
  for (int i = 0; i < D; ++i) {
    for (int j = 0; j <= i; ++j) {
      double s = S[i][j];
      for (int m = 0; m < j; ++m) s -= Lc[i][m] * Lc[j][m];
      if (i == j) {
        if (!(s > floor_) || !isfinite(s)) return 0;
        Lc[i][i] = sqrt(s);
        ld += log(s);
      } else {
        Lc[i][j] = s / Lc[j][j];
      }
    }
  }
  *logdet = ld;
  return 1;
}

/* ln f_k(v): f_k = (2 pi)^{-D/2} |Sigma|^{-1/2} exp(-(v-mu)^T Sigma^{-1} (v-mu)/2) */
static double log_gauss(int D, const comp *c, const double *v) {
  double d[OR_MAXD], y[OR_MAXD];
  for (int i = 0; i < D; ++i) d[i] = v[i] - c->mu[i];
  double maha = 0.0;
  for (int i = 0; i < D; ++i) { /* solve Lc y = d */
    double s = d[i];
    for (int m = 0; m < i; ++m) s -= c->Lc[i][m] * y[m];
    y[i] = s / c->Lc[i][i];
    maha += y[i] * y[i];
  }
  return -0.5 * maha - 0.5 * c->logdet - 0.5 * D * log(2.0 * OR_PI);
}

static int T_of(int D) { return D * (D + 3) / 2; }        /* T = D(D+3)/2, App. A */
static int P_of(int D) { return 1 + D + D * (D + 1) / 2; } /* numbers per component */

/* ln sum_k omega_k f_k(v), by log-sum-exp; also returns every
 * log(omega_k f_k(v)) in lf[] */
static double log_mix(int D, int K, const comp *cs, const double *v, double *lf) {
  double m = -INFINITY;
  for (int k = 0; k < K; ++k) {
    lf[k] = log(cs[k].w) + log_gauss(D, &cs[k], v);
    if (lf[k] > m) m = lf[k];
  }
  double s = 0.0;
  for (int k = 0; k < K; ++k) s += exp(lf[k] - m);
  return m + log(s);
}

/* Penalised log-likelihood, eq. (lnL-GM):
 *   L = sum_p alpha_p ln sum_k omega_k f_k(v_p) - (d/2) ln N - (T/2) sum_k ln omega_k
 * with T = D(D+3)/2 and d = K(T+1) - 1 (App. A). */
static double penalised_L(int D, int K, const comp *cs, int64_t N, const double *vv,
                          const double *ah) {
  double lf[OR_MAXK];
  double s = 0.0;
  for (int64_t p = 0; p < N; ++p) s += ah[p] * log_mix(D, K, cs, vv + p * D, lf);
  int T = T_of(D);
  double dpar = (double)K * (T + 1) - 1.0;
  double pen = 0.0;
  for (int k = 0; k < K; ++k) pen += log(cs[k].w);
  return s - 0.5 * dpar * log((double)N) - 0.5 * T * pen;
}

static void renormalise(int K, comp *cs) {
  double s = 0.0;
  for (int k = 0; k < K; ++k) s += cs[k].w;
  for (int k = 0; k < K; ++k) cs[k].w /= s;
}

static void remove_comp(int *K, comp *cs, int k) {
  for (int m = k; m < *K - 1; ++m) cs[m] = cs[m + 1];
  (*K)--;
}

static void store_params(int D, int Kmax, int K, const comp *cs, double *prm) {
  int P = P_of(D);
  memset(prm, 0, sizeof(double) * (size_t)Kmax * P);
  for (int k = 0; k < K; ++k) {
    double *r = prm + (size_t)k * P;
    r[0] = cs[k].w;
    for (int d = 0; d < D; ++d) r[1 + d] = cs[k].mu[d];
    int t = 1 + D;
    for (int i = 0; i < D; ++i)
      for (int j = i; j < D; ++j) r[t++] = cs[k].S[i][j];
  }
}

static void load_params(int D, int K, const double *prm, comp *cs) {
  int P = P_of(D);
  for (int k = 0; k < K; ++k) {
    const double *r = prm + (size_t)k * P;
    cs[k].w = r[0];
    for (int d = 0; d < D; ++d) cs[k].mu[d] = r[1 + d];
    int t = 1 + D;
    for (int i = 0; i < D; ++i)
      for (int j = i; j < D; ++j) { cs[k].S[i][j] = r[t]; cs[k].S[j][i] = r[t]; ++t; }
  }
}

/* ------------------------------------------------------------------------ */
/* Compression of one cell (Sec. 2.2-2.3).                                  */
/*   vv   : the cell's velocities, particle-major [N][D] (FP64)             */
/*   alpha: the cell's weights [N]                                          */
/* Optional: init_prm/init_K replace the random initialisation; Ltrace gets */
/* L after initialisation and after every sweep (trace_cap entries).        */
/* ------------------------------------------------------------------------ */
typedef struct cell_out {
  int32_t K;
  double W, lnL;
  int32_t sweeps, kwork;
  uint32_t status;
} cell_out;

static void em_cell(const oracle_cfg *cfg, int64_t cell, int64_t N, const double *vv,
                    const double *alpha, double *prm_out, cell_out *o,
                    const double *init_prm, int init_K, int only_sweeps,
                    double *Ltrace, int32_t *Ktrace, int trace_cap, int *ntrace) {
  const int D = cfg->D, T = T_of(D);
  const double halfT = 0.5 * T;
  comp cs[OR_MAXK];
  memset(o, 0, sizeof(*o));
  memset(prm_out, 0, sizeof(double) * (size_t)cfg->Kmax * P_of(D));
  if (ntrace) *ntrace = 0;
  if (N == 0) { o->status = ST_EMPTY; return; }

  /* Weights are normalised so that sum_p alpha_p = N (Sec. 2.2, below eq.
   * lnL-GM); W = sum alpha is kept for reconstruction. */
  double W = 0.0;
  for (int64_t p = 0; p < N; ++p) W += alpha[p];
  o->W = W;
  if (!(W > 0.0)) { o->status = ST_EMPTY | ST_DEGENERATE; return; }
  const double Nd = (double)N;
  double *ah = (double *)or_malloc(sizeof(double) * (size_t)N);
  double *gam = (double *)or_malloc(sizeof(double) * (size_t)N * OR_MAXK);
  for (int64_t p = 0; p < N; ++p) ah[p] = alpha[p] * Nd / W;
  if (N <= 10) o->status |= ST_TOO_FEW; /* Sec. 1: "more than 10" per cell */

  /* total (sample) mean and covariance, alpha-weighted, divided by N */
  double mean[OR_MAXD] = {0}, cov[OR_MAXD][OR_MAXD] = {{0}};
  for (int64_t p = 0; p < N; ++p)
    for (int d = 0; d < D; ++d) mean[d] += ah[p] * vv[p * D + d];
  for (int d = 0; d < D; ++d) mean[d] /= Nd;
  for (int64_t p = 0; p < N; ++p)
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j)
        cov[i][j] += ah[p] * (vv[p * D + i] - mean[i]) * (vv[p * D + j] - mean[j]);
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) cov[i][j] /= Nd;

  int K;
  {
    double Ltmp[OR_MAXD][OR_MAXD], ldtmp;
    if (!chol_floor(D, cov, mean, Ltmp, &ldtmp)) {
      /* every particle (numerically) at one velocity: a single degenerate
       * component carrying the sample moments, no likelihood */
      cs[0].w = 1.0;
      for (int d = 0; d < D; ++d) cs[0].mu[d] = mean[d];
      memcpy(cs[0].S, cov, sizeof(cov));
      store_params(D, cfg->Kmax, 1, cs, prm_out);
      o->K = 1; o->lnL = 0.0; o->sweeps = 0;
      o->status |= ST_DEGENERATE | ST_COV_NOT_PD;
      free(ah); free(gam);
      return;
    }
  }

  K = 0;
  if (init_prm && init_K > 0) {
    /* a supplied initial mixture (learned initialisation): components whose
     * covariance fails the Cholesky floor are dropped, the count is capped
     * so that N - T K / 2 > 0 (last components dropped), and an empty
     * result falls back to the random initialisation below */
    K = init_K < cfg->Kmax ? init_K : cfg->Kmax;
    load_params(D, K, init_prm, cs);
    for (int k = 0; k < K; ++k)
      if (!chol_floor(D, cs[k].S, cs[k].mu, cs[k].Lc, &cs[k].logdet) || !(cs[k].w > 0.0)) {
        remove_comp(&K, cs, k);
        --k;
      }
    while (K > 1 && Nd - halfT * K <= 0.0) --K;
  }
  if (K == 0) {
    /* Initialisation (Sec. 2.3): K ~ Kmax components, each mean a randomly
     * chosen particle, each covariance the total covariance, equal weights.
     * Reading: K0 = min(Kmax, N), lowered while N - T K/2 <= 0 so that the
     * denominator of eq. (omegak) stays positive; picks are distinct
     * indices drawn uniformly with a Philox stream keyed by (seed, cell). */
    K = cfg->Kmax < N ? cfg->Kmax : (int)N;
    while (K > 1 && Nd - halfT * K <= 0.0) --K;
    int64_t picks[OR_MAXK];
    int got = 0;
    for (uint32_t t = 0; got < K; ++t) {
      int64_t idx;
      if (t < 100000u) {
        uint32_t r[4];
        philox_draw(cfg->seed, t, TAG_INIT, cell, r);
        double u = oracle_uniform52(r[0], r[1]);
        idx = (int64_t)floor(u * Nd);
        if (idx >= N) idx = N - 1;
      } else { /* give up drawing: smallest unused index */
        idx = 0;
        for (;;) {
          int used = 0;
          for (int m = 0; m < got; ++m) used |= (picks[m] == idx);
          if (!used) break;
          ++idx;
        }
      }
      int dup = 0;
      for (int m = 0; m < got; ++m) dup |= (picks[m] == idx);
      if (!dup) picks[got++] = idx;
    }
    for (int k = 0; k < K; ++k) {
      cs[k].w = 1.0 / K;
      for (int d = 0; d < D; ++d) cs[k].mu[d] = vv[picks[k] * D + d];
      memcpy(cs[k].S, cov, sizeof(cov));
    }
  }
  for (int k = 0; k < K; ++k) /* Cholesky factors of the initial covariances */
    chol_floor(D, cs[k].S, cs[k].mu, cs[k].Lc, &cs[k].logdet);
  renormalise(K, cs);

  double Lprev = penalised_L(D, K, cs, N, vv, ah);
  if (Ltrace && *ntrace < trace_cap) { Ktrace[*ntrace] = K; Ltrace[(*ntrace)++] = Lprev; }
  int converged = 0, sweep = 0, kwork = 0;
  int max_sweeps = only_sweeps > 0 ? only_sweeps : cfg->max_sweeps;
  double lf[OR_MAXK];

  /* Component-wise EM (Sec. 2.3, after Celeux et al.): for each component
   * in storage order, an E-step for that component with the current
   * parameters of all components, then its M-step (eqs. muk, sigmak,
   * omegak), removal if N_k - T/2 <= 0, and renormalisation of the weights;
   * after the sweep, the convergence check on eq. (lnL-GM). */
  for (sweep = 1; sweep <= max_sweeps; ++sweep) {
    int annihilated = 0;
    int k = 0;
    while (k < K) {
      ++kwork;
      /* E-step, eq. (responsibility): gamma_pk = alpha_p w_k f_k / sum_j w_j f_j */
      double Nk = 0.0;
      for (int64_t p = 0; p < N; ++p) {
        double lm = log_mix(D, K, cs, vv + p * D, lf);
        gam[p] = ah[p] * exp(lf[k] - lm);
        Nk += gam[p];
      }
      /* annihilation: omega_k <= 0  <=>  N_k - T/2 <= 0 (eq. omegak).
       * Reading: the last component is never removed. */
      if (K > 1 && Nk - halfT <= 0.0) {
        remove_comp(&K, cs, k);
        annihilated = 1;
        renormalise(K, cs);
        continue;
      }
      /* M-step: eq. (muk), then eq. (sigmak) about the new mean */
      comp nc;
      for (int d = 0; d < D; ++d) {
        double s = 0.0;
        for (int64_t p = 0; p < N; ++p) s += gam[p] * vv[p * D + d];
        nc.mu[d] = s / Nk;
      }
      for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
          double s = 0.0;
          for (int64_t p = 0; p < N; ++p)
            s += gam[p] * (vv[p * D + i] - nc.mu[i]) * (vv[p * D + j] - nc.mu[j]);
          nc.S[i][j] = s / Nk;
        }
      if (!chol_floor(D, nc.S, nc.mu, nc.Lc, &nc.logdet)) {
        o->status |= ST_COV_NOT_PD;
        if (K > 1) {
          remove_comp(&K, cs, k);
          annihilated = 1;
          renormalise(K, cs);
          continue;
        }
        ++k; /* a lone component keeps its old parameters */
        continue;
      }
      /* eq. (omegak): omega_k = (N_k - T/2) / (N - T K / 2) */
      nc.w = (K == 1) ? 1.0 : (Nk - halfT) / (Nd - halfT * K);
      cs[k] = nc;
      renormalise(K, cs); /* step 3 */
      ++k;
    }
    double L = penalised_L(D, K, cs, N, vv, ah);
    if (Ltrace && *ntrace < trace_cap) { Ktrace[*ntrace] = annihilated ? -K : K; Ltrace[(*ntrace)++] = L; }
    /* Reading: converged when the relative change of L over a sweep with no
     * removal is at most tol. */
    if (!annihilated && fabs(L - Lprev) <= cfg->tol * fabs(Lprev)) { converged = 1; break; }
    Lprev = L;
  }
  if (!converged) {
    sweep = max_sweeps;
    if (only_sweeps <= 0) o->status |= ST_EM_MAXSWEEPS;
  }

  if (only_sweeps <= 0) {
    /* Final unpenalised step (Sec. 2.3.1): one simultaneous E-step over all
     * components, then eqs. (muk), (sigmak) and omega_k = N_k / N
     * (eq. omegak-mle), which restores the sample mass, mean and
     * covariance exactly. */
    double NkA[OR_MAXK] = {0};
    for (int64_t p = 0; p < N; ++p) {
      double lm = log_mix(D, K, cs, vv + p * D, lf);
      for (int k = 0; k < K; ++k) {
        gam[p * OR_MAXK + k] = ah[p] * exp(lf[k] - lm);
        NkA[k] += gam[p * OR_MAXK + k];
      }
    }
    comp fc[OR_MAXK];
    int Kf = 0, final_pd = 1;
    for (int k = 0; k < K; ++k) {
      if (!(NkA[k] > 0.0)) continue; /* a component that owns nothing */
      comp nc;
      for (int d = 0; d < D; ++d) {
        double s = 0.0;
        for (int64_t p = 0; p < N; ++p) s += gam[p * OR_MAXK + k] * vv[p * D + d];
        nc.mu[d] = s / NkA[k];
      }
      for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
          double s = 0.0;
          for (int64_t p = 0; p < N; ++p)
            s += gam[p * OR_MAXK + k] * (vv[p * D + i] - nc.mu[i]) * (vv[p * D + j] - nc.mu[j]);
          nc.S[i][j] = s / NkA[k];
        }
      nc.w = NkA[k] / Nd;
      if (!chol_floor(D, nc.S, nc.mu, nc.Lc, &nc.logdet)) { o->status |= ST_COV_NOT_PD; final_pd = 0; }
      fc[Kf++] = nc;
    }
    K = Kf;
    memcpy(cs, fc, sizeof(comp) * (size_t)K);
    o->lnL = final_pd ? penalised_L(D, K, cs, N, vv, ah) : 0.0;
  } else {
    o->lnL = penalised_L(D, K, cs, N, vv, ah);
  }
  store_params(D, cfg->Kmax, K, cs, prm_out);
  o->K = K;
  o->sweeps = sweep;
  o->kwork = kwork;
  free(ah);
  free(gam);
}

/* ------------------------------------------------------------------------ */
/* Shape functions (Sec. 2.4.1): B-splines of the distance in units of dx.  */
/* ------------------------------------------------------------------------ */
static double shape_S(int order, double s) {
  double a = fabs(s);
  if (order == 0) return a < 0.5 ? 1.0 : 0.0;
  if (order == 1) return a < 1.0 ? 1.0 - a : 0.0;
  /* order 2 */
  if (a <= 0.5) return 0.75 - a * a;
  if (a < 1.5) return 0.5 * (1.5 - a) * (1.5 - a);
  return 0.0;
}

static int64_t wrap(int64_t i, int64_t C) { i %= C; return i < 0 ? i + C : i; }

/* rho_i = (1/dx) sum_p q alpha_p S(x_i - x_p), node i at (i + 1/2) dx on the
 * periodic mesh; a particle of cell j reaches nodes j-1, j, j+1. */
static void deposit(const oracle_cfg *cfg, int64_t C, const int64_t *cell_off,
                    const double *x, const double *alpha, double *rho) {
  const double dx = cfg->L / (double)C;
  for (int64_t i = 0; i < C; ++i) rho[i] = 0.0;
  for (int64_t j = 0; j < C; ++j)
    for (int64_t p = cell_off[j]; p < cell_off[j + 1]; ++p)
      for (int64_t i = j - 1; i <= j + 1; ++i) {
        double xi = ((double)i + 0.5) * dx;
        rho[wrap(i, C)] += cfg->q * alpha[p] * shape_S(cfg->shape_order, (xi - x[p]) / dx) / dx;
      }
}

/* ------------------------------------------------------------------------ */
/* Exported: compression of all cells.                                      */
/* ------------------------------------------------------------------------ */
int oracle_compress(const oracle_cfg *cfg, int64_t C, const int64_t *cell_off,
                    const double *x, const double *v /* [D][Ntot] */, const double *alpha,
                    int32_t *K_out, double *params_out, double *W_out,
                    double *rho_target_out, double *lnL_out, int32_t *sweeps_out,
                    int32_t *kwork_out, uint32_t *status_out, const int64_t *cell_ids,
                    const int32_t *init_K /* [C] or NULL */,
                    const double *init_params /* [C][Kmax][P] or NULL */, int nthreads) {
  const int D = cfg->D;
  if (D != 1 && D != 3) return -1;
  if (cfg->Kmax < 1 || cfg->Kmax > OR_MAXK) return -1;
  const int64_t Ntot = cell_off[C];
  const size_t P = (size_t)P_of(D);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int64_t j = 0; j < C; ++j) {
    int64_t n = cell_off[j + 1] - cell_off[j];
    double *vv = (double *)or_malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * D);
    for (int64_t p = 0; p < n; ++p)
      for (int d = 0; d < D; ++d) vv[p * D + d] = v[(int64_t)d * Ntot + cell_off[j] + p];
    cell_out o;
    /* cell_ids (optional) gives each cell's index in a larger batch, which
     * keys its Philox stream */
    em_cell(cfg, cell_ids ? cell_ids[j] : j, n, vv, alpha + cell_off[j],
            params_out + (size_t)j * cfg->Kmax * P, &o,
            init_K ? init_params + (size_t)j * cfg->Kmax * P : NULL, init_K ? init_K[j] : 0, 0,
            NULL, NULL, 0, NULL);
    K_out[j] = o.K; W_out[j] = o.W; lnL_out[j] = o.lnL;
    if (sweeps_out) sweeps_out[j] = o.sweeps;
    if (kwork_out) kwork_out[j] = o.kwork;
    status_out[j] = o.status;
    free(vv);
  }
  /* stored charge density rho' from the original particles (Sec. 2.4.1) */
  if (rho_target_out) deposit(cfg, C, cell_off, x, alpha, rho_target_out);
  return 0;
}

/* Exported: one cell, for tests -- optional supplied initial parameters,
 * an optional fixed number of penalised sweeps with no final step
 * (only_sweeps > 0), and the trace of L. */
int oracle_em_cell(const oracle_cfg *cfg, int64_t cell, int64_t N, const double *vv /*[N][D]*/,
                   const double *alpha, const double *init_prm, int init_K, int only_sweeps,
                   double *params_out, int32_t *K_out, double *W_out, double *lnL_out,
                   int32_t *sweeps_out, uint32_t *status_out, double *Ltrace, int32_t *Ktrace,
                   int trace_cap, int32_t *ntrace) {
  cell_out o;
  int nt = 0;
  em_cell(cfg, cell, N, vv, alpha, params_out, &o, init_prm, init_K, only_sweeps, Ltrace,
          Ktrace, trace_cap, &nt);
  *K_out = o.K; *W_out = o.W; *lnL_out = o.lnL; *sweeps_out = o.sweeps; *status_out = o.status;
  if (ntrace) *ntrace = nt;
  return 0;
}

/* Exported: penalised L of given parameters on one cell (weights already
 * normalised to sum N), eq. (lnL-GM). */
double oracle_penalised_L(int D, int K, const double *prm, int64_t N, const double *vv,
                          const double *ah) {
  comp cs[OR_MAXK];
  load_params(D, K, prm, cs);
  for (int k = 0; k < K; ++k)
    if (!chol_floor(D, cs[k].S, cs[k].mu, cs[k].Lc, &cs[k].logdet)) return NAN;
  return penalised_L(D, K, cs, N, vv, ah);
}

/* ------------------------------------------------------------------------ */
/* Exported: cyclic tridiagonal solve, row i:                               */
/*   a_i x_{i-1} + b_i x_i + c_i x_{i+1} = d_i,  indices mod n, n >= 3.     */
/* Thomas elimination on the tridiagonal part plus the Sherman-Morrison     */
/* correction for the two corner entries (textbook direct solve).           */
/* ------------------------------------------------------------------------ */
static void thomas(int64_t n, const double *a, const double *b, const double *c,
                   const double *d, double *x, double *cp, double *dp) {
  cp[0] = c[0] / b[0];
  dp[0] = d[0] / b[0];
  for (int64_t i = 1; i < n; ++i) {
    double m = b[i] - a[i] * cp[i - 1];
    cp[i] = c[i] / m;
    dp[i] = (d[i] - a[i] * dp[i - 1]) / m;
  }
  x[n - 1] = dp[n - 1];
  for (int64_t i = n - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
}

int oracle_cyclic_tridiag(int64_t n, const double *a, const double *b, const double *c,
                          const double *d, double *x) {
  if (n < 3) return -1;
  double *bb = (double *)or_malloc(sizeof(double) * n);
  double *u = (double *)or_malloc(sizeof(double) * n);
  double *y = (double *)or_malloc(sizeof(double) * n);
  double *z = (double *)or_malloc(sizeof(double) * n);
  double *cp = (double *)or_malloc(sizeof(double) * n);
  double *dp = (double *)or_malloc(sizeof(double) * n);
  /* A = T + u v^T, u = (g, 0..0, c_{n-1}), v = (1, 0..0, a_0/g), g = -b_0 */
  double g = -b[0];
  for (int64_t i = 0; i < n; ++i) { bb[i] = b[i]; u[i] = 0.0; }
  bb[0] = b[0] - g;
  bb[n - 1] = b[n - 1] - c[n - 1] * a[0] / g;
  u[0] = g;
  u[n - 1] = c[n - 1];
  thomas(n, a, bb, c, d, y, cp, dp);
  thomas(n, a, bb, c, u, z, cp, dp);
  double vy = y[0] + a[0] / g * y[n - 1];
  double vz = z[0] + a[0] / g * z[n - 1];
  double f = vy / (1.0 + vz);
  for (int64_t i = 0; i < n; ++i) x[i] = y[i] - f * z[i];
  free(bb); free(u); free(y); free(z); free(cp); free(dp);
  return 0;
}

/* dense Gaussian elimination with partial pivoting, for meshes of 1-2 cells */
static int dense_solve(int n, double *A, double *b, double *x) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(A[r * n + c]) > fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0.0) return -1;
    if (piv != c) {
      for (int k = 0; k < n; ++k) { double t = A[c * n + k]; A[c * n + k] = A[piv * n + k]; A[piv * n + k] = t; }
      double t = b[c]; b[c] = b[piv]; b[piv] = t;
    }
    for (int r = c + 1; r < n; ++r) {
      double f = A[r * n + c] / A[c * n + c];
      for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
      b[r] -= f * b[c];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = b[r];
    for (int k = r + 1; k < n; ++k) s -= A[r * n + k] * x[k];
    x[r] = s / A[r * n + r];
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Reconstruction helpers shared by the 1D and 2D meshes (Sec. 2.4)          */
/* ------------------------------------------------------------------------ */

/* cell j's mixture with the Cholesky factors sampling needs (no floor: a
 * non-positive pivot gives a zero column) */
static void load_sampling_cell(int D, int Kj, const double *prm, comp *cs) {
  load_params(D, Kj, prm, cs);
  for (int k = 0; k < Kj; ++k) {
    memset(cs[k].Lc, 0, sizeof(cs[k].Lc));
    for (int a = 0; a < D; ++a)
      for (int b = 0; b <= a; ++b) {
        double s = cs[k].S[a][b];
        for (int m = 0; m < b; ++m) s -= cs[k].Lc[a][m] * cs[k].Lc[b][m];
        if (a == b) cs[k].Lc[a][a] = s > 0.0 ? sqrt(s) : 0.0;
        else cs[k].Lc[a][b] = cs[k].Lc[b][b] > 0.0 ? s / cs[k].Lc[b][b] : 0.0;
      }
  }
}

/* particle i of cell j (Sec. 2.4, eq. mix-dist-1): the uniform u0 of its
 * position inside the cell and its velocity: a component z with
 * probability omega_z (the smallest k with u1 < sum_{m <= k} omega_m), then
 * v = mu_z + Lc_z xi with xi from Box-Muller (Box & Muller 1958) on pairs
 * of uniforms.  Philox counter (i, TAG_SAMPLE | block, j): block 0 gives
 * u0 and u1 (52 bits each); block 1 one (radius, angle) pair of 52-bit
 * uniforms for D = 1, two pairs of 32-bit uniforms (one per word) for
 * D = 3. */
static double sample_one(const oracle_cfg *cfg, int D, const comp *cs, int Kj, int64_t j,
                         int64_t i, double *v) {
  uint32_t r0[4], r1[4];
  philox_draw(cfg->seed, (uint32_t)i, TAG_SAMPLE | 0u, j, r0);
  philox_draw(cfg->seed, (uint32_t)i, TAG_SAMPLE | 1u, j, r1);
  const double u0 = oracle_uniform52(r0[0], r0[1]);
  const double u1 = oracle_uniform52(r0[2], r0[3]);
  int z = Kj - 1;
  double cum = 0.0;
  for (int k = 0; k < Kj; ++k) {
    cum += cs[k].w;
    if (u1 < cum) { z = k; break; }
  }
  double xi[4];
  if (D == 1) {
    double ua = oracle_uniform52(r1[0], r1[1]), ub = oracle_uniform52(r1[2], r1[3]);
    double rr = sqrt(-2.0 * log(ua));
    xi[0] = rr * cos(2.0 * OR_PI * ub);
    xi[1] = rr * sin(2.0 * OR_PI * ub);
  } else {
    for (int q = 0; q < 2; ++q) {
      double ua = oracle_uniform32(r1[2 * q]), ub = oracle_uniform32(r1[2 * q + 1]);
      double rr = sqrt(-2.0 * log(ua));
      xi[2 * q] = rr * cos(2.0 * OR_PI * ub);
      xi[2 * q + 1] = rr * sin(2.0 * OR_PI * ub);
    }
  }
  for (int a = 0; a < D; ++a) {
    double sv = 0.0;
    if (Kj > 0) {
      sv = cs[z].mu[a];
      for (int b = 0; b <= a; ++b) sv += cs[z].Lc[a][b] * xi[b];
    }
    v[a] = sv;
  }
  return u0;
}

/* Lemons projection (Sec. 2.4.2), after the weight correction:
 * v' = a (v + beta), with targets p, E from the mixture and
 * N' = sum alpha', p' = sum alpha' v, E' = 1/2 sum alpha' |v|^2 (eq. beta),
 * a = sqrt((2 E N' - p^2) / (2 E' N' - p'^2)), beta = (p - a p')/(a N')
 * (eq. alpha).  A non-positive numerator skips the cell (Sec. 2.4.2:
 * "forgo the local moment-matching step"). */
static void lemons_project(const oracle_cfg *cfg, int64_t C, const int32_t *K, const double *params,
                           const double *W, const int64_t *out_off, const double *alpha_out,
                           double *v_out, uint32_t *status_out) {
  const int D = cfg->D;
  const size_t P = (size_t)P_of(D);
  const int64_t Nout = out_off[C];
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int64_t j = 0; j < C; ++j) {
    int64_t n = out_off[j + 1] - out_off[j];
    if (n == 0 || K[j] == 0) continue;
    comp cs[OR_MAXK];
    load_params(D, K[j], params + (size_t)j * cfg->Kmax * P, cs);
    double pt[OR_MAXD] = {0}, Et = 0.0;
    for (int k = 0; k < K[j]; ++k) {
      double tr = 0.0, mm = 0.0;
      for (int a = 0; a < D; ++a) {
        pt[a] += W[j] * cs[k].w * cs[k].mu[a];
        tr += cs[k].S[a][a];
        mm += cs[k].mu[a] * cs[k].mu[a];
      }
      Et += 0.5 * W[j] * cs[k].w * (tr + mm);
    }
    double Np = 0.0, pp[OR_MAXD] = {0}, Ep = 0.0;
    for (int64_t p = out_off[j]; p < out_off[j + 1]; ++p) {
      Np += alpha_out[p];
      for (int a = 0; a < D; ++a) {
        double va = v_out[(int64_t)a * Nout + p];
        pp[a] += alpha_out[p] * va;
        Ep += 0.5 * alpha_out[p] * va * va;
      }
    }
    double pt2 = 0.0, pp2 = 0.0;
    for (int a = 0; a < D; ++a) { pt2 += pt[a] * pt[a]; pp2 += pp[a] * pp[a]; }
    double num = 2.0 * Et * Np - pt2;
    double den = 2.0 * Ep * Np - pp2;
    if (!(num > 0.0) || !(den > 0.0) || !(Np > 0.0)) { status_out[j] |= ST_PROJ_SKIPPED; continue; }
    double aa = sqrt(num / den);
    double beta[OR_MAXD];
    for (int a = 0; a < D; ++a) beta[a] = (pt[a] - aa * pp[a]) / (aa * Np);
    for (int64_t p = out_off[j]; p < out_off[j + 1]; ++p)
      for (int a = 0; a < D; ++a) {
        double *va = &v_out[(int64_t)a * Nout + p];
        *va = aa * (*va + beta[a]);
      }
  }
}

/* ------------------------------------------------------------------------ */
/* Exported: reconstruction of all cells (Sec. 2.4).                        */
/* ------------------------------------------------------------------------ */
int oracle_reconstruct(const oracle_cfg *cfg, int64_t C, const int32_t *K, const double *params,
                       const double *W, const double *rho_target, const int64_t *out_off,
                       double *x_out, double *v_out /* [D][Nout] */, double *alpha_out,
                       uint32_t *status_out, double *dA_out /* [C] or NULL */,
                       double *v_raw_out /* [D][Nout] or NULL: velocities before projection */,
                       int nthreads) {
  const int D = cfg->D;
  const size_t P = (size_t)P_of(D);
  const int64_t Nout = out_off[C];
  const double dx = cfg->L / (double)C;
  if (D != 1 && D != 3) return -1;
  for (int64_t j = 0; j < C; ++j) status_out[j] = 0;

  /* 1. Sampling (Sec. 2.4): uniform position in the cell; ancestral
   *    sampling of the mixture, eq. (mix-dist-1): a component z with
   *    probability omega_z, then v ~ N(mu_z, Sigma_z) as v = mu + Lc xi
   *    with xi from Box-Muller; all particles of cell j get alpha = W_j/N'_j. */
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int64_t j = 0; j < C; ++j) {
    int64_t n = out_off[j + 1] - out_off[j];
    if (n == 0) continue;
    comp cs[OR_MAXK];
    int Kj = K[j];
    load_sampling_cell(D, Kj, params + (size_t)j * cfg->Kmax * P, cs);
    if (Kj == 0) status_out[j] |= ST_NO_MIXTURE;
    for (int64_t i = 0; i < n; ++i) {
      int64_t g = out_off[j] + i;
      double vv[OR_MAXD];
      const double u0 = sample_one(cfg, D, cs, Kj, j, i, vv);
      x_out[g] = ((double)j + u0) * dx;
      for (int a = 0; a < D; ++a) v_out[(int64_t)a * Nout + g] = vv[a];
      alpha_out[g] = W[j] / (double)n;
    }
  }
  if (v_raw_out) memcpy(v_raw_out, v_out, sizeof(double) * (size_t)D * Nout);

  /* 2. Gauss' law (Sec. 2.4.1): rho from the sampled particles, the mass
   *    matrix M_ij = sum_p q S0(x_j - x_p) S(x_i - x_p) (column j collects
   *    the particles of cell j), and the solve M dA = dx (rho' - rho). */
  double *rho = (double *)or_malloc(sizeof(double) * C);
  double *rhs = (double *)or_malloc(sizeof(double) * C);
  double *dA = (double *)or_malloc(sizeof(double) * C);
  deposit(cfg, C, out_off, x_out, alpha_out, rho);
  for (int64_t i = 0; i < C; ++i) rhs[i] = dx * (rho_target[i] - rho[i]);
  if (C >= 3) {
    double *a = (double *)or_calloc(C, sizeof(double)); /* M(i, i-1) */
    double *b = (double *)or_calloc(C, sizeof(double)); /* M(i, i)   */
    double *c = (double *)or_calloc(C, sizeof(double)); /* M(i, i+1) */
    for (int64_t j = 0; j < C; ++j)
      for (int64_t p = out_off[j]; p < out_off[j + 1]; ++p)
        for (int64_t i = j - 1; i <= j + 1; ++i) {
          double xi = ((double)i + 0.5) * dx;
          double m = cfg->q * shape_S(cfg->shape_order, (xi - x_out[p]) / dx);
          int64_t iw = wrap(i, C);
          if (i == j) b[iw] += m;
          else if (i == j - 1) c[iw] += m; /* row j-1, column j */
          else a[iw] += m;                 /* row j+1, column j */
        }
    /* Reading: a cell with no resampled particle has an empty column; it
     * gets a unit diagonal so its (inert) dA_j is defined. */
    for (int64_t j = 0; j < C; ++j)
      if (out_off[j + 1] == out_off[j]) {
        b[j] = 1.0; c[wrap(j - 1, C)] = 0.0; a[wrap(j + 1, C)] = 0.0;
        status_out[j] |= ST_MM_EMPTY_COL;
      }
    oracle_cyclic_tridiag(C, a, b, c, rhs, dA);
    free(a); free(b); free(c);
  } else {
    int n = (int)C;
    double A[4] = {0, 0, 0, 0}, bb[2], xx[2];
    for (int64_t j = 0; j < C; ++j)
      for (int64_t p = out_off[j]; p < out_off[j + 1]; ++p)
        for (int64_t i = j - 1; i <= j + 1; ++i) {
          double xi = ((double)i + 0.5) * dx;
          A[wrap(i, C) * n + j] += cfg->q * shape_S(cfg->shape_order, (xi - x_out[p]) / dx);
        }
    for (int64_t j = 0; j < C; ++j)
      if (out_off[j + 1] == out_off[j]) {
        for (int r = 0; r < n; ++r) A[r * n + j] = 0.0;
        A[j * n + j] = 1.0;
        status_out[j] |= ST_MM_EMPTY_COL;
      }
    for (int i = 0; i < n; ++i) bb[i] = rhs[i];
    dense_solve(n, A, bb, xx);
    for (int i = 0; i < n; ++i) dA[i] = xx[i];
  }
  /* eqs. (p-weight-correction), (new-p-weight): alpha'_p = alpha_p + dA_j */
  for (int64_t j = 0; j < C; ++j)
    for (int64_t p = out_off[j]; p < out_off[j + 1]; ++p) {
      alpha_out[p] += dA[j];
      if (!(alpha_out[p] > 0.0)) status_out[j] |= ST_NEG_WEIGHT;
    }
  if (dA_out) memcpy(dA_out, dA, sizeof(double) * C);
  free(rho); free(rhs); free(dA);

  /* 3. Lemons projection (Sec. 2.4.2), after the weight correction */
  lemons_project(cfg, C, K, params, W, out_off, alpha_out, v_out, status_out);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* The 2D periodic mesh (Sec. 2.4.1 in two dimensions, the geometry of the  */
/* 2D-3V Weibel runs of Sec. 3.2).  Cells and nodes are numbered            */
/* j = jy Cx + jx; node (ix, iy) sits at the cell centre                    */
/* ((ix + 1/2) dx, (iy + 1/2) dy); the shape function is the tensor product */
/* S(x) S(y) of the 1D B-spline of the chosen order, so a particle of cell  */
/* (jx, jy) reaches the 3 x 3 nodes around its cell.                        */
/* ------------------------------------------------------------------------ */
typedef struct oracle_mesh2d {
  int64_t Cx, Cy;
  double Lx, Ly;
} oracle_mesh2d;

#define OR_MAX_DENSE2D 2048 /* the direct solve below is dense: C <= this */

/* rho_i = (1 / (dx dy)) sum_p q alpha_p S(x_i - x_p) S(y_i - y_p) */
static void deposit2d(const oracle_cfg *cfg, const oracle_mesh2d *m, const int64_t *cell_off,
                      const double *x, const double *y, const double *alpha, double *rho) {
  const int64_t Cx = m->Cx, Cy = m->Cy, C = Cx * Cy;
  const double dx = m->Lx / (double)Cx, dy = m->Ly / (double)Cy;
  for (int64_t i = 0; i < C; ++i) rho[i] = 0.0;
  for (int64_t j = 0; j < C; ++j) {
    const int64_t jx = j % Cx, jy = j / Cx;
    for (int64_t p = cell_off[j]; p < cell_off[j + 1]; ++p)
      for (int64_t iy = jy - 1; iy <= jy + 1; ++iy)
        for (int64_t ix = jx - 1; ix <= jx + 1; ++ix) {
          const double xi = ((double)ix + 0.5) * dx, yi = ((double)iy + 0.5) * dy;
          const double w = shape_S(cfg->shape_order, (xi - x[p]) / dx) *
                           shape_S(cfg->shape_order, (yi - y[p]) / dy);
          rho[wrap(iy, Cy) * Cx + wrap(ix, Cx)] += cfg->q * alpha[p] * w / (dx * dy);
        }
  }
}

/* Exported: the 2D charge density of particles sorted by cell */
int oracle_deposit2d(const oracle_cfg *cfg, const oracle_mesh2d *m, const int64_t *cell_off,
                     const double *x, const double *y, const double *alpha, double *rho) {
  if (m->Cx < 1 || m->Cy < 1) return -1;
  deposit2d(cfg, m, cell_off, x, y, alpha, rho);
  return 0;
}

/* Exported: reconstruction on the 2D mesh (Sec. 2.4): positions uniform in
 * the cell (x from the 1D sampler's u0, y from Philox block 3:
 * counter (i, TAG_SAMPLE | 3, j), words 0-1), velocities and weights as in
 * 1D; Gauss' law with M_ij = sum_{p in j} q S(x_i - x_p) S(y_i - y_p) (a
 * 9-point column per cell) and M dA = dx dy (rho' - rho), solved directly
 * (dense Gaussian elimination with partial pivoting, C <= OR_MAX_DENSE2D;
 * a cell with no resampled particle gets a unit diagonal); then the weight
 * update and the Lemons projection, as in 1D.  xy_out [2][Nout]. */
int oracle_reconstruct2d(const oracle_cfg *cfg, const oracle_mesh2d *m, const int32_t *K,
                         const double *params, const double *W, const double *rho_target,
                         const int64_t *out_off, double *xy_out, double *v_out, double *alpha_out,
                         uint32_t *status_out, double *dA_out, int nthreads) {
  const int D = cfg->D;
  const size_t P = (size_t)P_of(D);
  const int64_t Cx = m->Cx, Cy = m->Cy, C = Cx * Cy;
  if (D != 1 && D != 3) return -1;
  if (Cx < 1 || Cy < 1) return -1;
  if (C > OR_MAX_DENSE2D) return -2;
  const int64_t Nout = out_off[C];
  const double dx = m->Lx / (double)Cx, dy = m->Ly / (double)Cy;
  double *x_out = xy_out, *y_out = xy_out + Nout;
  for (int64_t j = 0; j < C; ++j) status_out[j] = 0;

  /* 1. sampling */
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int64_t j = 0; j < C; ++j) {
    int64_t n = out_off[j + 1] - out_off[j];
    if (n == 0) continue;
    const int64_t jx = j % Cx, jy = j / Cx;
    comp cs[OR_MAXK];
    int Kj = K[j];
    load_sampling_cell(D, Kj, params + (size_t)j * cfg->Kmax * P, cs);
    if (Kj == 0) status_out[j] |= ST_NO_MIXTURE;
    for (int64_t i = 0; i < n; ++i) {
      int64_t g = out_off[j] + i;
      double vv[OR_MAXD];
      uint32_t r3[4];
      const double u0 = sample_one(cfg, D, cs, Kj, j, i, vv);
      philox_draw(cfg->seed, (uint32_t)i, TAG_SAMPLE | 3u, j, r3);
      const double uy = oracle_uniform52(r3[0], r3[1]);
      x_out[g] = ((double)jx + u0) * dx;
      y_out[g] = ((double)jy + uy) * dy;
      for (int a = 0; a < D; ++a) v_out[(int64_t)a * Nout + g] = vv[a];
      alpha_out[g] = W[j] / (double)n;
    }
  }

  /* 2. Gauss' law */
  double *rho = (double *)or_malloc(sizeof(double) * C);
  double *rhs = (double *)or_malloc(sizeof(double) * C);
  double *dA = (double *)or_malloc(sizeof(double) * C);
  double *A = (double *)or_calloc((size_t)C * C, sizeof(double));
  deposit2d(cfg, m, out_off, x_out, y_out, alpha_out, rho);
  for (int64_t i = 0; i < C; ++i) rhs[i] = dx * dy * (rho_target[i] - rho[i]);
  for (int64_t j = 0; j < C; ++j) {
    const int64_t jx = j % Cx, jy = j / Cx;
    for (int64_t p = out_off[j]; p < out_off[j + 1]; ++p)
      for (int64_t iy = jy - 1; iy <= jy + 1; ++iy)
        for (int64_t ix = jx - 1; ix <= jx + 1; ++ix) {
          const double xi = ((double)ix + 0.5) * dx, yi = ((double)iy + 0.5) * dy;
          const double w = shape_S(cfg->shape_order, (xi - x_out[p]) / dx) *
                           shape_S(cfg->shape_order, (yi - y_out[p]) / dy);
          A[(wrap(iy, Cy) * Cx + wrap(ix, Cx)) * C + j] += cfg->q * w;
        }
    if (out_off[j + 1] == out_off[j]) {
      A[j * C + j] = 1.0;
      status_out[j] |= ST_MM_EMPTY_COL;
    }
  }
  int rc = dense_solve((int)C, A, rhs, dA);
  free(A);
  if (rc != 0) { free(rho); free(rhs); free(dA); return -3; }
  for (int64_t j = 0; j < C; ++j)
    for (int64_t p = out_off[j]; p < out_off[j + 1]; ++p) {
      alpha_out[p] += dA[j];
      if (!(alpha_out[p] > 0.0)) status_out[j] |= ST_NEG_WEIGHT;
    }
  if (dA_out) memcpy(dA_out, dA, sizeof(double) * C);
  free(rho); free(rhs); free(dA);

  /* 3. Lemons projection */
  lemons_project(cfg, C, K, params, W, out_off, alpha_out, v_out, status_out);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Exported: per-cell moments of particles (Sec. 2.3.1 quantities) and the  */
/* charge density.  W = sum alpha, p = sum alpha v, M2 = sum alpha v v^T    */
/* (upper triangle row-major), E = 1/2 sum alpha |v|^2.                     */
/* ------------------------------------------------------------------------ */
int oracle_moments(const oracle_cfg *cfg, int64_t C, const int64_t *cell_off, const double *x,
                   const double *v /*[D][Ntot]*/, const double *alpha, double *W, double *p,
                   double *M2, double *E, double *rho) {
  const int D = cfg->D;
  const int64_t Ntot = cell_off[C];
  const int nm = D * (D + 1) / 2;
  for (int64_t j = 0; j < C; ++j) {
    double w = 0.0, pm[OR_MAXD] = {0}, m2[6] = {0}, e = 0.0;
    for (int64_t q = cell_off[j]; q < cell_off[j + 1]; ++q) {
      w += alpha[q];
      int t = 0;
      for (int a = 0; a < D; ++a) {
        double va = v[(int64_t)a * Ntot + q];
        pm[a] += alpha[q] * va;
        e += 0.5 * alpha[q] * va * va;
        for (int b = a; b < D; ++b) m2[t++] += alpha[q] * va * v[(int64_t)b * Ntot + q];
      }
    }
    W[j] = w;
    for (int a = 0; a < D; ++a) p[j * D + a] = pm[a];
    for (int t = 0; t < nm; ++t) M2[j * nm + t] = m2[t];
    E[j] = e;
  }
  if (rho) deposit(cfg, C, cell_off, x, alpha, rho);
  return 0;
}

/* Exported: the same moments of the mixtures: W_j, p = W sum_k w_k mu_k,
 * M2 = W sum_k w_k (Sigma_k + mu_k mu_k^T), E = tr(M2)/2. */
int oracle_mixture_moments(const oracle_cfg *cfg, int64_t C, const int32_t *K,
                           const double *params, const double *Wc, double *W, double *p,
                           double *M2, double *E) {
  const int D = cfg->D;
  const size_t P = (size_t)P_of(D);
  const int nm = D * (D + 1) / 2;
  for (int64_t j = 0; j < C; ++j) {
    comp cs[OR_MAXK];
    load_params(D, K[j], params + (size_t)j * cfg->Kmax * P, cs);
    double pm[OR_MAXD] = {0}, m2[6] = {0};
    for (int k = 0; k < K[j]; ++k) {
      int t = 0;
      for (int a = 0; a < D; ++a) {
        pm[a] += Wc[j] * cs[k].w * cs[k].mu[a];
        for (int b = a; b < D; ++b)
          m2[t++] += Wc[j] * cs[k].w * (cs[k].S[a][b] + cs[k].mu[a] * cs[k].mu[b]);
      }
    }
    W[j] = Wc[j];
    double e = 0.0;
    int t = 0;
    for (int a = 0; a < D; ++a) {
      p[j * D + a] = pm[a];
      for (int b = a; b < D; ++b) {
        if (a == b) e += 0.5 * m2[t];
        M2[j * nm + t] = m2[t];
        ++t;
      }
    }
    E[j] = e;
  }
  return 0;
}

/* Exported: shape function value, for tests */
double oracle_shape(int order, double s) { return shape_S(order, s); }

/* Exported: number of OpenMP threads a parallel region would use */
int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ======================================================================== */
/* Standard (non-adaptive) EM, K-means initialisation and Anderson          */
/* acceleration: the acceleration study of Sec. 4 ("On the acceleration of   */
/* convergence of the EM-GM nonlinear algorithm"), where the paper applies   */
/* both to the non-adaptive EM-GM algorithm.                                 */
/* ======================================================================== */

#define AA_MAXM 8
#define AA_MAXN (OR_MAXK * 10)
/* Reading: AA starts once the relative change of L over an EM iteration is
 * at most this (the paper does not say when; extrapolating the first,
 * large EM moves from a random start led to poorer stationary points) */
#define AA_START 1e-4

/* Anderson acceleration of a fixed-point map G (Walker & Ni 2011, the
 * "type II" form): with f_i = G(x_i) - x_i and the differences of the last
 * m pairs (f, G), gamma minimises || f_i - dF gamma ||_2 and
 * x_{i+1} = G(x_i) - dG gamma. */
typedef struct aa_state {
  int n, m, h, have_prev;
  double dF[AA_MAXM][AA_MAXN], dG[AA_MAXM][AA_MAXN];
  double f_prev[AA_MAXN], g_prev[AA_MAXN];
} aa_state;

static void aa_init(aa_state *s, int n, int m) {
  s->n = n; s->m = m < AA_MAXM ? m : AA_MAXM; s->h = 0; s->have_prev = 0;
}

/* forgets the stored differences; the last (f, G) pair stays the previous one */
static void aa_clear(aa_state *s) { s->h = 0; }

/* One step: the new difference joins the history (oldest dropped beyond m);
 * gamma from the normal equations (dF^T dF + 1e-12 max_a (dF^T dF)_aa I)
 * gamma = dF^T f by Cholesky (Reading: the paper does not say how the
 * least-squares problem is solved).  Returns 1 and out = G - dG gamma, or 0
 * and out = G when there is no history or a pivot is not positive. */
static int aa_step(aa_state *s, const double *x, const double *g, double *out) {
  const int n = s->n;
  double f[AA_MAXN];
  for (int i = 0; i < n; ++i) f[i] = g[i] - x[i];
  if (s->m > 0 && s->have_prev) {
    if (s->h == s->m) {
      for (int c = 1; c < s->m; ++c) {
        memcpy(s->dF[c - 1], s->dF[c], sizeof(double) * (size_t)n);
        memcpy(s->dG[c - 1], s->dG[c], sizeof(double) * (size_t)n);
      }
      s->h--;
    }
    for (int i = 0; i < n; ++i) {
      s->dF[s->h][i] = f[i] - s->f_prev[i];
      s->dG[s->h][i] = g[i] - s->g_prev[i];
    }
    s->h++;
  }
  memcpy(s->f_prev, f, sizeof(double) * (size_t)n);
  memcpy(s->g_prev, g, sizeof(double) * (size_t)n);
  s->have_prev = 1;
  const int h = s->h;
  memcpy(out, g, sizeof(double) * (size_t)n);
  if (h == 0) return 0;
  double A[AA_MAXM][AA_MAXM], b[AA_MAXM], Lm[AA_MAXM][AA_MAXM], z[AA_MAXM], gam[AA_MAXM];
  double dmax = 0.0;
  for (int a = 0; a < h; ++a) {
    for (int c = 0; c <= a; ++c) {
      double t = 0.0;
      for (int i = 0; i < n; ++i) t += s->dF[a][i] * s->dF[c][i];
      A[a][c] = A[c][a] = t;
    }
    double t = 0.0;
    for (int i = 0; i < n; ++i) t += s->dF[a][i] * f[i];
    b[a] = t;
    if (A[a][a] > dmax) dmax = A[a][a];
  }
  if (!(dmax > 0.0)) return 0;
  for (int a = 0; a < h; ++a) A[a][a] += 1e-12 * dmax;
  for (int a = 0; a < h; ++a)
    for (int c = 0; c <= a; ++c) {
      double t = A[a][c];
      for (int e = 0; e < c; ++e) t -= Lm[a][e] * Lm[c][e];
      if (a == c) {
        if (!(t > 0.0)) return 0;
        Lm[a][a] = sqrt(t);
      } else {
        Lm[a][c] = t / Lm[c][c];
      }
    }
  for (int a = 0; a < h; ++a) {
    double t = b[a];
    for (int e = 0; e < a; ++e) t -= Lm[a][e] * z[e];
    z[a] = t / Lm[a][a];
  }
  for (int a = h - 1; a >= 0; --a) {
    double t = z[a];
    for (int e = a + 1; e < h; ++e) t -= Lm[e][a] * gam[e];
    gam[a] = t / Lm[a][a];
  }
  for (int i = 0; i < n; ++i) {
    double t = g[i];
    for (int c = 0; c < h; ++c) t -= s->dG[c][i] * gam[c];
    out[i] = t;
  }
  return 1;
}

/* The accelerated unknowns (Sec. 4): per component omega_k, mu_k and the
 * second-moment matrix M2_k = Sigma_k + mu_k mu_k^T (upper triangle), which
 * is linear in the mixture; Reading: in the cell's whitened coordinates
 * (v - mean) / sd per dimension, so that all unknowns have unit scale. */
static void theta_pack(int D, int K, const comp *cs, const double *mean, const double *sd,
                       double *th) {
  int t = 0;
  for (int k = 0; k < K; ++k) {
    double mw[OR_MAXD];
    th[t++] = cs[k].w;
    for (int d = 0; d < D; ++d) th[t++] = mw[d] = (cs[k].mu[d] - mean[d]) / sd[d];
    for (int i = 0; i < D; ++i)
      for (int j = i; j < D; ++j) th[t++] = cs[k].S[i][j] / (sd[i] * sd[j]) + mw[i] * mw[j];
  }
}

/* back to a mixture (original coordinates); 0 if a weight is not positive
 * or a covariance M2 - mu mu^T fails the Cholesky floor (in the whitened and
 * in the original coordinates) */
static int theta_unpack(int D, int K, const double *th, const double *mean, const double *sd,
                        comp *cs) {
  int t = 0;
  for (int k = 0; k < K; ++k) {
    double mw[OR_MAXD], Sw[OR_MAXD][OR_MAXD], Lw[OR_MAXD][OR_MAXD], ldw;
    cs[k].w = th[t++];
    for (int d = 0; d < D; ++d) mw[d] = th[t++];
    for (int i = 0; i < D; ++i)
      for (int j = i; j < D; ++j) { Sw[i][j] = Sw[j][i] = th[t++] - mw[i] * mw[j]; }
    if (!(cs[k].w > 0.0)) return 0;
    if (!chol_floor(D, Sw, mw, Lw, &ldw)) return 0;
    for (int d = 0; d < D; ++d) cs[k].mu[d] = mean[d] + sd[d] * mw[d];
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) cs[k].S[i][j] = Sw[i][j] * sd[i] * sd[j];
    if (!chol_floor(D, cs[k].S, cs[k].mu, cs[k].Lc, &cs[k].logdet)) return 0;
  }
  return 1;
}

/* Unpenalised log-likelihood sum_p alpha_p ln sum_k omega_k f_k(v_p) */
static double plain_L(int D, int K, const comp *cs, int64_t N, const double *vv, const double *ah) {
  double lf[OR_MAXK], s = 0.0;
  for (int64_t p = 0; p < N; ++p) s += ah[p] * log_mix(D, K, cs, vv + p * D, lf);
  return s;
}

/* One standard EM step: the E-step (eq. responsibility) for all components
 * with the same parameters, then eqs. (muk), (sigmak) and omega_k = N_k / N
 * (eq. omegak-mle).  Returns L at the input parameters; out receives the
 * update.  Reading: a component that owns nothing or whose covariance fails
 * the floor is dropped (the count only shrinks; status COV_NOT_PD for the
 * floor). */
static double std_em_step(int D, int K, const comp *cs, int64_t N, const double *vv,
                          const double *ah, double *gam, comp *out, int *Kout, uint32_t *status) {
  double lf[OR_MAXK], Nk[OR_MAXK] = {0}, L = 0.0;
  const double Nd = (double)N;
  for (int64_t p = 0; p < N; ++p) {
    double lm = log_mix(D, K, cs, vv + p * D, lf);
    L += ah[p] * lm;
    for (int k = 0; k < K; ++k) {
      gam[p * OR_MAXK + k] = ah[p] * exp(lf[k] - lm);
      Nk[k] += gam[p * OR_MAXK + k];
    }
  }
  int Ko = 0;
  for (int k = 0; k < K; ++k) {
    if (!(Nk[k] > 0.0)) continue;
    comp nc;
    for (int d = 0; d < D; ++d) {
      double s = 0.0;
      for (int64_t p = 0; p < N; ++p) s += gam[p * OR_MAXK + k] * vv[p * D + d];
      nc.mu[d] = s / Nk[k];
    }
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) {
        double s = 0.0;
        for (int64_t p = 0; p < N; ++p)
          s += gam[p * OR_MAXK + k] * (vv[p * D + i] - nc.mu[i]) * (vv[p * D + j] - nc.mu[j]);
        nc.S[i][j] = s / Nk[k];
      }
    nc.w = Nk[k] / Nd;
    if (!chol_floor(D, nc.S, nc.mu, nc.Lc, &nc.logdet)) { *status |= ST_COV_NOT_PD; continue; }
    out[Ko++] = nc;
  }
  *Kout = Ko;
  return L;
}

/* One simultaneous penalised EM step (NEXT variant of Sec. 2.3: the E-step
 * of every component with the same parameters theta_i, then every M-step):
 * gamma from eq. (responsibility); a component with N_k - T/2 <= 0 is
 * annihilated (eq. omegak, a tie annihilated), as is one whose new
 * covariance (eqs. muk, sigmak) fails the floor (status COV_NOT_PD); the
 * survivors get omega_k = (N_k - T/2) / sum_survivors (N_j - T/2), which is
 * eq. (omegak) renormalised (step 3).  Reading: the last component is never
 * removed: if nothing survives, the component with the largest N_k (lowest
 * index on ties) stays with omega = 1, updated if its covariance passes the
 * floor, else with its old parameters.  Returns the penalised L (eq.
 * lnL-GM) at the input parameters; *annihilated is set if the count fell. */
static double mml_em_step(int D, int K, const comp *cs, int64_t N, const double *vv,
                          const double *ah, double *gam, comp *out, int *Kout,
                          int *annihilated, uint32_t *status) {
  const int T = T_of(D);
  const double halfT = 0.5 * T;
  double lf[OR_MAXK], Nk[OR_MAXK] = {0}, L = 0.0;
  for (int64_t p = 0; p < N; ++p) {
    double lm = log_mix(D, K, cs, vv + p * D, lf);
    L += ah[p] * lm;
    for (int k = 0; k < K; ++k) {
      gam[p * OR_MAXK + k] = ah[p] * exp(lf[k] - lm);
      Nk[k] += gam[p * OR_MAXK + k];
    }
  }
  double pen = 0.0;
  for (int k = 0; k < K; ++k) pen += log(cs[k].w);
  const double dpar = (double)K * (T + 1) - 1.0;
  L = L - 0.5 * dpar * log((double)N) - 0.5 * T * pen;

  comp nc[OR_MAXK];
  int ok[OR_MAXK];
  for (int k = 0; k < K; ++k) {
    ok[k] = 0;
    if (!(Nk[k] > 0.0)) continue;
    for (int d = 0; d < D; ++d) {
      double s = 0.0;
      for (int64_t p = 0; p < N; ++p) s += gam[p * OR_MAXK + k] * vv[p * D + d];
      nc[k].mu[d] = s / Nk[k];
    }
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) {
        double s = 0.0;
        for (int64_t p = 0; p < N; ++p)
          s += gam[p * OR_MAXK + k] * (vv[p * D + i] - nc[k].mu[i]) * (vv[p * D + j] - nc[k].mu[j]);
        nc[k].S[i][j] = s / Nk[k];
      }
    ok[k] = chol_floor(D, nc[k].S, nc[k].mu, nc[k].Lc, &nc[k].logdet);
    if (!ok[k]) *status |= ST_COV_NOT_PD;
  }
  double den = 0.0;
  int Ko = 0;
  for (int k = 0; k < K; ++k)
    if (Nk[k] - halfT > 0.0 && ok[k]) den += Nk[k] - halfT;
  for (int k = 0; k < K; ++k) {
    if (!(Nk[k] - halfT > 0.0 && ok[k])) continue;
    out[Ko] = nc[k];
    out[Ko].w = (Nk[k] - halfT) / den;
    ++Ko;
  }
  if (Ko == 0) {
    int kb = 0;
    for (int k = 1; k < K; ++k)
      if (Nk[k] > Nk[kb]) kb = k;
    out[0] = ok[kb] ? nc[kb] : cs[kb];
    out[0].w = 1.0;
    Ko = 1;
  }
  *annihilated = Ko < K;
  *Kout = Ko;
  return L;
}

/* K-means (Lloyd) initialisation in the whitened coordinates
 * y = (v - mean) * (1 / sd), stored in FP32; the centres start at the picked
 * particles.  Each pass assigns every particle to the nearest centre
 * (squared distance in FP32, fmaf in dimension order, the lowest index on
 * ties), stops when no assignment changed, else moves every centre to the
 * weighted mean of its particles with the weights rounded to FP32 (sums in
 * FP64, the centre rounded to FP32; an empty cluster keeps its centre); at
 * most iters passes.  Reading: the assignment decisions are taken on the
 * FP32 coordinates and weights the GPU kernel stages.  The mixture: one component per non-empty cluster,
 * weight = its share of the normalised weights, mean and biased covariance
 * of its particles (the total covariance if that fails the floor).
 * Returns the number of components. */
static int kmeans_init(int D, int K, int64_t N, const double *vv, const double *ah,
                       const double *mean, const double *sd, const double cov[OR_MAXD][OR_MAXD],
                       const int64_t *picks, int iters, comp *cs, int *passes) {
  double isd[OR_MAXD];
  for (int d = 0; d < D; ++d) isd[d] = 1.0 / sd[d];
  float *y = (float *)or_malloc(sizeof(float) * (size_t)N * D);
  int *as = (int *)or_malloc(sizeof(int) * (size_t)N);
  for (int64_t p = 0; p < N; ++p)
    for (int d = 0; d < D; ++d) y[p * D + d] = (float)((vv[p * D + d] - mean[d]) * isd[d]);
  float c[OR_MAXK][OR_MAXD];
  for (int k = 0; k < K; ++k)
    for (int d = 0; d < D; ++d) c[k][d] = y[picks[k] * D + d];
  int it;
  for (it = 0; it < iters; ++it) {
    int64_t changed = 0;
    for (int64_t p = 0; p < N; ++p) {
      int best = 0;
      float bd = 0.0f;
      for (int k = 0; k < K; ++k) {
        const float d0 = y[p * D] - c[k][0];
        float dist = d0 * d0;
        if (D == 3) {
          const float d1 = y[p * D + 1] - c[k][1], d2 = y[p * D + 2] - c[k][2];
          dist = fmaf(d2, d2, fmaf(d1, d1, d0 * d0));
        }
        if (k == 0 || dist < bd) { bd = dist; best = k; }
      }
      if (it == 0 || as[p] != best) ++changed;
      as[p] = best;
    }
    if (it > 0 && changed == 0) break;
    double A[OR_MAXK] = {0}, S[OR_MAXK][OR_MAXD] = {{0}};
    for (int64_t p = 0; p < N; ++p) {
      const double af = (double)(float)ah[p];
      A[as[p]] += af;
      for (int d = 0; d < D; ++d) S[as[p]][d] += af * (double)y[p * D + d];
    }
    for (int k = 0; k < K; ++k)
      if (A[k] > 0.0)
        for (int d = 0; d < D; ++d) c[k][d] = (float)(S[k][d] / A[k]);
  }
  *passes = it < iters ? it + 1 : iters;
  int Ko = 0;
  for (int k = 0; k < K; ++k) {
    double A = 0.0;
    comp nc;
    memset(&nc, 0, sizeof(nc));
    for (int64_t p = 0; p < N; ++p)
      if (as[p] == k) {
        A += ah[p];
        for (int d = 0; d < D; ++d) nc.mu[d] += ah[p] * vv[p * D + d];
      }
    if (!(A > 0.0)) continue;
    for (int d = 0; d < D; ++d) nc.mu[d] /= A;
    for (int64_t p = 0; p < N; ++p)
      if (as[p] == k)
        for (int i = 0; i < D; ++i)
          for (int j = 0; j < D; ++j)
            nc.S[i][j] += ah[p] * (vv[p * D + i] - nc.mu[i]) * (vv[p * D + j] - nc.mu[j]);
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) nc.S[i][j] /= A;
    nc.w = A / (double)N;
    if (!chol_floor(D, nc.S, nc.mu, nc.Lc, &nc.logdet)) {
      memcpy(nc.S, cov, sizeof(double) * OR_MAXD * OR_MAXD);
      chol_floor(D, nc.S, nc.mu, nc.Lc, &nc.logdet);
    }
    cs[Ko++] = nc;
  }
  free(y);
  free(as);
  return Ko;
}

typedef struct std_out {
  int32_t K, iters, aa_steps, aa_resets, km_passes;
  double W, lnL;
  uint32_t status;
} std_out;

/* Standard EM of one cell.  init: 0 = the paper's random particles (the
 * same Philox picks as the adaptive EM, K = min(Kmax, N), total
 * covariance, equal weights), 1 = K-means from those picks.  aa_m: Anderson
 * memory (0 = plain EM).  Iteration i evaluates g_i = G(theta_i), one
 * standard EM step, whose E-step also gives L(theta_i); EM stops when
 * |L_i - L_{i-1}| <= tol |L_{i-1}| (or after max_sweeps evaluations), and
 * the output is that last g: a standard EM step after the accelerated
 * iteration, which makes the moments exact (Sec. 4, as for the penalised
 * EM's final step).  With AA, from the first i with |L_i - L_{i-1}| <=
 * AA_START |L_{i-1}| on, theta_{i+1} is the Anderson extrapolation, unless it has a non-positive
 * weight or an indefinite covariance: then the history is cleared and
 * theta_{i+1} = g_i (Sec. 4); a dropped component restarts AA.  Ltrace:
 * L(theta_i) per evaluation.  mml = 1 replaces the EM map by the
 * simultaneous penalised step (mml_em_step; no AA): K0 lowered while
 * N - T K0 / 2 <= 0, convergence when the relative change of the penalised
 * L over an iteration without annihilation is at most tol, Ltrace the
 * penalised L, and the output one standard EM step from the last iterate
 * (the final unpenalised step of Sec. 2.3.1). */
static void std_cell(const oracle_cfg *cfg, int64_t cell, int64_t N, const double *vv,
                     const double *alpha, int init, int aa_m, int km_iters, int mml, double *prm_out,
                     std_out *o, double *Ltrace, int trace_cap, int *ntrace,
                     const double *init_prm, int init_K) {
  const int D = cfg->D, P = P_of(D);
  memset(o, 0, sizeof(*o));
  memset(prm_out, 0, sizeof(double) * (size_t)cfg->Kmax * P);
  if (ntrace) *ntrace = 0;
  if (N == 0) { o->status = ST_EMPTY; return; }
  double W = 0.0;
  for (int64_t p = 0; p < N; ++p) W += alpha[p];
  o->W = W;
  if (!(W > 0.0)) { o->status = ST_EMPTY | ST_DEGENERATE; return; }
  const double Nd = (double)N;
  double *ah = (double *)or_malloc(sizeof(double) * (size_t)N);
  double *gam = (double *)or_malloc(sizeof(double) * (size_t)N * OR_MAXK);
  for (int64_t p = 0; p < N; ++p) ah[p] = alpha[p] * Nd / W;
  if (N <= 10) o->status |= ST_TOO_FEW;
  double mean[OR_MAXD] = {0}, cov[OR_MAXD][OR_MAXD] = {{0}}, sd[OR_MAXD];
  for (int64_t p = 0; p < N; ++p)
    for (int d = 0; d < D; ++d) mean[d] += ah[p] * vv[p * D + d];
  for (int d = 0; d < D; ++d) mean[d] /= Nd;
  for (int64_t p = 0; p < N; ++p)
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j)
        cov[i][j] += ah[p] * (vv[p * D + i] - mean[i]) * (vv[p * D + j] - mean[j]);
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) cov[i][j] /= Nd;
  comp cs[OR_MAXK], g[OR_MAXK];
  {
    double Ltmp[OR_MAXD][OR_MAXD], ldtmp;
    if (!chol_floor(D, cov, mean, Ltmp, &ldtmp)) {
      cs[0].w = 1.0;
      for (int d = 0; d < D; ++d) cs[0].mu[d] = mean[d];
      memcpy(cs[0].S, cov, sizeof(cov));
      store_params(D, cfg->Kmax, 1, cs, prm_out);
      o->K = 1; o->status |= ST_DEGENERATE | ST_COV_NOT_PD;
      free(ah); free(gam);
      return;
    }
  }
  for (int d = 0; d < D; ++d) sd[d] = sqrt(cov[d][d]);
  /* the initial picks: the adaptive EM's procedure with K = min(Kmax, N)
   * (penalised: lowered while N - T K / 2 <= 0, as in the adaptive EM) */
  int K = cfg->Kmax < N ? cfg->Kmax : (int)N;
  if (mml)
    while (K > 1 && Nd - 0.5 * T_of(D) * K <= 0.0) --K;
  int64_t picks[OR_MAXK];
  {
    int got = 0;
    for (uint32_t t = 0; got < K; ++t) {
      int64_t idx;
      if (t < 100000u) {
        uint32_t r[4];
        philox_draw(cfg->seed, t, TAG_INIT, cell, r);
        double u = oracle_uniform52(r[0], r[1]);
        idx = (int64_t)floor(u * Nd);
        if (idx >= N) idx = N - 1;
      } else {
        idx = 0;
        for (;;) {
          int used = 0;
          for (int m = 0; m < got; ++m) used |= (picks[m] == idx);
          if (!used) break;
          ++idx;
        }
      }
      int dup = 0;
      for (int m = 0; m < got; ++m) dup |= (picks[m] == idx);
      if (!dup) picks[got++] = idx;
    }
  }
  if (init == 2 && init_prm && init_K > 0) {
    /* a supplied mixture (for tests: continue EM from a given fit) */
    K = init_K < cfg->Kmax ? init_K : cfg->Kmax;
    load_params(D, K, init_prm, cs);
    for (int k = 0; k < K; ++k) chol_floor(D, cs[k].S, cs[k].mu, cs[k].Lc, &cs[k].logdet);
  } else if (init == 1) {
    int passes = 0;
    K = kmeans_init(D, K, N, vv, ah, mean, sd, cov, picks, km_iters > 0 ? km_iters : 100, cs, &passes);
    o->km_passes = passes;
  } else {
    for (int k = 0; k < K; ++k) {
      cs[k].w = 1.0 / K;
      for (int d = 0; d < D; ++d) cs[k].mu[d] = vv[picks[k] * D + d];
      memcpy(cs[k].S, cov, sizeof(cov));
      chol_floor(D, cs[k].S, cs[k].mu, cs[k].Lc, &cs[k].logdet);
    }
  }
  aa_state *aa = (aa_state *)or_malloc(sizeof(aa_state));
  aa_init(aa, K * P, aa_m);
  double th[AA_MAXN], tg[AA_MAXN], tn[AA_MAXN];
  double Lprev = 0.0;
  int converged = 0, it, Kg = K, aa_on = 0, ann = 0, ann_prev = 0;
  if (mml) {
    /* simultaneous penalised EM (eq. omegak, annihilation) to convergence of
     * eq. (lnL-GM) over an iteration without annihilation, then the final
     * unpenalised step of Sec. 2.3.1 from the converged parameters */
    for (it = 0; it < cfg->max_sweeps; ++it) {
      const double L = mml_em_step(D, K, cs, N, vv, ah, gam, g, &Kg, &ann, &o->status);
      if (Ltrace && *ntrace < trace_cap) Ltrace[(*ntrace)++] = L;
      if (it > 0 && !ann_prev && fabs(L - Lprev) <= cfg->tol * fabs(Lprev)) { converged = 1; break; }
      if (it + 1 >= cfg->max_sweeps) break;
      Lprev = L;
      ann_prev = ann;
      K = Kg;
      memcpy(cs, g, sizeof(comp) * (size_t)K);
    }
    if (!converged) { o->status |= ST_EM_MAXSWEEPS; it = cfg->max_sweeps - 1; }
    /* the final step is from the last iterate whose L was evaluated */
    std_em_step(D, K, cs, N, vv, ah, gam, g, &Kg, &o->status);
    o->iters = it + 1;
    o->K = Kg;
    o->lnL = plain_L(D, Kg, g, N, vv, ah);
    store_params(D, cfg->Kmax, Kg, g, prm_out);
    free(ah);
    free(gam);
    return;
  }
  for (it = 0; it < cfg->max_sweeps; ++it) {
    const double L = std_em_step(D, K, cs, N, vv, ah, gam, g, &Kg, &o->status);
    if (Ltrace && *ntrace < trace_cap) Ltrace[(*ntrace)++] = L;
    if (it > 0 && fabs(L - Lprev) <= cfg->tol * fabs(Lprev)) { converged = 1; break; }
    if (!aa_on && it > 0 && fabs(L - Lprev) <= AA_START * fabs(Lprev)) aa_on = 1;
    Lprev = L;
    if (Kg < K || aa_m == 0 || !aa_on) { /* a dropped component restarts AA */
      if (Kg < K) aa_init(aa, Kg * P, aa_m);
      K = Kg;
      memcpy(cs, g, sizeof(comp) * (size_t)K);
      continue;
    }
    theta_pack(D, K, cs, mean, sd, th);
    theta_pack(D, K, g, mean, sd, tg);
    comp cand[OR_MAXK];
    if (aa_step(aa, th, tg, tn) && theta_unpack(D, K, tn, mean, sd, cand)) {
      renormalise(K, cand);
      memcpy(cs, cand, sizeof(comp) * (size_t)K);
      o->aa_steps++;
    } else {
      if (aa->h > 0) { aa_clear(aa); o->aa_resets++; }
      memcpy(cs, g, sizeof(comp) * (size_t)K);
    }
  }
  if (!converged) { it = cfg->max_sweeps - 1; o->status |= ST_EM_MAXSWEEPS; }
  K = Kg;
  o->iters = it + 1;
  o->K = K;
  o->lnL = plain_L(D, K, g, N, vv, ah);
  store_params(D, cfg->Kmax, K, g, prm_out);
  free(aa);
  free(ah);
  free(gam);
}

/* Exported: standard EM of a batch of cells (layout as oracle_compress);
 * iters/aa_steps/aa_resets/km_passes per cell (each may be NULL); mml = 1
 * runs the simultaneous penalised EM with annihilation (aa_m must be 0). */
int oracle_standard(const oracle_cfg *cfg, int64_t C, const int64_t *cell_off, const double *x,
                    const double *v, const double *alpha, int init, int aa_m, int km_iters,
                    int mml, int32_t *K_out, double *params_out, double *W_out, double *rho_target_out,
                    double *lnL_out, int32_t *iters_out, int32_t *aa_steps_out,
                    int32_t *aa_resets_out, int32_t *km_out, uint32_t *status_out,
                    const int64_t *cell_ids, int nthreads) {
  const int D = cfg->D;
  if (D != 1 && D != 3) return -1;
  if (cfg->Kmax < 1 || cfg->Kmax > OR_MAXK || aa_m < 0 || (mml && aa_m > 0)) return -1;
  const int64_t Ntot = cell_off[C];
  const size_t P = (size_t)P_of(D);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int64_t j = 0; j < C; ++j) {
    int64_t n = cell_off[j + 1] - cell_off[j];
    double *vv = (double *)or_malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * D);
    for (int64_t p = 0; p < n; ++p)
      for (int d = 0; d < D; ++d) vv[p * D + d] = v[(int64_t)d * Ntot + cell_off[j] + p];
    std_out o;
    std_cell(cfg, cell_ids ? cell_ids[j] : j, n, vv, alpha + cell_off[j], init, aa_m, km_iters, mml,
             params_out + (size_t)j * cfg->Kmax * P, &o, NULL, 0, NULL, NULL, 0);
    K_out[j] = o.K; W_out[j] = o.W; lnL_out[j] = o.lnL; status_out[j] = o.status;
    if (iters_out) iters_out[j] = o.iters;
    if (aa_steps_out) aa_steps_out[j] = o.aa_steps;
    if (aa_resets_out) aa_resets_out[j] = o.aa_resets;
    if (km_out) km_out[j] = o.km_passes;
    free(vv);
  }
  if (rho_target_out) deposit(cfg, C, cell_off, x, alpha, rho_target_out);
  return 0;
}

/* Exported: standard EM of one cell with the trace of L(theta_i); init = 2
 * starts from the supplied mixture init_prm [init_K][P] */
int oracle_std_cell(const oracle_cfg *cfg, int64_t cell, int64_t N, const double *vv /*[N][D]*/,
                    const double *alpha, int init, int aa_m, int km_iters, int mml,
                    double *params_out, int32_t *K_out, double *lnL_out, int32_t *iters_out, int32_t *aa_steps_out,
                    int32_t *aa_resets_out, int32_t *km_out, uint32_t *status_out, double *Ltrace,
                    int trace_cap, int32_t *ntrace, const double *init_prm, int init_K) {
  std_out o;
  int nt = 0;
  std_cell(cfg, cell, N, vv, alpha, init, aa_m, km_iters, mml, params_out, &o, Ltrace, trace_cap, &nt,
           init_prm, init_K);
  *K_out = o.K; *lnL_out = o.lnL; *iters_out = o.iters; *aa_steps_out = o.aa_steps;
  *aa_resets_out = o.aa_resets; *km_out = o.km_passes; *status_out = o.status;
  if (ntrace) *ntrace = nt;
  return 0;
}

/* Exported: the Anderson iteration above on the affine map G(x) = A x + b
 * (n <= AA_MAXN, row-major A), from x0 for iters steps; writes the iterate
 * and the residual norm ||G(x_i) - x_i|| per step.  For a test of the
 * extrapolation itself. */
int oracle_aa_affine(int n, const double *A, const double *b, const double *x0, int m, int iters,
                     double *x_out, double *res_trace) {
  if (n < 1 || n > AA_MAXN) return -1;
  aa_state *s = (aa_state *)or_malloc(sizeof(aa_state));
  aa_init(s, n, m);
  double x[AA_MAXN], g[AA_MAXN], xn[AA_MAXN];
  memcpy(x, x0, sizeof(double) * (size_t)n);
  for (int it = 0; it < iters; ++it) {
    double r = 0.0;
    for (int i = 0; i < n; ++i) {
      double t = b[i];
      for (int j = 0; j < n; ++j) t += A[i * n + j] * x[j];
      g[i] = t;
      r += (t - x[i]) * (t - x[i]);
    }
    res_trace[it] = sqrt(r);
    aa_step(s, x, g, xn);
    memcpy(x, xn, sizeof(double) * (size_t)n);
  }
  memcpy(x_out, x, sizeof(double) * (size_t)n);
  free(s);
  return 0;
}

/* Exported: the K-means initialisation alone on one cell ([N][D]), from the
 * given initial centre indices; normalised weights ah (sum N) */
int oracle_kmeans(int D, int K, int64_t N, const double *vv, const double *ah,
                  const int64_t *picks, int iters, double *params_out, int32_t *K_out,
                  int32_t *passes_out) {
  if (D != 1 && D != 3) return -1;
  if (K < 1 || K > OR_MAXK || N < 1) return -1;
  const double Nd = (double)N;
  double mean[OR_MAXD] = {0}, cov[OR_MAXD][OR_MAXD] = {{0}}, sd[OR_MAXD];
  for (int64_t p = 0; p < N; ++p)
    for (int d = 0; d < D; ++d) mean[d] += ah[p] * vv[p * D + d];
  for (int d = 0; d < D; ++d) mean[d] /= Nd;
  for (int64_t p = 0; p < N; ++p)
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j)
        cov[i][j] += ah[p] * (vv[p * D + i] - mean[i]) * (vv[p * D + j] - mean[j]);
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) cov[i][j] /= Nd;
  for (int d = 0; d < D; ++d) sd[d] = sqrt(cov[d][d]);
  comp cs[OR_MAXK];
  int passes = 0;
  const int Ko = kmeans_init(D, K, N, vv, ah, mean, sd, cov, picks, iters, cs, &passes);
  store_params(D, K, Ko, cs, params_out);
  *K_out = Ko;
  *passes_out = passes;
  return 0;
}
