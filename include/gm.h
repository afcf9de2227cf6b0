/*
 * gm.h -- C ABI of the GB300 Gaussian-mixture checkpoint-restart library
 * (method of Chen, Chacon & Nguyen, arXiv 2007.12273).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - All array arguments are DEVICE pointers owned by the caller, unless a
 *    comment says otherwise.  The library never frees or keeps them.
 *  - Particles are sorted by spatial cell (CSR): the particles of cell j are
 *    indices cell_off[j] .. cell_off[j+1]-1 (cell_off has C+1 int64 entries,
 *    cell_off[0] = 0, non-decreasing).  Positions are absolute, in
 *    [j*dx, (j+1)*dx) for a particle of cell j, with dx = L / C.
 *  - Velocities are structure-of-arrays: v[d * n + i] is component d of
 *    particle i, d < D, n the number of particles of that array.
 *  - The mesh is 1D and periodic: node i sits at (i + 1/2) dx.
 *  - A component's parameter record (the checkpoint payload, Sec. 1) is
 *      [ omega, mu_0 .. mu_{D-1}, Sigma upper triangle row-major ]
 *    P = 1 + D + D(D+1)/2 doubles (3 for D = 1, 10 for D = 3); a cell's
 *    records are params[(j * Kmax + k) * P + t]; slots k >= K[j] are zero.
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = the legacy
 *    default stream).  Return value: GM_OK or a negative GM_ERR_* code;
 *    gm_last_error() then describes the failure (per host thread).
 *    Per-cell outcomes that are not errors go in status bits (GM_ST_*).
 *  - The library keeps one internal device workspace per process (grown on
 *    demand, freed by gm_shutdown()).  Concurrent calls from several host
 *    threads or on several streams must be serialised by the caller.
 */
#ifndef GMCR_GM_H
#define GMCR_GM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define GM_OK 0
#define GM_ERR_ARG (-1)         /* invalid argument; nothing was launched */
#define GM_ERR_CUDA (-2)        /* a CUDA call or launch failed */
#define GM_ERR_NOMEM (-3)       /* workspace allocation failed */
#define GM_ERR_UNSUPPORTED (-4) /* e.g. no sm_103 device */

/* per-cell status bits */
#define GM_ST_EM_MAXSWEEPS 0x01u  /* EM stopped at max_sweeps, not converged */
#define GM_ST_COV_NOT_PD 0x02u    /* a covariance failed its Cholesky factorisation */
#define GM_ST_TOO_FEW 0x04u       /* cell has at most 10 particles (Sec. 1) */
#define GM_ST_EMPTY 0x08u         /* no particles, or non-positive total weight */
#define GM_ST_DEGENERATE 0x10u    /* all velocities (numerically) equal */
#define GM_ST_PROJ_SKIPPED 0x100u /* Lemons numerator <= 0: projection skipped */
#define GM_ST_NEG_WEIGHT 0x200u   /* a corrected weight alpha' <= 0 */
#define GM_ST_MM_EMPTY_COL 0x400u /* no resampled particle: unit mass-matrix column */
#define GM_ST_NO_MIXTURE 0x800u   /* K[j] = 0 but particles were requested */
#define GM_ST_MM_NOT_CONVERGED 0x1000u /* 2D mass-matrix solve stopped at its iteration cap */
#define GM_ST_BAD_RANGE 0x2000u   /* out_off[j] .. out_off[j+1] not inside [0, n_out): the
                                     cell gets no particles and nothing is written for it */

typedef struct gm_config {
  int32_t D;           /* velocity dimensions: 1 or 3 */
  int32_t Kmax;        /* initial components per cell, 1..16 */
  int32_t shape_order; /* 1 = CIC (linear B-spline), 2 = quadratic B-spline */
  int32_t max_sweeps;  /* cap on EM sweeps (e.g. 1000) */
  double tol;          /* EM stops when |L - L_prev| <= tol |L_prev| (e.g. 1e-6) */
  uint64_t seed;       /* Philox key: initial picks (compress) / sampler (reconstruct) */
  double L;            /* periodic domain length; dx = L / C */
  double q;            /* species charge q_p; nonzero for the reconstructions (GM_ERR_ARG) */
  int32_t threads_per_cell; /* EM CTA size: 0 = library choice, else 64, 128 or 256 */
  int32_t smem_particles;   /* EM shared-memory tile in particles: 0 = library choice;
                               cells with more particles use an L2-resident global tile */
  int32_t precision;        /* penalised sweeps' M-step: 0 (default) = FP64 -- the
                               cross-warp statistic sums, covariance, its factor and
                               inverse, the weight -- with the convergence test's
                               log-likelihood corrected to first order for the
                               rounding of the FP32 E-step constants; 1 = FP32
                               M-step and uncorrected test (faster; its stopping
                               sweep follows the FP64 method less closely).  Either
                               way the component means are accumulated to about 48
                               bits (FP64, or a pair of FP32 numbers) and the final
                               unpenalised step is entirely FP64.  Another value,
                               like a threads_per_cell or smem_particles out of
                               range, is GM_ERR_ARG (before any device call) */
  int32_t reserved;         /* must be 0 */
} gm_config;

/*
 * gm_compress -- per-cell adaptive Gaussian-mixture fit (Sec. 2.2-2.3).
 *
 * For every cell: weights are normalised to sum N (Sec. 2.2); Kmax
 * components start at randomly chosen particles (Philox key cfg->seed,
 * counter (draw, 0x494E4954, cell)) with the total covariance; the
 * component-wise penalised EM (eqs. responsibility, muk, sigmak, omegak)
 * removes a component when N_k - T/2 <= 0 and stops when the penalised
 * log-likelihood, eq. (lnL-GM), changes by at most tol (relative) over a
 * sweep with no removal; a final unpenalised step (eq. omegak-mle,
 * Sec. 2.3.1) then makes the mixture's mass, mean and covariance equal the
 * cell's weighted sample moments.  Also deposits the target charge density
 * rho'_i = (q/dx) sum_p alpha_p S(x_i - x_p) (Sec. 2.4.1).
 *
 * In:  cell_off [C+1] int64; x [n] f64; v [D][n] f32 (v_is_f64 = 0) or f64
 *      (v_is_f64 = 1); alpha [n] f64.  n = n_particles = cell_off[C].
 * Out: K_out [C] int32; params_out [C][Kmax][P] f64; W_out [C] f64 (sum of
 *      weights); rho_target_out [C] f64; lnL_out [C] f64 (eq. lnL-GM at the
 *      final parameters, with the normalised weights); sweeps_out [C] int32;
 *      kwork_out [C] int32 (component E-steps performed, may be NULL);
 *      status_out [C] uint32.
 *      x and rho_target_out may both be NULL: no 1D deposit (a 2D mesh
 *      takes its target charge from gm_deposit_2d).
 * E-step densities and responsibilities are FP32; the per-component
 * statistics are FP32 per thread and warp and summed across warps in the
 * M-step's precision (cfg->precision); component means are accumulated in
 * FP64; the log-likelihood of the convergence test is summed in FP64; the
 * whole final step (which makes the moments exact) is FP64.
 */
int gm_compress(const gm_config* cfg, int64_t C, int64_t n_particles, const int64_t* cell_off,
                const double* x, const void* v, int32_t v_is_f64, const double* alpha,
                int32_t* K_out, double* params_out, double* W_out, double* rho_target_out,
                double* lnL_out, int32_t* sweeps_out, int32_t* kwork_out, uint32_t* status_out,
                void* stream);

/*
 * gm_reconstruct -- resample every cell from its mixture (Sec. 2.4).
 *
 * Cell j gets N'_j = out_off[j+1] - out_off[j] particles: position uniform
 * in the cell; a component z with probability omega_z and v ~ N(mu_z,
 * Sigma_z) (ancestral sampling, eq. mix-dist-1), Philox key cfg->seed,
 * counter (i, 0x53000000 | block, cell); weight W_j / N'_j.  Then the
 * Gauss'-law correction: alpha'_p = alpha_p + dA_j with M dA = dx (rho' -
 * rho), M_ij = sum_p q S0(x_j - x_p) S(x_i - x_p) (eqs. p-weight-correction,
 * new-p-weight; solved directly in FP64).  Then the Lemons projection
 * v' = a (v + beta) restoring the mixture's momentum and energy per cell
 * (eqs. alpha, beta); a cell whose numerator 2 E N' - p^2 is not positive
 * keeps its samples and gets GM_ST_PROJ_SKIPPED.
 *
 * In:  K [C] int32; params [C][Kmax][P] f64; W [C] f64; rho_target [C] f64;
 *      out_off [C+1] int64, n_out = out_off[C].
 * Out: x_out [n_out] f64; v_out [D][n_out] f64; alpha_out [n_out] f64;
 *      status_out [C] uint32; dA_out [C] f64 (may be NULL).
 * Box-Muller normals are FP32; everything else is FP64.  For D = 3 the
 * counter's block 1 gives two (radius, angle) pairs of 32-bit uniforms;
 * for D = 1 one pair of 52-bit uniforms.  The three output arrays
 * also hold each particle's draw between the call's two particle passes:
 * until the call completes on the stream their contents are not the
 * result, and they must not alias each other or the inputs.
 * Errors: GM_ERR_ARG (bad cfg, q = 0, negative sizes, NULL required
 * pointers), GM_ERR_UNSUPPORTED (no sm_103 device), GM_ERR_NOMEM
 * (workspace), GM_ERR_CUDA (launch); per-cell outcomes in status bits.
 */
int gm_reconstruct(const gm_config* cfg, int64_t C, const int32_t* K, const double* params,
                   const double* W, const double* rho_target, int64_t n_out,
                   const int64_t* out_off, double* x_out, double* v_out, double* alpha_out,
                   uint32_t* status_out, double* dA_out, void* stream);

/*
 * The 2D doubly periodic mesh (the geometry of the paper's 2D-3V Weibel
 * runs, Sec. 3.2): Cx x Cy cells of dx = Lx / Cx, dy = Ly / Cy, numbered
 * j = jy * Cx + jx (particles sorted by that index, CSR as everywhere);
 * node (ix, iy) at the cell centre ((ix + 1/2) dx, (iy + 1/2) dy); the
 * shape function is the tensor product S(x) S(y) of cfg->shape_order.
 * cfg->L is not used by these calls.
 */
typedef struct gm_mesh2d {
  int64_t Cx, Cy; /* cells along x and y (1 .. 2^24 each, Cx * Cy < 2^31) */
  double Lx, Ly;  /* domain lengths */
} gm_mesh2d;

/*
 * gm_deposit_2d -- charge density on the 2D mesh (Sec. 2.4.1):
 * rho_i = (q / (dx dy)) sum_p alpha_p S(x_i - x_p) S(y_i - y_p).
 * In: cell_off [Cx Cy + 1] int64; x, y [n] f64 (each particle inside its
 * cell); alpha [n] f64 or NULL (unit weights).  Out: rho_out [Cy][Cx] f64
 * (node jy * Cx + jx).  This is the target rho' of the 2D reconstruction
 * when called on the particles before compression.  Errors: GM_ERR_ARG (bad
 * cfg or mesh, NULL required pointers), GM_ERR_UNSUPPORTED, GM_ERR_NOMEM,
 * GM_ERR_CUDA.
 */
int gm_deposit_2d(const gm_config* cfg, const gm_mesh2d* mesh, const int64_t* cell_off,
                  const double* x, const double* y, const double* alpha, double* rho_out,
                  void* stream);

/*
 * gm_reconstruct_2d -- gm_reconstruct on the 2D mesh (Sec. 2.4).
 *
 * Positions uniform in the cell: x from the same uniform as in 1D, y from
 * Philox block 3 (counter (i, 0x53000003, cell), words 0-1); velocities and
 * weights W_j / N'_j as in gm_reconstruct.  Gauss' law: alpha'_p = alpha_p +
 * dA_j with M dA = dx dy (rho' - rho), M_ij = q sum_{p in j} S(x_i - x_p)
 * S(y_i - y_p) (eqs. p-weight-correction, new-p-weight; a 3 x 3 column per
 * cell).  In 2D with the quadratic B-spline M is not diagonally dominant; it
 * is solved by defect correction preconditioned with the matrix of
 * uniformly filled cells (cyclic tridiagonal solves along x and along y),
 * until max |residual| <= 1e-14 max |dx dy rho'| or 64 iterations
 * (GM_ST_MM_NOT_CONVERGED on every cell).  A cell without resampled
 * particles gets a unit column (GM_ST_MM_EMPTY_COL), as in 1D.  Then the
 * Lemons projection per cell, as in gm_reconstruct.
 *
 * In: as gm_reconstruct with rho_target [Cy][Cx] and out_off [Cx Cy + 1]
 * (cfg->q must be nonzero).  Out: x_out, y_out [n_out] f64, v_out
 * [D][n_out] f64, alpha_out [n_out] f64, status_out [Cx Cy] uint32, dA_out
 * [Cx Cy] f64 (may be NULL).  Errors as gm_reconstruct (and a bad mesh);
 * a solve that stops at its iteration cap sets GM_ST_MM_NOT_CONVERGED.
 */
int gm_reconstruct_2d(const gm_config* cfg, const gm_mesh2d* mesh, const int32_t* K,
                      const double* params, const double* W, const double* rho_target,
                      int64_t n_out, const int64_t* out_off, double* x_out, double* y_out,
                      double* v_out, double* alpha_out, uint32_t* status_out, double* dA_out,
                      void* stream);

/*
 * gm_moments -- per-cell particle moments (the quantities of Sec. 2.3.1 and
 * 2.4.2): W = sum alpha, p = sum alpha v [C][D], M2 = sum alpha v v^T upper
 * triangle row-major [C][D(D+1)/2], E = (1/2) sum alpha |v|^2, and the
 * charge density rho [C] with the shape function of cfg (Sec. 2.4.1).
 * Any output pointer may be NULL.  FP64 accumulation.  Errors: GM_ERR_ARG
 * (bad cfg, negative sizes, NULL inputs), GM_ERR_UNSUPPORTED, GM_ERR_NOMEM,
 * GM_ERR_CUDA; C = 0 is a no-op.
 */
int gm_moments(const gm_config* cfg, int64_t C, int64_t n_particles, const int64_t* cell_off,
               const double* x, const void* v, int32_t v_is_f64, const double* alpha, double* W,
               double* p, double* M2, double* E, double* rho, void* stream);

/*
 * gm_mixture_moments -- the same moments of each cell's mixture (W given):
 * p = W sum_k w_k mu_k, M2 = W sum_k w_k (Sigma_k + mu_k mu_k^T),
 * E = tr(M2)/2 (eq. equal-mean and the variance identity of Sec. 2.3.1).
 * In: K [C] int32, params [C][Kmax][P] f64, Wc [C] f64; out as
 * gm_moments.  Errors as gm_moments; C = 0 is a no-op.
 */
int gm_mixture_moments(const gm_config* cfg, int64_t C, const int32_t* K, const double* params,
                       const double* Wc, double* W, double* p, double* M2, double* E,
                       void* stream);

/*
 * gm_reconstruct_noalloc -- gm_reconstruct without any device allocation.
 *
 * The paper has no counterpart: this is a library-usage variant.  Some
 * callers cannot allocate device memory while they run -- a host code whose
 * device memory is owned by its own allocator or by a fixed budget, or one
 * that must not pay the device-wide synchronisation that cudaFree/cudaMalloc
 * imply (gm_reconstruct grows its workspace that way).  This entry point
 * computes exactly what gm_reconstruct computes, with the same arguments,
 * but takes its scratch from a fixed 40 MiB array that the library reserves
 * statically on every GPU that loads it, held until the process exits.
 *
 * Limits and rules:
 *  - at most 32768 cells per call (C > 32768 returns GM_ERR_ARG);
 *  - the first call on a device looks up the array's device address (once
 *    per device, with that device current).  Under CUDA's lazy module
 *    loading that first use of the library's device module on a device is
 *    also when the CUDA runtime loads the module and reserves the array,
 *    which may allocate device memory and synchronise.  A call with C = 0
 *    does only this set-up (device check, address lookup; nothing is
 *    launched): make such a call, or the first real call, before any
 *    stream capture and before the point where no allocation may happen;
 *  - out_off is read on the device: a cell whose range out_off[j] ..
 *    out_off[j+1] does not lie inside [0, n_out) gets no particles and
 *    GM_ST_BAD_RANGE, and nothing is written for it;
 *  - every call shares the one array: calls that overlap on the GPU (other
 *    streams, other host threads) race and must be serialised by the
 *    caller; the array keeps the last call's contents, and nothing in it has
 *    to start at zero (each call writes every entry before reading it);
 *  - no cudaMalloc, cudaFree or allocating library routine is called.
 */
/*
 * Per-kernel device times (the library's stage timer; the paper has no
 * counterpart).  gm_trace_begin starts a trace: from then on, outside CUDA
 * graph capture, the library records a CUDA event on the launching stream
 * after each of its main kernels and at the start of each call; the time
 * between consecutive events is the kernel's.  gm_trace_end synchronises
 * the events, stops the trace and returns the number of distinct kernel
 * names (or a negative GM_ERR_*); gm_trace_get(i, ...) returns name i
 * (NUL-terminated, truncated to name_len - 1), its total milliseconds and
 * its number of launches.  Host-side only besides the events; one trace
 * per process at a time.
 */
int gm_trace_begin(void);
int gm_trace_end(void);
int gm_trace_get(int32_t i, char* name, int32_t name_len, double* ms, int32_t* launches);

/*
 * gm_convert -- the library's FP32 <-> FP64 conversions (no counterpart in
 * the paper).  GB300 runs FP64, and conversions to and from it, at 1/64 of
 * the FP32 rate, so the kernels convert on the integer pipe instead; this
 * entry point applies those conversions to an array so that they can be
 * checked against the hardware's.
 *   dir 0: in [n] FP32 -> out [n] FP64, exact for every finite value
 *          (subnormals and signed zeros included); infinities stay
 *          infinities, a NaN becomes a quiet NaN;
 *   dir 1: in [n] FP64 -> out [n] FP32 with the mantissa truncated toward
 *          zero; below FP32's normal range the value truncates to a
 *          subnormal or a signed zero, from 2^128 up (and infinities) it
 *          becomes a signed infinity, a NaN a quiet NaN.
 * in and out are caller-owned device arrays; asynchronous on stream.
 * Returns GM_ERR_ARG for n < 0, dir not 0 or 1, or a null array with n > 0;
 * GM_ERR_CUDA if the launch fails.
 */
int gm_convert(int32_t dir, int64_t n, const void* in, void* out, void* stream);

/* gm_noalloc_limits_ok -- 1 if the scratch a call of 32768 cells needs
 * (D = 1 and D = 3, Kmax = 16) fits the 40 MiB array of gm_reconstruct_noalloc, else 0:
 * a host-side self-check of that limit (no counterpart in the paper); it
 * touches no device and returns no error code. */
int gm_noalloc_limits_ok(void);
int gm_reconstruct_noalloc(const gm_config* cfg, int64_t C, const int32_t* K, const double* params,
                           const double* W, const double* rho_target, int64_t n_out,
                           const int64_t* out_off, double* x_out, double* v_out,
                           double* alpha_out, uint32_t* status_out, double* dA_out,
                           void* stream);

/*
 * gm_gemm_bf16 -- C[M,N] = A[M,K] B[N,K]^T (+ bias[N]) (ReLU if relu != 0)
 * (entries set to 0 where mask[row * ldm + col] <= 0, if mask != NULL), on
 * the tcgen05 tensor cores with FP32 accumulation.  Used by the learned
 * initialisation network (not part of the paper's method).
 *
 * A, B: BF16, row-major with K contiguous, leading dimensions lda, ldb
 * (multiples of 8, >= K), 16-byte aligned; bias: FP32 [N] or NULL; mask:
 * BF16 [M][ldm] or NULL; outputs C_f32 (FP32) and/or C_bf16 (BF16), row
 * stride ldc.  err (device, may be NULL) gets bit 0 set if a tensor-core
 * completion wait timed out (results then undefined).  Errors: GM_ERR_ARG
 * (negative sizes, NULL operands, leading dimensions or alignment as
 * above), GM_ERR_UNSUPPORTED (no sm_103 device), GM_ERR_CUDA (launch).
 */
int gm_gemm_bf16(int32_t M, int32_t N, int32_t K, const void* A, int32_t lda, const void* B,
                 int32_t ldb, const float* bias, int32_t relu, const void* mask, int32_t ldm,
                 float* C_f32, void* C_bf16, int32_t ldc, uint32_t* err, void* stream);

/*
 * gm_compress_from -- gm_compress started from given initial mixtures
 * instead of the paper's random initialisation (Sec. 2.3); used by the
 * learned initialisation.  init_K [C] int32 and init_params [C][Kmax][P]
 * f64 (original coordinates, gm_compress's record layout).  Components
 * whose covariance fails the Cholesky floor are dropped, the count is
 * capped so that N - T K / 2 > 0, and a cell left with none falls back to
 * the random initialisation.  Everything after the initialisation is the
 * paper's method, as in gm_compress; so are the errors (and GM_ERR_ARG
 * when init_K or init_params is NULL).
 */
int gm_compress_from(const gm_config* cfg, int64_t C, int64_t n_particles,
                     const int64_t* cell_off, const double* x, const void* v, int32_t v_is_f64,
                     const double* alpha, const int32_t* init_K, const double* init_params,
                     int32_t* K_out, double* params_out, double* W_out, double* rho_target_out,
                     double* lnL_out, int32_t* sweeps_out, int32_t* kwork_out,
                     uint32_t* status_out, void* stream);

/*
 * Learned initialisation (not in the paper).  A small network maps per-cell
 * features to an initial mixture from which gm_compress_from runs the
 * paper's EM.
 *
 * Features of a cell (gm_features): with W = sum alpha, the alpha-weighted
 * mean and per-dimension standard deviation sd (written to wstat [C][2D]:
 * mean, then sd), y = (v - mean)/sd and alpha-weighted expectations E[.]:
 *   D = 1: [E y^3, E y^4 - 3, ln(N)/10, 64-bin histogram of y on [-4, 4)]
 *   D = 3: [E y_d^3 (3), E y_d^4 - 3 (3), E y0y1, E y0y2, E y1y2, ln(N)/10,
 *           8x8x8 histogram of y on [-2.5, 2.5)^3, index b0*64 + b1*8 + b2]
 * (histogram entry = alpha mass in the bin / W * number of bins; values
 * outside the range go to the edge bins), zero-padded to F = 128 (D = 1) or
 * 576 (D = 3), BF16 [C][F].
 *
 * Network: h1 = relu(x W1^T + b1), h2 = relu(h1 W2^T + b2),
 * h3 = relu(h2 W3^T + b3), out = h3 W4^T + b4 (FP32 [M][O]); hidden width
 * H = 256.  out holds Kmax slots of SP = 2 + 2D + D(D-1)/2 values
 * [presence logit, log weight, mu (D), log diag of L (D), L10, L20, L21] in
 * the whitened coordinates y (Sigma = L L^T), O = Kmax SP rounded up to a
 * multiple of 16.
 */
typedef struct gm_mlp {
  int32_t D, Kmax;  /* velocity dimensions, slots */
  int32_t F, H, O;  /* widths: features, hidden, output */
  float* W[4];      /* FP32 master weights, row-major [out][in]: HxF, HxH, HxH, OxH */
  float* b[4];      /* FP32 biases [out] */
  void* W16[4];     /* BF16 copies [out][in] */
  void* WT16[4];    /* BF16 transposes [in][out] */
  float* gW[4];     /* gradients (written by gm_mlp_train_step) */
  float* gb[4];
  float* mW[4];     /* Adam first / second moments */
  float* vW[4];
  float* mb[4];
  float* vb[4];
} gm_mlp;

/* Features (see above) of every cell (learned initialisation, not in the
 * paper); wstat [C][2D] gets mean and sd.  Device arrays as gm_compress;
 * feat BF16 [C][F] and wstat caller-owned.  GM_ERR_ARG for a bad cfg,
 * negative sizes or a NULL required pointer. */
int gm_features(const gm_config* cfg, int64_t C, int64_t n_particles, const int64_t* cell_off,
                const void* v, int32_t v_is_f64, const double* alpha, void* feat, double* wstat,
                void* stream);

/* Training targets (learned initialisation, not in the paper) from the
 * paper's fits (K, params: gm_compress outputs, Sec. 2.2-2.3) and the
 * cells' wstat: components sorted by whitened mu_0; slot s < K gets
 * presence 1 and [ln w, mu, ln diag L, L10, L20, L21] of the whitened
 * component, slots s >= K presence 0.  T, Mk: FP32 [C][O], caller-owned;
 * Mk marks the entries that enter the loss.  GM_ERR_ARG for a bad cfg,
 * O < Kmax SP or a NULL pointer. */
int gm_mlp_targets(const gm_config* cfg, int64_t C, const int32_t* K, const double* params,
                   const double* wstat, int32_t O, float* T, float* Mk, void* stream);

/* BF16 copies and transposes of the FP32 master weights (after the caller
 * sets or loads W).  Not in the paper.  GM_ERR_ARG for a malformed net. */
int gm_mlp_sync(const gm_mlp* net, void* stream);

/* Device scratch that gm_mlp_forward / gm_mlp_train_step need for M rows
 * (not in the paper); 0 for a NULL net or M <= 0 (no error code). */
size_t gm_mlp_scratch_bytes(const gm_mlp* net, int32_t M);

/* out [M][O] = network(X [M][F] BF16), FP32 (learned initialisation, not
 * in the paper).  M any; scratch of at least gm_mlp_scratch_bytes(net, M)
 * bytes, caller-owned.  GM_ERR_ARG for a malformed net, M < 0, a NULL
 * pointer or short scratch; *err (device, may be NULL) as gm_gemm_bf16. */
int gm_mlp_forward(const gm_mlp* net, int32_t M, const void* X, void* scratch,
                   size_t scratch_bytes, float* out, uint32_t* err, void* stream);

/* One training step (learned initialisation, not in the paper) on a batch
 * of M rows (M a multiple of 64, else GM_ERR_ARG; so are NULL pointers,
 * short scratch and step < 1 with lr > 0): forward,
 * loss (mean over rows: sum over slots of softplus(p) - t p on presence
 * logits plus squared errors on the entries Mk marks) added to *loss
 * (device FP64), backward into net->gW / net->gb, and, if lr > 0, an Adam
 * update (beta1 0.9, beta2 0.999, eps 1e-8, bias correction with step
 * number `step` >= 1) that also refreshes the BF16 copies. */
int gm_mlp_train_step(const gm_mlp* net, int32_t M, const void* X, const float* T,
                      const float* Mk, float lr, int32_t step, void* scratch,
                      size_t scratch_bytes, float* out, double* loss, uint32_t* err,
                      void* stream);

/* Initial mixtures from the network's output: slots whose presence logit
 * exceeds presence_logit (at least the most likely one; 0 = presence
 * probability above 1/2, negative values start EM with more components,
 * which the annihilation may remove again), capped so that N - T K0 / 2 > 0
 * by dropping the smallest log weights; weights by softmax of the log
 * weights; mu = mean + sd * mu_w, Sigma = diag(sd) L L^T diag(sd) with
 * ln diag L clamped to [-10, 5].  K0 [C], init_params [C][Kmax][P]
 * (caller-owned, the layout gm_compress_from takes).  Learned
 * initialisation, not in the paper; the cap is eq. (omegak)'s survival
 * condition (Sec. 2.2).  GM_ERR_ARG for a bad cfg, O < Kmax SP, a NULL
 * pointer or a NaN presence_logit. */
int gm_mlp_decode(const gm_config* cfg, int64_t C, const float* out, int32_t O,
                  const double* wstat, const int64_t* cell_off, float presence_logit, int32_t* K0,
                  double* init_params, void* stream);

/*
 * gm_compress_standard -- standard (non-adaptive) EM with optional K-means
 * initialisation and Anderson acceleration: the acceleration study of
 * Sec. 4, where the paper applies both to the non-adaptive EM-GM algorithm
 * (the adaptive, penalised EM of gm_compress is the paper's main method).
 *
 * K = min(Kmax, N) components start at the paper's random particles (the
 * same Philox picks as gm_compress) with the total covariance and equal
 * weights, or (opts->init = 1) at a K-means partition grown from those
 * picks: Lloyd passes in the cell's whitened coordinates until no
 * assignment changes (at most opts->kmeans_iters, 0 = 100), one component
 * per non-empty cluster with its weight share, mean and covariance (the
 * total covariance if that fails the Cholesky floor).  Each iteration is
 * one standard EM step -- the E-step of all components with the same
 * parameters, then eqs. (muk), (sigmak) and omega_k = N_k / N (eq.
 * omegak-mle); it stops when the unpenalised log-likelihood
 * sum_p alpha_p ln sum_k omega_k f_k(v_p) changes by at most cfg->tol
 * (relative), or after cfg->max_sweeps steps (GM_ST_EM_MAXSWEEPS).  With
 * opts->aa_memory = m > 0 (at most 8), once that relative change is at
 * most 1e-4 the next iterate is the Anderson extrapolation of the last m
 * steps on (omega_k, mu_k, M2_k = Sigma_k + mu_k mu_k^T) in whitened
 * coordinates, unless it has a non-positive weight or an indefinite
 * covariance, in which case the history is cleared and the plain EM step
 * is taken.  A component that owns nothing or whose covariance fails the
 * floor is dropped.  The output is one more standard EM step, in FP64,
 * which makes the mixture's mass, mean and covariance the cell's weighted
 * sample moments; lnL_out is the unpenalised log-likelihood of the output.
 *
 * opts->penalised = 1 runs the simultaneous variant of the paper's
 * adaptive EM instead (Sec. 2.2-2.3 with all components updated at once;
 * opts->aa_memory must be 0): K0 = min(Kmax, N) lowered while
 * N - T K0 / 2 <= 0 (T = D(D+3)/2); each iteration the E-step of all
 * components with the same parameters, then every M-step, with
 * omega_k = (N_k - T/2) / sum over survivors (N_j - T/2) (eq. omegak,
 * renormalised); a component with N_k - T/2 <= 0 or a covariance failing
 * the floor is annihilated, the last one never (the one with the largest
 * N_k stays).  It stops when the penalised log-likelihood (eq. lnL-GM)
 * changes by at most cfg->tol (relative) over an iteration with no
 * annihilation; the output is the final unpenalised FP64 step of
 * Sec. 2.3.1 from the last iterate, as above.
 *
 * Arguments as gm_compress (cfg->threads_per_cell and cfg->precision are
 * not used; cfg->smem_particles sets the shared tile); iters_out [C]: EM
 * steps evaluated; aa_steps_out, aa_resets_out: extrapolations taken and
 * history resets; km_passes_out: Lloyd passes (each of these may be NULL).
 * Errors as gm_compress, and GM_ERR_ARG for options out of range (init not
 * 0 or 1, aa_memory outside 0..8, Anderson with the penalised variant).
 */
typedef struct gm_std_opts {
  int32_t init;         /* 0 = random particles (Sec. 2.3), 1 = K-means */
  int32_t aa_memory;    /* Anderson memory m, 0 = plain EM, at most 8 */
  int32_t kmeans_iters; /* cap on Lloyd passes, 0 = 100 */
  int32_t penalised;    /* 1 = simultaneous penalised EM with annihilation, else 0 */
} gm_std_opts;
int gm_compress_standard(const gm_config* cfg, const gm_std_opts* opts, int64_t C,
                         int64_t n_particles, const int64_t* cell_off, const double* x,
                         const void* v, int32_t v_is_f64, const double* alpha, int32_t* K_out,
                         double* params_out, double* W_out, double* rho_target_out,
                         double* lnL_out, int32_t* iters_out, int32_t* aa_steps_out,
                         int32_t* aa_resets_out, int32_t* km_passes_out, uint32_t* status_out,
                         void* stream);

/*
 * gm_anderson_affine -- the Anderson extrapolation of gm_compress_standard
 * (Sec. 4), run by itself on the affine map G(x) = A x + b: iters steps
 * from x0 with memory m (0..8), n <= 160 unknowns.  A [n][n] row-major, b,
 * x0 [n] in; x_out [n] the last iterate, res_out [iters] the residual norm
 * ||G(x_i) - x_i|| of every step (device arrays, FP64).  It exists to check
 * the extrapolation's arithmetic apart from the EM map (on a linear map
 * Anderson acceleration with m >= n reaches the fixed point in about n + 1
 * steps).  GM_ERR_ARG for sizes out of range or NULL pointers.
 */
int gm_anderson_affine(int32_t n, const double* A, const double* b, const double* x0,
                       int32_t memory, int32_t iters, double* x_out, double* res_out,
                       void* stream);

/*
 * Pipeline capture into a CUDA graph.  The paper has no counterpart: this
 * is how a caller replays a fixed compress / reconstruct (and learned
 * initialisation) pipeline with one launch.
 *
 * gm_graph_begin starts capturing `stream` (relaxed capture mode).  Every
 * library call this host thread issues until gm_graph_end must go to that
 * stream; each one that needs device workspace gets a buffer of its own,
 * allocated at capture time and owned by the graph (so graphs and direct
 * calls never share workspace).  gm_graph_end ends the capture and
 * instantiates the graph into *out.  gm_graph_launch replays it on any
 * stream: the captured calls run again with the same pointers, sizes and
 * configuration, so the caller keeps every captured buffer alive (and its
 * inputs in place) for the graph's lifetime.  gm_graph_destroy frees the
 * graph and its workspace; it waits for the device to finish first.
 * Errors: GM_ERR_ARG (no capture in progress on this thread, a capture
 * already in progress, NULL arguments), GM_ERR_CUDA (capture, instantiation
 * or launch failed -- a library call that failed during capture also
 * invalidates it).  The capture is always ended by gm_graph_end.
 */
typedef struct gm_graph gm_graph;
int gm_graph_begin(void* stream);
int gm_graph_end(void* stream, gm_graph** out);
int gm_graph_launch(const gm_graph* g, void* stream);
int gm_graph_destroy(gm_graph* g);

/*
 * gm_autotune -- picks the EM launch shape for a batch of cells.  The paper
 * has no counterpart (it runs one cell per process on CPUs).
 *
 * Times gm_compress on a sample of the batch (the first 128 x #SM cells,
 * many per CTA) for every candidate shape: threads_per_cell in
 * {64, 128, 256} and shared-tile capacities smem_particles covering the
 * library default and the 90th, 99th, 100th and 50th percentiles of the
 * cell sizes (only those that fit in shared memory; larger cells use the
 * L2-resident global tile; small CTAs with small tiles put more cells on
 * an SM at once, which pays where per-cell serial phases dominate).  Each trial runs a fixed number of sweeps (tol = 0, max_sweeps =
 * sweeps_per_trial, 0 = 24) so that every candidate does the same work,
 * and the fastest of two repetitions counts; the library default (256
 * threads, default tile) is kept unless another candidate is more than 3 %
 * faster.  Writes the winner into
 * cfg->threads_per_cell and cfg->smem_particles and, if timings_ms is not
 * NULL, the trial times (host array of at least GM_TUNE_CANDIDATES floats,
 * -1 for skipped candidates; candidate i has threads_per_cell
 * {64, 128, 256}[i % 3] and tile i / 3).
 * Arguments as gm_compress (device arrays); cell_off is copied to the host,
 * so the call synchronises `stream`.  Results of later gm_compress calls do
 * not depend on the tile; the CTA size changes the order of FP32 partial
 * sums only.  Returns GM_OK or an error code; cfg is unchanged on error.
 */
#define GM_TUNE_CANDIDATES 15
int gm_autotune(gm_config* cfg, int64_t C, int64_t n_particles, const int64_t* cell_off,
                const double* x, const void* v, int32_t v_is_f64, const double* alpha,
                int32_t sweeps_per_trial, float* timings_ms, void* stream);

/*
 * gm_autotune_from -- gm_autotune for fits that start from supplied
 * mixtures (gm_compress_from): the trials run gm_compress_from with the
 * first cells' init_K / init_params (same layout as gm_compress_from, for
 * the whole batch), each trial the fit on the sample with cfg->tol,
 * capped at sweeps_per_trial sweeps (0 = 64).  No counterpart in the
 * paper.  A learned start leaves many cells with one component, whose fit
 * is the prologue's closed form, so the cost balance (and the best launch
 * shape) differs from that of the paper's random start.  Both init
 * pointers are required (GM_ERR_ARG otherwise); other errors and the
 * outputs as gm_autotune.
 */
int gm_autotune_from(gm_config* cfg, int64_t C, int64_t n_particles, const int64_t* cell_off,
                     const double* x, const void* v, int32_t v_is_f64, const double* alpha,
                     const int32_t* init_K, const double* init_params, int32_t sweeps_per_trial,
                     float* timings_ms, void* stream);

/* Description of the last error on this host thread ("" if none); library
 * bookkeeping with no counterpart in the paper. */
const char* gm_last_error(void);

/* Frees the internal workspace (no counterpart in the paper).  The library
 * stays usable; returns GM_OK. */
int gm_shutdown(void);

#ifdef __cplusplus
}
#endif

#endif /* GMCR_GM_H */
