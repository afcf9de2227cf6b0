// gm_kernels.cuh -- launchers shared between the translation units of the
// library (kernels live in gm_em*.cu, gm_moments.cu, gm_reconstruct.cu).
#pragma once

#include "gm_common.cuh"
#include "em_kernel.cuh"
#include "em_k1.cuh"

namespace gmcr {

// EM (compression); returns the launch error
cudaError_t launch_em1(const EmParams& p, int nt, int fp64_mstep, int v_f64, size_t smem, int grid,
                       cudaStream_t s);
size_t em_k1_raw_bytes(int D, int64_t C);
cudaError_t launch_em_k1(int D, int v_f64, const K1Params& p, int sms, cudaStream_t s);
cudaError_t launch_em3(const EmParams& p, int nt, int fp64_mstep, int v_f64, size_t smem, int grid,
                       cudaStream_t s);
// CTAs of an EM kernel that fit on one SM with `smem` dynamic bytes
int em_blocks_per_sm(int D, int nt, int fp64_mstep, int v_f64, size_t smem);

size_t deposit_ws_bytes(int64_t C);
// rho from records that em_k1_kernel wrote (the deposit fused with the
// closed-form pre-pass)
cudaError_t launch_deposit_combine(int64_t C, double dx, double q, int order, const void* ws,
                                   double* rho, cudaStream_t s);
cudaError_t launch_deposit(int64_t C, const int64_t* cell_off, const double* x,
                           const double* alpha, double dx, double q, int order, void* ws,
                           double* rho, cudaStream_t s);
cudaError_t launch_moments(int D, int64_t C, int64_t n, const int64_t* cell_off, const void* v,
                           int v_f64, const double* alpha, double* W, double* p, double* M2,
                           double* E, cudaStream_t s);
cudaError_t launch_mixture_moments(int D, int64_t C, int Kmax, const int32_t* K, const double* prm,
                                   const double* Wc, double* W, double* p, double* M2, double* E,
                                   cudaStream_t s);

int solve_blocks(int64_t C);

// standard EM (gm_compress_standard); the parameter block is declared in
// std_kernel.cuh
struct StdParams;
cudaError_t launch_std(int D, const StdParams& p, int v_f64, size_t smem, int sms, cudaStream_t s);
cudaError_t launch_aa_affine(int n, const double* A, const double* b, const double* x0, int m,
                             int iters, double* x_out, double* res_out, cudaStream_t s);
// sets the calling thread's gm_last_error() text; returns code
int record_error(int code, const char* msg);
// the C ABI's own argument and device checks (gm_api.cu), shared by the
// entry points defined in other translation units
int api_check_reconstruct(const gm_config* cfg, int64_t C, const int32_t* K, const double* params,
                          const double* W, const double* rho_target, int64_t n_out,
                          const int64_t* out_off, const double* x_out, const double* v_out,
                          const double* alpha_out, const uint32_t* status_out);
int api_check_device();
// per-kernel device times (gm_trace.cu): an event after each traced kernel
// on its stream (name = the kernel), or a boundary (name = nullptr) at the
// start of an API call; a no-op unless a trace is on
void trace_mark(const char* name, cudaStream_t s);
size_t reconstruct_ws_bytes(int D, int64_t C, int Kmax);
cudaError_t launch_reconstruct(int D, int64_t C, int Kmax, const int32_t* K, const double* prm,
                               const double* W, const double* rho_target, int64_t n_out,
                               const int64_t* out_off, uint64_t seed, double dx, double q,
                               int order, double* x_out, double* v_out, double* alpha_out,
                               uint32_t* status_out, double* dA_user, void* ws, cudaStream_t s);

// the 2D periodic mesh (gm_mesh2d.cu)
constexpr int kMesh2dMaxIter = 64;    // defect-correction iterations, at most
constexpr double kMesh2dTol = 1e-14;  // max |residual| / max |dx dy rho'| to stop
cudaError_t launch_deposit2d(int64_t Cx, int64_t Cy, const int64_t* cell_off, const double* x,
                             const double* y, const double* alpha, double dx, double dy, double q,
                             int order, double* part, double* rho, cudaStream_t s);
size_t reconstruct2d_ws_bytes(int D, int64_t Cx, int64_t Cy);
cudaError_t launch_reconstruct2d(int D, int64_t Cx, int64_t Cy, int Kmax, const int32_t* K,
                                 const double* prm, const double* W, const double* rho_target,
                                 int64_t n_out, const int64_t* out_off, uint64_t seed, double dx,
                                 double dy, double q, int order, double* x_out, double* y_out,
                                 double* v_out, double* alpha_out, uint32_t* status_out,
                                 double* dA_user, void* ws, cudaStream_t s);

// BF16 tcgen05 GEMM: C = A B^T (+bias, ReLU, mask), see tc_gemm.cu
size_t tc_gemm_smem(int bn);
cudaError_t launch_tc_gemm(const void* A, const void* B, int M, int N, int K, int lda, int ldb,
                           const float* bias, int relu, const void* mask, int ldm, float* Cf,
                           void* Cb, int ldc, unsigned int* err, cudaStream_t s,
                           int accumulate = 0);

}  // namespace gmcr

namespace gmcr {
// learned-initialisation network helpers (mlp_kernels.cu)
cudaError_t launch_features(int D, int64_t C, int64_t n, const int64_t* cell_off, const void* v,
                            int v_f64, const double* alpha, void* feat, double* wstat,
                            cudaStream_t s);
cudaError_t launch_targets(int D, int64_t C, int Kmax, int O, const int32_t* K, const double* prm,
                           const double* wstat, float* T, float* Mk, cudaStream_t s);
cudaError_t launch_decode(int D, int64_t C, int Kmax, int O, const float* out, const double* wstat,
                          const int64_t* cell_off, float presence_logit, int32_t* K0, double* prm,
                          cudaStream_t s);
cudaError_t launch_loss_grad(int B, int O, int D, int Kmax, const float* out, const float* T,
                             const float* Mk, float* G32, void* G16, double* loss, cudaStream_t s);
cudaError_t launch_transpose_bf16(int R, int Cc, const void* in, int ldi, void* out, int ldo,
                                  cudaStream_t s);
cudaError_t launch_colsum(int R, int Cc, const void* G, int ld, int g_is_bf16, float* db,
                          cudaStream_t s);
cudaError_t launch_adam(int n_out, int n_in, float* w, const float* g, float* m, float* v, float lr,
                        int step, void* w16, void* wt16, cudaStream_t s);
cudaError_t launch_cast_weights(int n_out, int n_in, const float* w, void* w16, void* wt16,
                                cudaStream_t s);
cudaError_t launch_split_bf16(int64_t total, int cols, float* x, const void* mask, int ldm,
                              void* hi, void* lo, cudaStream_t s);
}  // namespace gmcr
