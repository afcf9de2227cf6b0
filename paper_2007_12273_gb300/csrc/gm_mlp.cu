// gm_mlp.cu -- C ABI of the learned-initialisation network: the BF16
// tensor-core GEMM and the network's forward / backward / update steps.
#include <string>

#include "gm_kernels.cuh"

extern "C" {

int gm_gemm_bf16(int32_t M, int32_t N, int32_t K, const void* A, int32_t lda, const void* B,
                 int32_t ldb, const float* bias, int32_t relu, const void* mask, int32_t ldm,
                 float* C_f32, void* C_bf16, int32_t ldc, uint32_t* err, void* stream) {
  gmcr::record_error(GM_OK, "");
  if (M < 0 || N < 0 || K < 0) return gmcr::record_error(GM_ERR_ARG, "negative GEMM size");
  if (M == 0 || N == 0 || K == 0) return GM_OK;
  if (!A || !B || (!C_f32 && !C_bf16)) return gmcr::record_error(GM_ERR_ARG, "a GEMM pointer is NULL");
  if (lda < K || ldb < K || (lda & 7) || (ldb & 7) || ldc < N)
    return gmcr::record_error(GM_ERR_ARG, "GEMM leading dimensions: lda, ldb >= K and multiples of 8; ldc >= N");
  if ((((uintptr_t)A) & 15) || (((uintptr_t)B) & 15))
    return gmcr::record_error(GM_ERR_ARG, "GEMM operands must be 16-byte aligned");
  int dev = 0, major = 0, minor = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (major != 10 || minor != 3)
    return gmcr::record_error(GM_ERR_UNSUPPORTED, "this library is built for sm_103a");
  cudaError_t e = gmcr::launch_tc_gemm(A, B, M, N, K, lda, ldb, bias, relu, mask, ldm, C_f32,
                                       C_bf16, ldc, err, (cudaStream_t)stream);
  if (e != cudaSuccess)
    return gmcr::record_error(GM_ERR_CUDA, (std::string("GEMM launch: ") + cudaGetErrorString(e)).c_str());
  return GM_OK;
}

}  // extern "C"

namespace {

int check_sm103() {
  int dev = 0, major = 0, minor = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (major != 10 || minor != 3)
    return gmcr::record_error(GM_ERR_UNSUPPORTED, "this library is built for sm_103a");
  return GM_OK;
}

int cuda_err(cudaError_t e, const char* what) {
  return gmcr::record_error(GM_ERR_CUDA, (std::string(what) + ": " + cudaGetErrorString(e)).c_str());
}

size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

int check_net(const gm_mlp* net) {
  if (!net) return gmcr::record_error(GM_ERR_ARG, "net is NULL");
  if (net->D != 1 && net->D != 3) return gmcr::record_error(GM_ERR_ARG, "net->D must be 1 or 3");
  const int F = net->D == 1 ? 128 : 576;
  const int SP = 2 + 2 * net->D + net->D * (net->D - 1) / 2;
  if (net->F != F || net->H != 256 || net->O < net->Kmax * SP || (net->O & 15) || net->Kmax < 1 ||
      net->Kmax > gmcr::kMaxK)
    return gmcr::record_error(GM_ERR_ARG, "gm_mlp widths: F = 128 (D=1) / 576 (D=3), H = 256, "
                                          "O >= Kmax * slot size and a multiple of 16");
  for (int l = 0; l < 4; ++l)
    if (!net->W[l] || !net->b[l] || !net->W16[l] || !net->WT16[l])
      return gmcr::record_error(GM_ERR_ARG, "a gm_mlp weight pointer is NULL");
  return GM_OK;
}

// scratch layout for M rows
struct MlpScratch {
  void *H[3], *Ghi, *Glo, *dZhi, *dZlo, *TLhi, *TLlo, *TR;
  float *G32, *dZ32;
};
size_t scratch_layout(const gm_mlp* net, int M, char* base, MlpScratch* sc) {
  const size_t H = net->H, O = net->O, F = net->F;
  const size_t big = (H > O ? (H > F ? H : F) : (O > F ? O : F));
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* p = base ? base + off : nullptr;
    off += al(bytes);
    return p;
  };
  for (int l = 0; l < 3; ++l) sc->H[l] = take((size_t)M * H * 2);
  sc->G32 = (float*)take((size_t)M * O * 4);
  sc->Ghi = take((size_t)M * O * 2);
  sc->Glo = take((size_t)M * O * 2);
  sc->dZ32 = (float*)take((size_t)M * H * 4);
  sc->dZhi = take((size_t)M * H * 2);
  sc->dZlo = take((size_t)M * H * 2);
  sc->TLhi = take(big * (size_t)M * 2);
  sc->TLlo = take(big * (size_t)M * 2);
  sc->TR = take(big * (size_t)M * 2);
  return off;
}

int gemm(const void* A, const void* B, int M, int N, int K, int lda, int ldb, const float* bias,
         int relu, const void* mask, int ldm, float* Cf, void* Cb, int ldc, uint32_t* err,
         cudaStream_t s, int accumulate = 0) {
  cudaError_t e = gmcr::launch_tc_gemm(A, B, M, N, K, lda, ldb, bias, relu, mask, ldm, Cf, Cb, ldc,
                                       err, s, accumulate);
  return e == cudaSuccess ? GM_OK : cuda_err(e, "GEMM launch");
}

// C (FP32) = (Ahi + Alo) B^T: a gradient carried as two BF16 parts keeps
// FP32-level accuracy through the tensor-core products
int gemm_split(const void* Ahi, const void* Alo, const void* B, int M, int N, int K, int lda,
               int ldb, float* Cf, int ldc, uint32_t* err, cudaStream_t s) {
  int rc = gemm(Ahi, B, M, N, K, lda, ldb, nullptr, 0, nullptr, 0, Cf, nullptr, ldc, err, s, 0);
  if (rc) return rc;
  return gemm(Alo, B, M, N, K, lda, ldb, nullptr, 0, nullptr, 0, Cf, nullptr, ldc, err, s, 1);
}

int forward_impl(const gm_mlp* net, int M, const void* X, const MlpScratch& sc, float* out,
                 uint32_t* err, cudaStream_t s) {
  const int F = net->F, H = net->H, O = net->O;
  int rc;
  if ((rc = gemm(X, net->W16[0], M, H, F, F, F, net->b[0], 1, nullptr, 0, nullptr, sc.H[0], H, err, s)))
    return rc;
  if ((rc = gemm(sc.H[0], net->W16[1], M, H, H, H, H, net->b[1], 1, nullptr, 0, nullptr, sc.H[1], H,
                 err, s)))
    return rc;
  if ((rc = gemm(sc.H[1], net->W16[2], M, H, H, H, H, net->b[2], 1, nullptr, 0, nullptr, sc.H[2], H,
                 err, s)))
    return rc;
  return gemm(sc.H[2], net->W16[3], M, O, H, H, H, net->b[3], 0, nullptr, 0, out, nullptr, O, err, s);
}

}  // namespace

extern "C" {

int gm_features(const gm_config* cfg, int64_t C, int64_t n_particles, const int64_t* cell_off,
                const void* v, int32_t v_is_f64, const double* alpha, void* feat, double* wstat,
                void* stream) {
  gmcr::record_error(GM_OK, "");
  if (!cfg || (cfg->D != 1 && cfg->D != 3)) return gmcr::record_error(GM_ERR_ARG, "bad cfg");
  if (C < 0 || n_particles < 0) return gmcr::record_error(GM_ERR_ARG, "negative size");
  if (C == 0) return GM_OK;
  if (!cell_off || !v || !alpha || !feat || !wstat)
    return gmcr::record_error(GM_ERR_ARG, "a required pointer is NULL");
  int rc = check_sm103();
  if (rc) return rc;
  gmcr::trace_mark(nullptr, (cudaStream_t)stream);
  cudaError_t e = gmcr::launch_features(cfg->D, C, n_particles, cell_off, v, v_is_f64, alpha, feat,
                                        wstat, (cudaStream_t)stream);
  gmcr::trace_mark("features_kernel", (cudaStream_t)stream);
  return e == cudaSuccess ? GM_OK : cuda_err(e, "features launch");
}

int gm_mlp_targets(const gm_config* cfg, int64_t C, const int32_t* K, const double* params,
                   const double* wstat, int32_t O, float* T, float* Mk, void* stream) {
  gmcr::record_error(GM_OK, "");
  if (!cfg || (cfg->D != 1 && cfg->D != 3) || cfg->Kmax < 1 || cfg->Kmax > gmcr::kMaxK)
    return gmcr::record_error(GM_ERR_ARG, "bad cfg");
  const int SP = 2 + 2 * cfg->D + cfg->D * (cfg->D - 1) / 2;
  if (O < cfg->Kmax * SP) return gmcr::record_error(GM_ERR_ARG, "O too small");
  if (C == 0) return GM_OK;
  if (!K || !params || !wstat || !T || !Mk)
    return gmcr::record_error(GM_ERR_ARG, "a required pointer is NULL");
  int rc = check_sm103();
  if (rc) return rc;
  cudaError_t e = gmcr::launch_targets(cfg->D, C, cfg->Kmax, O, K, params, wstat, T, Mk,
                                       (cudaStream_t)stream);
  return e == cudaSuccess ? GM_OK : cuda_err(e, "targets launch");
}

int gm_mlp_sync(const gm_mlp* net, void* stream) {
  gmcr::record_error(GM_OK, "");
  int rc = check_net(net);
  if (rc || (rc = check_sm103())) return rc;
  const int rows[4] = {net->H, net->H, net->H, net->O};
  const int cols[4] = {net->F, net->H, net->H, net->H};
  for (int l = 0; l < 4; ++l) {
    cudaError_t e = gmcr::launch_cast_weights(rows[l], cols[l], net->W[l], net->W16[l],
                                              net->WT16[l], (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_err(e, "cast launch");
  }
  return GM_OK;
}

size_t gm_mlp_scratch_bytes(const gm_mlp* net, int32_t M) {
  if (!net || M <= 0) return 0;
  MlpScratch sc;
  return scratch_layout(net, M, nullptr, &sc);
}

int gm_mlp_forward(const gm_mlp* net, int32_t M, const void* X, void* scratch,
                   size_t scratch_bytes, float* out, uint32_t* err, void* stream) {
  gmcr::record_error(GM_OK, "");
  int rc = check_net(net);
  if (rc) return rc;
  if (M < 0) return gmcr::record_error(GM_ERR_ARG, "M < 0");
  if (M == 0) return GM_OK;
  if (!X || !out || !scratch) return gmcr::record_error(GM_ERR_ARG, "a required pointer is NULL");
  if (scratch_bytes < gm_mlp_scratch_bytes(net, M))
    return gmcr::record_error(GM_ERR_ARG, "scratch too small (see gm_mlp_scratch_bytes)");
  if ((rc = check_sm103())) return rc;
  MlpScratch sc;
  scratch_layout(net, M, (char*)scratch, &sc);
  gmcr::trace_mark(nullptr, (cudaStream_t)stream);
  rc = forward_impl(net, M, X, sc, out, err, (cudaStream_t)stream);
  gmcr::trace_mark("mlp_forward (tc_gemm_kernel x4)", (cudaStream_t)stream);
  return rc;
}

int gm_mlp_train_step(const gm_mlp* net, int32_t M, const void* X, const float* T,
                      const float* Mk, float lr, int32_t step, void* scratch,
                      size_t scratch_bytes, float* out, double* loss, uint32_t* err,
                      void* stream) {
  gmcr::record_error(GM_OK, "");
  int rc = check_net(net);
  if (rc) return rc;
  if (M <= 0 || (M % 64)) return gmcr::record_error(GM_ERR_ARG, "M must be a positive multiple of 64");
  if (!X || !T || !Mk || !out || !loss || !scratch)
    return gmcr::record_error(GM_ERR_ARG, "a required pointer is NULL");
  for (int l = 0; l < 4; ++l)
    if (!net->gW[l] || !net->gb[l] || (lr > 0.0f && (!net->mW[l] || !net->vW[l] || !net->mb[l] || !net->vb[l])))
      return gmcr::record_error(GM_ERR_ARG, "a gm_mlp gradient / moment pointer is NULL");
  if (lr > 0.0f && step < 1) return gmcr::record_error(GM_ERR_ARG, "step must be >= 1");
  if (scratch_bytes < gm_mlp_scratch_bytes(net, M))
    return gmcr::record_error(GM_ERR_ARG, "scratch too small (see gm_mlp_scratch_bytes)");
  if ((rc = check_sm103())) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  MlpScratch sc;
  scratch_layout(net, M, (char*)scratch, &sc);
  const int F = net->F, H = net->H, O = net->O;
  if ((rc = forward_impl(net, M, X, sc, out, err, s))) return rc;
  cudaError_t e = gmcr::launch_loss_grad(M, O, net->D, net->Kmax, out, T, Mk, sc.G32, sc.Ghi, loss, s);
  if (e != cudaSuccess) return cuda_err(e, "loss launch");
  // Backward pass.  Each layer's gradient dZ is kept in FP32 and fed to the
  // tensor cores as hi + lo BF16 parts (two products each).
  //   layer 4: gW4 = G^T H3, gb4 = colsum(G), dZ3 = (G W4) * (H3 > 0)
  if ((e = gmcr::launch_split_bf16((int64_t)M * O, O, sc.G32, nullptr, 0, sc.Ghi, sc.Glo, s)) != cudaSuccess)
    return cuda_err(e, "split");
  if ((e = gmcr::launch_colsum(M, O, sc.G32, O, 0, net->gb[3], s)) != cudaSuccess) return cuda_err(e, "colsum");
  if ((e = gmcr::launch_transpose_bf16(M, O, sc.Ghi, O, sc.TLhi, M, s)) != cudaSuccess) return cuda_err(e, "transpose");
  if ((e = gmcr::launch_transpose_bf16(M, O, sc.Glo, O, sc.TLlo, M, s)) != cudaSuccess) return cuda_err(e, "transpose");
  if ((e = gmcr::launch_transpose_bf16(M, H, sc.H[2], H, sc.TR, M, s)) != cudaSuccess) return cuda_err(e, "transpose");
  if ((rc = gemm_split(sc.TLhi, sc.TLlo, sc.TR, O, H, M, M, M, net->gW[3], H, err, s))) return rc;
  if ((rc = gemm_split(sc.Ghi, sc.Glo, net->WT16[3], M, H, O, O, O, sc.dZ32, H, err, s))) return rc;
  if ((e = gmcr::launch_split_bf16((int64_t)M * H, H, sc.dZ32, sc.H[2], H, sc.dZhi, sc.dZlo, s)) != cudaSuccess)
    return cuda_err(e, "split");
  //   layers 3, 2: gW = dZ^T H_prev, gb = colsum(dZ), dZ_prev = (dZ W) * (H_prev > 0)
  for (int l = 2; l >= 1; --l) {
    if ((e = gmcr::launch_colsum(M, H, sc.dZ32, H, 0, net->gb[l], s)) != cudaSuccess) return cuda_err(e, "colsum");
    if ((e = gmcr::launch_transpose_bf16(M, H, sc.dZhi, H, sc.TLhi, M, s)) != cudaSuccess) return cuda_err(e, "transpose");
    if ((e = gmcr::launch_transpose_bf16(M, H, sc.dZlo, H, sc.TLlo, M, s)) != cudaSuccess) return cuda_err(e, "transpose");
    if ((e = gmcr::launch_transpose_bf16(M, H, sc.H[l - 1], H, sc.TR, M, s)) != cudaSuccess) return cuda_err(e, "transpose");
    if ((rc = gemm_split(sc.TLhi, sc.TLlo, sc.TR, H, H, M, M, M, net->gW[l], H, err, s))) return rc;
    if ((rc = gemm_split(sc.dZhi, sc.dZlo, net->WT16[l], M, H, H, H, H, sc.dZ32, H, err, s))) return rc;
    if ((e = gmcr::launch_split_bf16((int64_t)M * H, H, sc.dZ32, sc.H[l - 1], H, sc.dZhi, sc.dZlo, s)) != cudaSuccess)
      return cuda_err(e, "split");
  }
  //   layer 1: gW1 = dZ1^T X, gb1 = colsum(dZ1)
  if ((e = gmcr::launch_colsum(M, H, sc.dZ32, H, 0, net->gb[0], s)) != cudaSuccess) return cuda_err(e, "colsum");
  if ((e = gmcr::launch_transpose_bf16(M, H, sc.dZhi, H, sc.TLhi, M, s)) != cudaSuccess) return cuda_err(e, "transpose");
  if ((e = gmcr::launch_transpose_bf16(M, H, sc.dZlo, H, sc.TLlo, M, s)) != cudaSuccess) return cuda_err(e, "transpose");
  if ((e = gmcr::launch_transpose_bf16(M, F, X, F, sc.TR, M, s)) != cudaSuccess) return cuda_err(e, "transpose");
  if ((rc = gemm_split(sc.TLhi, sc.TLlo, sc.TR, H, F, M, M, M, net->gW[0], F, err, s))) return rc;
  if (lr > 0.0f) {
    const int rows[4] = {H, H, H, O};
    const int cols[4] = {F, H, H, H};
    for (int l = 0; l < 4; ++l) {
      if ((e = gmcr::launch_adam(rows[l], cols[l], net->W[l], net->gW[l], net->mW[l], net->vW[l], lr,
                                 step, net->W16[l], net->WT16[l], s)) != cudaSuccess)
        return cuda_err(e, "adam");
      if ((e = gmcr::launch_adam(rows[l], 1, net->b[l], net->gb[l], net->mb[l], net->vb[l], lr, step,
                                 nullptr, nullptr, s)) != cudaSuccess)
        return cuda_err(e, "adam");
    }
  }
  return GM_OK;
}

int gm_mlp_decode(const gm_config* cfg, int64_t C, const float* out, int32_t O,
                  const double* wstat, const int64_t* cell_off, float presence_logit, int32_t* K0,
                  double* init_params, void* stream) {
  gmcr::record_error(GM_OK, "");
  if (!cfg || (cfg->D != 1 && cfg->D != 3) || cfg->Kmax < 1 || cfg->Kmax > gmcr::kMaxK)
    return gmcr::record_error(GM_ERR_ARG, "bad cfg");
  const int SP = 2 + 2 * cfg->D + cfg->D * (cfg->D - 1) / 2;
  if (O < cfg->Kmax * SP) return gmcr::record_error(GM_ERR_ARG, "O too small");
  if (C == 0) return GM_OK;
  if (!out || !wstat || !cell_off || !K0 || !init_params)
    return gmcr::record_error(GM_ERR_ARG, "a required pointer is NULL");
  int rc = check_sm103();
  if (rc) return rc;
  if (!(presence_logit == presence_logit)) return gmcr::record_error(GM_ERR_ARG, "presence_logit is NaN");
  gmcr::trace_mark(nullptr, (cudaStream_t)stream);
  cudaError_t e = gmcr::launch_decode(cfg->D, C, cfg->Kmax, O, out, wstat, cell_off, presence_logit,
                                      K0, init_params, (cudaStream_t)stream);
  gmcr::trace_mark("decode_kernel", (cudaStream_t)stream);
  return e == cudaSuccess ? GM_OK : cuda_err(e, "decode launch");
}

}  // extern "C"
