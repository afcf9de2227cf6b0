// mlp_kernels.cu -- the learned-initialisation network around the tcgen05
// GEMM: per-cell features, training targets, loss gradient, transposes,
// bias gradients, Adam, and the decoding of the network's output into an
// initial mixture for EM.  (Not part of the paper, whose EM starts from
// randomly chosen particles; the EM that follows is the paper's.)
//
// Interface (identical to the oracle's definition, written independently):
//   features: alpha-weighted whitened moments + histogram, widths 128 (1V)
//   and 576 (3V); output slots [presence, log w, mu (D), log diag L (D),
//   L10, L20, L21] in whitened coordinates; targets sorted by mu_0.
#include <cuda_bf16.h>

#include "gm_kernels.cuh"

namespace gmcr {

namespace {

__host__ __device__ constexpr int mlp_F(int D) { return D == 1 ? 128 : 576; }
__host__ __device__ constexpr int mlp_SP(int D) { return 2 + 2 * D + D * (D - 1) / 2; }

}  // namespace

// ---------------------------------------------------------------------------
// features: one warp per cell (NW cells per CTA), two passes over the cell's
// particles, both FP32.  The first sums W, the first and the diagonal second
// moments about the cell's first particle (a shift inside the cell's spread,
// so that the variance keeps FP32's relative accuracy); the second whitens
// with the resulting mean and standard deviation and accumulates the higher
// moments and the histogram.  The features are stored in BF16 and the
// whitening only maps the network's start back to the cell, so FP32 is
// ample -- and GB300 runs FP64 at 1/64 of the FP32 rate.
// ---------------------------------------------------------------------------
template <int D, typename VT, int NW>
__global__ void __launch_bounds__(NW * 32) features_kernel(int64_t C, int64_t n, const int64_t* cell_off,
                                                           const VT* v, const double* alpha,
                                                           __nv_bfloat16* feat, double* wstat) {
  constexpr int F = mlp_F(D);
  constexpr int NB = D == 1 ? 64 : 512;
  constexpr int NMOM = D == 1 ? 3 : 10;
  constexpr int NC = D == 1 ? 2 : 9;  // higher moments accumulated
  // the histogram in fixed point (units of 2^-30 of the cell's weight):
  // integer shared-memory atomics add in any order to the same sum, so the
  // features -- and a network trained on them -- are deterministic
  __shared__ unsigned int hists[NW][NB];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned int* hist = hists[wid];
  for (int64_t j = (int64_t)blockIdx.x * NW + wid; j < C; j += (int64_t)gridDim.x * NW) {
    const int64_t o = cell_off[j];
    const int N = (int)(cell_off[j + 1] - o);
    for (int b = lane; b < NB; b += 32) hist[b] = 0u;
    // W, and the first and diagonal second moments about the first particle
    float sh[D];
#pragma unroll
    for (int d = 0; d < D; ++d) sh[d] = N > 0 ? (float)v[(int64_t)d * n + o] : 0.0f;
    float W = 0.0f, s1[D], s2[D];
#pragma unroll
    for (int d = 0; d < D; ++d) s1[d] = s2[d] = 0.0f;
#pragma unroll 4
    for (int p = lane; p < N; p += 32) {
      const float a = d2f_trunc(alpha[o + p]);
      W += a;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const float dv = (float)v[(int64_t)d * n + o + p] - sh[d];
        const float ad = a * dv;
        s1[d] += ad;
        s2[d] = fmaf(ad, dv, s2[d]);
      }
    }
    W = warp_sum(W);
    // mean = sh + m1 (FP64, the shift kept exact) and sd = sqrt(var) are
    // stored; the FP32 pass below uses mf = fl32(sh + m1), the FP32 sum
    // (the same value as the FP64 sum rounded to FP32), and 1 / sd
    float mf[D], sdf[D];
    bool ok = W > 0.0f;
    const float iW0 = ok ? 1.0f / W : 0.0f;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const float m1 = warp_sum(s1[d]) * iW0;
      const float var = fmaxf(warp_sum(s2[d]) * iW0 - m1 * m1, 0.0f);
      mf[d] = __fadd_rn(sh[d], m1);  // no contraction with the product m1
      sdf[d] = ok ? sqrtf(var) : 0.0f;
      ok = ok && sdf[d] > 0.0f;
      if (lane == d) {  // one FP64 addition per dimension, on lane d
        wstat[j * 2 * D + d] = f2d_exact(sh[d]) + f2d_exact(m1);
        wstat[j * 2 * D + D + d] = f2d_exact(sdf[d]);
      }
    }
    __nv_bfloat16* fj = feat + (size_t)j * F;
    if (!ok) {
      for (int i = lane; i < F; i += 32) fj[i] = __float2bfloat16(0.0f);
      __syncwarp();
      continue;
    }
    __syncwarp();  // histogram zeroed
    // higher moments and the histogram (FP32)
    float isf[D];
#pragma unroll
    for (int d = 0; d < D; ++d) isf[d] = 1.0f / sdf[d];
    const float iW = iW0;
    float s3[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) s3[i] = 0.0f;
#pragma unroll 4
    for (int p = lane; p < N; p += 32) {
      const float w = d2f_trunc(alpha[o + p]) * iW;
      float y[D];
#pragma unroll
      for (int d = 0; d < D; ++d) y[d] = ((float)v[(int64_t)d * n + o + p] - mf[d]) * isf[d];
      if (D == 1) {
        const float wy2 = w * y[0] * y[0];
        s3[0] = fmaf(wy2, y[0], s3[0]);
        s3[1] = fmaf(wy2, y[0] * y[0], s3[1]);
        int b = (int)floorf((y[0] + 4.0f) * 8.0f);
        b = b < 0 ? 0 : (b > 63 ? 63 : b);
        atomicAdd(&hist[b], __float2uint_rn(w * 1073741824.0f));
      } else {
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const float wy2 = w * y[d] * y[d];
          s3[d] = fmaf(wy2, y[d], s3[d]);
          s3[3 + d] = fmaf(wy2, y[d] * y[d], s3[3 + d]);
        }
        s3[6] = fmaf(w * y[0], y[1], s3[6]);
        s3[7] = fmaf(w * y[0], y[2], s3[7]);
        s3[8] = fmaf(w * y[1], y[2], s3[8]);
        int b[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          b[d] = (int)floorf((y[d] + 2.5f) * 1.6f);
          b[d] = b[d] < 0 ? 0 : (b[d] > 7 ? 7 : b[d]);
        }
        atomicAdd(&hist[b[0] * 64 + b[1] * 8 + b[2]], __float2uint_rn(w * 1073741824.0f));
      }
    }
#pragma unroll
    for (int i = 0; i < NC; ++i) s3[i] = warp_sum(s3[i]);
    __syncwarp();  // histogram complete
    // assemble
    for (int i = lane; i < F; i += 32) {
      float val = 0.0f;
      if (i < NMOM) {
        if (D == 1) {
          val = i == 0 ? s3[0] : (i == 1 ? s3[1] - 3.0f : logf((float)N) * 0.1f);
        } else {
          if (i < 3) val = s3[i];
          else if (i < 6) val = s3[i] - 3.0f;
          else if (i < 9) val = s3[i];
          else val = logf((float)N) * 0.1f;
        }
      } else if (i < NMOM + NB) {
        val = (float)hist[i - NMOM] * (9.3132257461547852e-10f /* 2^-30 */ * (float)NB);
      }
      fj[i] = __float2bfloat16(val);
    }
    __syncwarp();  // before the next cell clears the histogram
  }
}

// ---------------------------------------------------------------------------
// training targets of one cell (one thread per cell)
// ---------------------------------------------------------------------------
template <int D>
__global__ void targets_kernel(int64_t C, int Kmax, int O, const int32_t* K, const double* prm,
                               const double* wstat, float* T, float* Mk) {
  constexpr int NM = D * (D + 1) / 2;
  constexpr int P = 1 + D + NM;
  constexpr int SP = mlp_SP(D);
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < C;
       j += (int64_t)gridDim.x * blockDim.x) {
    float* t = T + (size_t)j * O;
    float* m = Mk + (size_t)j * O;
    for (int i = 0; i < O; ++i) { t[i] = 0.0f; m[i] = 0.0f; }
    const double* mean = wstat + j * 2 * D;
    const double* sd = mean + D;
    const int Kj = K[j] < Kmax ? K[j] : Kmax;
    // sort components by whitened mu_0 (insertion sort)
    int ord[kMaxK];
    double key[kMaxK];
    for (int k = 0; k < Kj; ++k) {
      const double* r = prm + ((size_t)j * Kmax + k) * P;
      key[k] = (r[1] - mean[0]) / sd[0];
      ord[k] = k;
      for (int q = k; q > 0 && key[q] < key[q - 1]; --q) {
        const double tk = key[q]; key[q] = key[q - 1]; key[q - 1] = tk;
        const int to = ord[q]; ord[q] = ord[q - 1]; ord[q - 1] = to;
      }
    }
    for (int s = 0; s < Kmax; ++s) {
      const int base = s * SP;
      m[base] = 1.0f;
      if (s >= Kj || !(sd[0] > 0.0)) continue;
      const double* r = prm + ((size_t)j * Kmax + ord[s]) * P;
      double Sw[3][3];
      int q = 1 + D;
      for (int a = 0; a < D; ++a)
        for (int b = a; b < D; ++b, ++q) Sw[a][b] = Sw[b][a] = r[q] / (sd[a] * sd[b]);
      double L[3][3] = {{0}};
      bool pd = true;
      for (int a = 0; a < D && pd; ++a)
        for (int b = 0; b <= a && pd; ++b) {
          double x = Sw[a][b];
          for (int e = 0; e < b; ++e) x -= L[a][e] * L[b][e];
          if (a == b) {
            if (!(x > 0.0)) pd = false;
            else L[a][a] = sqrt(x);
          } else {
            L[a][b] = x / L[b][b];
          }
        }
      if (!pd || !(r[0] > 0.0)) continue;
      t[base] = 1.0f;
      t[base + 1] = (float)log(r[0]);
      for (int d = 0; d < D; ++d) t[base + 2 + d] = (float)((r[1 + d] - mean[d]) / sd[d]);
      for (int d = 0; d < D; ++d) t[base + 2 + D + d] = (float)log(L[d][d]);
      if (D == 3) {
        t[base + 8] = (float)L[1][0];
        t[base + 9] = (float)L[2][0];
        t[base + 10] = (float)L[2][1];
      }
      for (int i = 1; i < SP; ++i) m[base + i] = 1.0f;
    }
  }
}

// ---------------------------------------------------------------------------
// loss and d loss / d out (mean over the batch of B rows)
// ---------------------------------------------------------------------------
__global__ void loss_grad_kernel(int B, int O, int SP, int nslot, const float* out, const float* T,
                                 const float* Mk, float* G32, __nv_bfloat16* G16, double* loss) {
  __shared__ double red[8];
  double acc = 0.0;
  const float inv = 1.0f / (float)B;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)B * O;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int col = (int)(i % O);
    const float p = out[i], t = T[i];
    float g = 0.0f;
    if (col < nslot * SP && col % SP == 0) {  // presence logit: BCE
      const float sp = p > 0.0f ? p + log1pf(expf(-p)) : log1pf(expf(p));
      acc += (double)(sp - t * p);
      g = 1.0f / (1.0f + expf(-p)) - t;
    } else if (Mk[i] > 0.0f) {
      const float d = p - t;
      acc += (double)d * d;
      g = 2.0f * d;
    }
    g *= inv;
    G32[i] = g;
    G16[i] = __float2bfloat16(g);
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    atomicAdd(loss, s / (double)B);
  }
}

// out[c][r] = in[r][c] (BF16), 32 x 32 tiles
__global__ void transpose_bf16_kernel(int R, int Cc, const __nv_bfloat16* in, int ldi,
                                      __nv_bfloat16* out, int ldo) {
  __shared__ __nv_bfloat16 tile[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < R && c < Cc) ? in[(size_t)r * ldi + c] : __float2bfloat16(0.0f);
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (c < Cc && r < R) out[(size_t)c * ldo + r] = tile[threadIdx.x][i];
  }
}

// db[c] = sum_r G[r][c] (FP32 or BF16 input)
template <typename TG>
__global__ void colsum_kernel(int R, int Cc, const TG* G, int ld, float* db) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < Cc; c += gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int r = 0; r < R; ++r) s += (float)G[(size_t)r * ld + c];
    db[c] = s;
  }
}

// Adam on one tensor [n_out][n_in] (n_in = 1 for a bias); refreshes the BF16
// copy and its transpose when given
__global__ void adam_kernel(int n_out, int n_in, float* w, const float* g, float* m, float* v,
                            float lr, float b1, float b2, float eps, float c1, float c2,
                            __nv_bfloat16* w16, __nv_bfloat16* wt16) {
  const int64_t total = (int64_t)n_out * n_in;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (w16) w16[i] = __float2bfloat16(wi);
    if (wt16) {
      const int64_t r = i / n_in, c = i % n_in;
      wt16[c * n_out + r] = __float2bfloat16(wi);
    }
  }
}

// x (FP32, zeroed where mask <= 0 if a mask is given) as hi + lo BF16
// parts: hi = bf16(x), lo = bf16(x - hi)
__global__ void split_bf16_kernel(int64_t total, int cols, float* x, const __nv_bfloat16* mask,
                                  int ldm, __nv_bfloat16* hi, __nv_bfloat16* lo) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    float v = x[i];
    if (mask && !(__bfloat162float(mask[(i / cols) * ldm + i % cols]) > 0.0f)) {
      v = 0.0f;
      x[i] = 0.0f;
    }
    const __nv_bfloat16 h = __float2bfloat16(v);
    hi[i] = h;
    lo[i] = __float2bfloat16(v - __bfloat162float(h));
  }
}

// BF16 copy and transpose of FP32 weights
__global__ void cast_weights_kernel(int n_out, int n_in, const float* w, __nv_bfloat16* w16,
                                    __nv_bfloat16* wt16) {
  const int64_t total = (int64_t)n_out * n_in;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const __nv_bfloat16 b = __float2bfloat16(w[i]);
    w16[i] = b;
    if (wt16) wt16[(i % n_in) * n_out + i / n_in] = b;
  }
}

// ---------------------------------------------------------------------------
// decode the network's output of a cell into an initial mixture (original
// coordinates): present slots (positive presence logit, at least the most
// likely one), capped so that N - T K0 / 2 > 0 by dropping the smallest
// weights; weights by softmax of the log weights; Sigma = L L^T
// ---------------------------------------------------------------------------
template <int D>
__global__ void decode_kernel(int64_t C, int Kmax, int O, const float* out, const double* wstat,
                              const int64_t* cell_off, float presence_logit, int32_t* K0,
                              double* prm) {
  constexpr int NM = D * (D + 1) / 2;
  constexpr int P = 1 + D + NM;
  constexpr int SP = mlp_SP(D);
  const double halfT = 0.5 * (D * (D + 3) / 2);
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < C;
       j += (int64_t)gridDim.x * blockDim.x) {
    const float* o = out + (size_t)j * O;
    const double* mean = wstat + j * 2 * D;
    const double* sd = mean + D;
    const int64_t N = cell_off[j + 1] - cell_off[j];
    double* r = prm + (size_t)j * Kmax * P;
    for (int i = 0; i < Kmax * P; ++i) r[i] = 0.0;
    int sel[kMaxK], ns = 0, best = 0;
    for (int s = 0; s < Kmax; ++s) {
      if (o[s * SP] > o[best * SP]) best = s;
      if (o[s * SP] > presence_logit) sel[ns++] = s;
    }
    if (ns == 0) sel[ns++] = best;
    while (ns > 1 && (double)N - halfT * ns <= 0.0) {
      int dmin = 0;
      for (int i = 1; i < ns; ++i)
        if (o[sel[i] * SP + 1] < o[sel[dmin] * SP + 1]) dmin = i;
      for (int i = dmin; i < ns - 1; ++i) sel[i] = sel[i + 1];
      --ns;
    }
    if (N == 0 || !(sd[0] > 0.0)) {
      K0[j] = 0;
      continue;
    }
    double lmax = -1e300;
    for (int i = 0; i < ns; ++i) lmax = fmax(lmax, (double)o[sel[i] * SP + 1]);
    double wsum = 0.0, w[kMaxK];
    for (int i = 0; i < ns; ++i) {
      w[i] = exp((double)o[sel[i] * SP + 1] - lmax);
      wsum += w[i];
    }
    for (int i = 0; i < ns; ++i) {
      const float* so = o + sel[i] * SP;
      double L[3][3] = {{0}};
      for (int d = 0; d < D; ++d) {
        double ld = (double)so[2 + D + d];
        ld = ld < -10.0 ? -10.0 : (ld > 5.0 ? 5.0 : ld);
        L[d][d] = exp(ld);
      }
      if (D == 3) {
        L[1][0] = so[8];
        L[2][0] = so[9];
        L[2][1] = so[10];
      }
      double* ri = r + i * P;
      ri[0] = w[i] / wsum;
      for (int d = 0; d < D; ++d) ri[1 + d] = mean[d] + sd[d] * (double)so[2 + d];
      int q = 1 + D;
      for (int a = 0; a < D; ++a)
        for (int b = a; b < D; ++b, ++q) {
          double s = 0.0;
          for (int e = 0; e <= b; ++e) s += L[a][e] * L[b][e];
          ri[q] = s * sd[a] * sd[b];
        }
    }
    K0[j] = ns;
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_features(int D, int64_t C, int64_t n, const int64_t* cell_off, const void* v,
                            int v_f64, const double* alpha, void* feat, double* wstat,
                            cudaStream_t s) {
  if (C == 0) return cudaSuccess;
  constexpr int NW = 4;
  const int64_t ncta = (C + NW - 1) / NW;
  const int g = (int)(ncta < 152 * 16 ? ncta : 152 * 16);
  __nv_bfloat16* f = (__nv_bfloat16*)feat;
  if (D == 1) {
    if (v_f64) features_kernel<1, double, NW><<<g, NW * 32, 0, s>>>(C, n, cell_off, (const double*)v, alpha, f, wstat);
    else features_kernel<1, float, NW><<<g, NW * 32, 0, s>>>(C, n, cell_off, (const float*)v, alpha, f, wstat);
  } else {
    if (v_f64) features_kernel<3, double, NW><<<g, NW * 32, 0, s>>>(C, n, cell_off, (const double*)v, alpha, f, wstat);
    else features_kernel<3, float, NW><<<g, NW * 32, 0, s>>>(C, n, cell_off, (const float*)v, alpha, f, wstat);
  }
  return cudaGetLastError();
}

cudaError_t launch_targets(int D, int64_t C, int Kmax, int O, const int32_t* K, const double* prm,
                           const double* wstat, float* T, float* Mk, cudaStream_t s) {
  if (C == 0) return cudaSuccess;
  const int g = (int)((C + 127) / 128 < 4096 ? (C + 127) / 128 : 4096);
  if (D == 1) targets_kernel<1><<<g, 128, 0, s>>>(C, Kmax, O, K, prm, wstat, T, Mk);
  else targets_kernel<3><<<g, 128, 0, s>>>(C, Kmax, O, K, prm, wstat, T, Mk);
  return cudaGetLastError();
}

cudaError_t launch_decode(int D, int64_t C, int Kmax, int O, const float* out, const double* wstat,
                          const int64_t* cell_off, float presence_logit, int32_t* K0, double* prm,
                          cudaStream_t s) {
  if (C == 0) return cudaSuccess;
  const int g = (int)((C + 127) / 128 < 4096 ? (C + 127) / 128 : 4096);
  if (D == 1) decode_kernel<1><<<g, 128, 0, s>>>(C, Kmax, O, out, wstat, cell_off, presence_logit, K0, prm);
  else decode_kernel<3><<<g, 128, 0, s>>>(C, Kmax, O, out, wstat, cell_off, presence_logit, K0, prm);
  return cudaGetLastError();
}

cudaError_t launch_loss_grad(int B, int O, int D, int Kmax, const float* out, const float* T,
                             const float* Mk, float* G32, void* G16, double* loss,
                             cudaStream_t s) {
  const int64_t total = (int64_t)B * O;
  const int g = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  loss_grad_kernel<<<g, 256, 0, s>>>(B, O, mlp_SP(D), Kmax, out, T, Mk, G32,
                                     (__nv_bfloat16*)G16, loss);
  return cudaGetLastError();
}

cudaError_t launch_transpose_bf16(int R, int Cc, const void* in, int ldi, void* out, int ldo,
                                  cudaStream_t s) {
  dim3 grid((Cc + 31) / 32, (R + 31) / 32), block(32, 8);
  transpose_bf16_kernel<<<grid, block, 0, s>>>(R, Cc, (const __nv_bfloat16*)in, ldi,
                                               (__nv_bfloat16*)out, ldo);
  return cudaGetLastError();
}

cudaError_t launch_colsum(int R, int Cc, const void* G, int ld, int g_is_bf16, float* db,
                          cudaStream_t s) {
  const int g = (Cc + 127) / 128;
  if (g_is_bf16)
    colsum_kernel<__nv_bfloat16><<<g, 128, 0, s>>>(R, Cc, (const __nv_bfloat16*)G, ld, db);
  else
    colsum_kernel<float><<<g, 128, 0, s>>>(R, Cc, (const float*)G, ld, db);
  return cudaGetLastError();
}

cudaError_t launch_adam(int n_out, int n_in, float* w, const float* g, float* m, float* v, float lr,
                        int step, void* w16, void* wt16, cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  const int64_t total = (int64_t)n_out * n_in;
  const int nb = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  adam_kernel<<<nb, 256, 0, s>>>(n_out, n_in, w, g, m, v, lr, b1, b2, 1e-8f, c1, c2,
                                (__nv_bfloat16*)w16, (__nv_bfloat16*)wt16);
  return cudaGetLastError();
}

cudaError_t launch_cast_weights(int n_out, int n_in, const float* w, void* w16, void* wt16,
                                cudaStream_t s) {
  const int64_t total = (int64_t)n_out * n_in;
  const int g = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  cast_weights_kernel<<<g, 256, 0, s>>>(n_out, n_in, w, (__nv_bfloat16*)w16, (__nv_bfloat16*)wt16);
  return cudaGetLastError();
}

cudaError_t launch_split_bf16(int64_t total, int cols, float* x, const void* mask, int ldm,
                              void* hi, void* lo, cudaStream_t s) {
  const int g = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  split_bf16_kernel<<<g, 256, 0, s>>>(total, cols, x, (const __nv_bfloat16*)mask, ldm,
                                      (__nv_bfloat16*)hi, (__nv_bfloat16*)lo);
  return cudaGetLastError();
}

}  // namespace gmcr
