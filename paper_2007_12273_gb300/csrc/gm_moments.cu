// gm_moments.cu -- charge deposition (Sec. 2.4.1) and per-cell moments.
#include "gm_kernels.cuh"

namespace gmcr {

// Block-wide FP64 sum of NV values held per thread; result valid in thread 0.
template <int NT, int NV>
__device__ __forceinline__ void block_sum_to0(double (&v)[NV], double (*red)[NV]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) red[w][i] = v[i];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int q = 1; q < NT / 32; ++q)
#pragma unroll
      for (int i = 0; i < NV; ++i) v[i] += red[q][i];
}

// Per-cell partial deposits: part[j] = sum_{p in j} alpha_p S(x_i - x_p)
// for i = j-1, j, j+1 (alpha = NULL means unit weights).  One warp per
// cell.  With s = xi - 1/2 (xi the position inside the cell) the quadratic
// B-spline weights are (1/2 - s)^2 / 2, 3/4 - s^2, (1/2 + s)^2 / 2, so the
// three sums follow from A0 = sum alpha, A1 = sum alpha s, A2 = sum alpha
// s^2; for CIC they are sum alpha max(-s, 0), A0 - (the other two),
// sum alpha max(s, 0).
template <int NW>
__global__ void __launch_bounds__(NW * 32) deposit_partials_kernel(int64_t C, const int64_t* cell_off,
                                                                   const double* x, const double* alpha,
                                                                   double inv_dx, int order,
                                                                   double* part /*[C][3]*/) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t j = (int64_t)blockIdx.x * NW + wid; j < C; j += (int64_t)gridDim.x * NW) {
    const int64_t o = cell_off[j], n = cell_off[j + 1] - o;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    // equal weights (bit for bit) and at most 2^14 particles: the sums of s
    // and s^2 (or of the CIC parts) exactly on the integer pipe, s = k 2^-53
    // with k = round(xi 2^53) - 2^52 from the bits of the FP64 in-cell
    // position xi in [0, 1); the weight multiplies the sums once
    bool fixed = false;
    if (n > 0 && n <= kFixMaxN) {
      const long long wb = alpha ? __double_as_longlong(alpha[o]) : __double_as_longlong(1.0);
      bool same = true;
      if (alpha)
        for (int64_t p = lane; p < n; p += 32) same = same && (__double_as_longlong(alpha[o + p]) == wb);
      fixed = __all_sync(0xffffffffu, same);
      if (fixed) {
        __int128 k0 = 0, k1 = 0;
        for (int64_t p = lane; p < n; p += 32) {
          const double xi = cell_frac(x[o + p], j, inv_dx);
          // xi = m 2^(e - 1075) (m with its implicit bit), k = round(xi 2^53) - 2^52
          const unsigned long long u = (unsigned long long)__double_as_longlong(xi);
          const int e = (int)((u >> 52) & 0x7FFull);
          const long long m = (long long)((u & ((1ull << 52) - 1ull)) | (e ? (1ull << 52) : 0ull));
          const int sh = (e ? e : 1) - 1022;  // xi 2^53 = m 2^sh, sh <= 0
          long long r = 0;
          if (sh == 0) r = m;
          else if (sh > -60) r = (m + (1ll << (-sh - 1))) >> (-sh);
          const long long k = r - (1ll << 52);
          if (order == 1) {
            k0 += (__int128)(k < 0 ? -k : 0);
            k1 += (__int128)(k > 0 ? k : 0);
          } else {
            k0 += (__int128)k;
            k1 += (__int128)k * (__int128)k;
          }
        }
#pragma unroll
        for (int q = 16; q > 0; q >>= 1) {
          k0 += shfl_xor_i128(k0, q);
          k1 += shfl_xor_i128(k1, q);
        }
        const double al = __longlong_as_double(wb);
        a0 = al * (double)n;
        if (order == 1) {
          a1 = al * i128_to_f64(k0, -53);
          a2 = al * i128_to_f64(k1, -53);
        } else {
          a1 = al * i128_to_f64(k0, -53);
          a2 = al * i128_to_f64(k1, -106);
        }
      }
    }
    if (!fixed) {
      for (int64_t p = lane; p < n; p += 32) {
        const double sx = cell_frac(x[o + p], j, inv_dx) - 0.5;
        const double al = alpha ? alpha[o + p] : 1.0;
        if (order == 1) {
          a0 += al;
          a1 = sx < 0.0 ? fma(-al, sx, a1) : a1;
          a2 = sx > 0.0 ? fma(al, sx, a2) : a2;
        } else {
          const double as = al * sx;
          a0 += al;
          a1 += as;
          a2 = fma(as, sx, a2);
        }
      }
      a0 = warp_sum(a0);
      a1 = warp_sum(a1);
      a2 = warp_sum(a2);
    }
    if (lane == 0) {
      if (order == 1) {
        part[3 * j + 0] = a1;
        part[3 * j + 1] = a0 - a1 - a2;
        part[3 * j + 2] = a2;
      } else {
        part[3 * j + 0] = 0.5 * (0.25 * a0 - a1 + a2);
        part[3 * j + 1] = 0.75 * a0 - a2;
        part[3 * j + 2] = 0.5 * (0.25 * a0 + a1 + a2);
      }
    }
  }
}

// rho_i = (q/dx) (part[i-1][+] + part[i][0] + part[i+1][-]), periodic
__global__ void deposit_combine_kernel(int64_t C, const double* part, double q_over_dx,
                                       double* rho) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < C;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t im = (i == 0) ? C - 1 : i - 1;
    const int64_t ip = (i == C - 1) ? 0 : i + 1;
    rho[i] = q_over_dx * (part[3 * im + 2] + part[3 * i + 1] + part[3 * ip + 0]);
  }
}

// W, p, M2 (upper triangle), E of each cell's particles
template <int D, int NT, typename VT>
__global__ void __launch_bounds__(NT) moments_kernel(int64_t C, int64_t n, const int64_t* cell_off,
                                                     const VT* v, const double* alpha, double* W,
                                                     double* p, double* M2, double* E) {
  constexpr int NM = D * (D + 1) / 2;
  constexpr int NV = 1 + D + NM + 1;
  __shared__ double red[NT / 32][NV];
  for (int64_t j = blockIdx.x; j < C; j += gridDim.x) {
    const int64_t o = cell_off[j], cnt = cell_off[j + 1] - o;
    double acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.0;
    for (int64_t q = threadIdx.x; q < cnt; q += NT) {
      const double al = alpha[o + q];
      double vv[D];
#pragma unroll
      for (int d = 0; d < D; ++d) vv[d] = (double)v[(int64_t)d * n + o + q];
      acc[0] += al;
      int t = 1 + D;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        acc[1 + a] += al * vv[a];
        acc[NV - 1] += 0.5 * al * vv[a] * vv[a];
#pragma unroll
        for (int b = a; b < D; ++b, ++t) acc[t] += al * vv[a] * vv[b];
      }
    }
    block_sum_to0<NT, NV>(acc, red);
    if (threadIdx.x == 0) {
      if (W) W[j] = acc[0];
      if (p)
        for (int a = 0; a < D; ++a) p[j * D + a] = acc[1 + a];
      if (M2)
        for (int t = 0; t < NM; ++t) M2[j * NM + t] = acc[1 + D + t];
      if (E) E[j] = acc[NV - 1];
    }
    __syncthreads();
  }
}

// the same moments of the mixtures (one thread per cell)
template <int D>
__global__ void mixture_moments_kernel(int64_t C, int Kmax, const int32_t* K, const double* prm,
                                       const double* Wc, double* W, double* p, double* M2,
                                       double* E) {
  constexpr int NM = D * (D + 1) / 2;
  constexpr int P = 1 + D + NM;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < C;
       j += (int64_t)gridDim.x * blockDim.x) {
    double pm[D], m2[NM];
    for (int a = 0; a < D; ++a) pm[a] = 0.0;
    for (int t = 0; t < NM; ++t) m2[t] = 0.0;
    const double w = Wc[j];
    for (int k = 0; k < K[j]; ++k) {
      const double* r = prm + ((size_t)j * Kmax + k) * P;
      int t = 0;
      for (int a = 0; a < D; ++a) {
        pm[a] += w * r[0] * r[1 + a];
        for (int b = a; b < D; ++b, ++t) m2[t] += w * r[0] * (r[1 + D + t] + r[1 + a] * r[1 + b]);
      }
    }
    if (W) W[j] = w;
    double e = 0.0;
    int t = 0;
    for (int a = 0; a < D; ++a) {
      if (p) p[j * D + a] = pm[a];
      for (int b = a; b < D; ++b, ++t) {
        if (a == b) e += 0.5 * m2[t];
        if (M2) M2[j * NM + t] = m2[t];
      }
    }
    if (E) E[j] = e;
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static int grid_for(int64_t C, int cap) { return (int)(C < cap ? (C > 0 ? C : 1) : cap); }

cudaError_t launch_deposit(int64_t C, const int64_t* cell_off, const double* x,
                           const double* alpha, double dx, double q, int order, double* part,
                           double* rho, cudaStream_t s) {
  if (C == 0) return cudaSuccess;
  deposit_partials_kernel<4><<<grid_for((C + 3) / 4, 152 * 16), 128, 0, s>>>(C, cell_off, x, alpha,
                                                                              1.0 / dx, order, part);
  deposit_combine_kernel<<<grid_for((C + 255) / 256, 1024), 256, 0, s>>>(C, part, q / dx, rho);
  return cudaGetLastError();
}

cudaError_t launch_moments(int D, int64_t C, int64_t n, const int64_t* cell_off, const void* v,
                           int v_f64, const double* alpha, double* W, double* p, double* M2,
                           double* E, cudaStream_t s) {
  if (C == 0) return cudaSuccess;
  const int g = grid_for(C, 152 * 16);
  if (D == 1) {
    if (v_f64)
      moments_kernel<1, 128, double><<<g, 128, 0, s>>>(C, n, cell_off, (const double*)v, alpha, W, p, M2, E);
    else
      moments_kernel<1, 128, float><<<g, 128, 0, s>>>(C, n, cell_off, (const float*)v, alpha, W, p, M2, E);
  } else {
    if (v_f64)
      moments_kernel<3, 128, double><<<g, 128, 0, s>>>(C, n, cell_off, (const double*)v, alpha, W, p, M2, E);
    else
      moments_kernel<3, 128, float><<<g, 128, 0, s>>>(C, n, cell_off, (const float*)v, alpha, W, p, M2, E);
  }
  return cudaGetLastError();
}

cudaError_t launch_mixture_moments(int D, int64_t C, int Kmax, const int32_t* K, const double* prm,
                                   const double* Wc, double* W, double* p, double* M2, double* E,
                                   cudaStream_t s) {
  if (C == 0) return cudaSuccess;
  const int g = grid_for((C + 127) / 128, 4096);
  if (D == 1)
    mixture_moments_kernel<1><<<g, 128, 0, s>>>(C, Kmax, K, prm, Wc, W, p, M2, E);
  else
    mixture_moments_kernel<3><<<g, 128, 0, s>>>(C, Kmax, K, prm, Wc, W, p, M2, E);
  return cudaGetLastError();
}

}  // namespace gmcr
