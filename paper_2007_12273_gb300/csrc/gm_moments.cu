// gm_moments.cu -- charge deposition (Sec. 2.4.1) and per-cell moments.
#include "deposit_cell.cuh"
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
// for i = j-1, j, j+1 (alpha = NULL means unit weights).  With s = xi - 1/2
// (xi the position inside the cell) the quadratic B-spline weights are
// (1/2 - s)^2 / 2, 3/4 - s^2, (1/2 + s)^2 / 2, so the three sums follow
// from A0 = sum alpha, A1 = sum alpha s, A2 = sum alpha s^2; for CIC they
// are sum alpha max(-s, 0), A0 - (the other two), sum alpha max(s, 0).
//
// deposit_partials_kernel, one warp per cell, writes each cell's sums to a
// record (deposit_cell.cuh); deposit_combine_kernel, one thread per node,
// turns the records of the node's three cells into the charge, so the
// per-cell FP64 work runs 32 cells to a warp instruction.
size_t deposit_ws_bytes(int64_t C) { return (size_t)kDepWords * 8 * (size_t)(C > 0 ? C : 0) + 256; }

template <int NW>
__global__ void __launch_bounds__(NW * 32) deposit_partials_kernel(int64_t C, const int64_t* cell_off,
                                                                   const double* x, const double* alpha,
                                                                   double inv_dx, int order,
                                                                   long long* rec) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t j = (int64_t)blockIdx.x * NW + wid; j < C; j += (int64_t)gridDim.x * NW) {
    const int64_t o = cell_off[j], n = cell_off[j + 1] - o;
    const bool same = n > 0 && n <= kFixMaxN && equal_weights(alpha, o, n, lane);
    deposit_cell(j, o, n, x, alpha, inv_dx, order, rec + (size_t)j * kDepWords, lane, same);
  }
}

// the three partial deposits of a cell (on its nodes j-1, j, j+1) from its
// record
__device__ __forceinline__ void dep_parts(const long long* r, int order, double (&pt)[3]) {
  double a0, a1, a2;
  if (r[5] >= 0) {
    const double al = __longlong_as_double(r[4]);
    const __int128 k0 = ((__int128)r[1] << 64) | (__int128)(unsigned long long)r[0];
    const __int128 k1 = ((__int128)r[3] << 64) | (__int128)(unsigned long long)r[2];
    a0 = al * (double)r[5];
    a1 = al * i128_to_f64(k0, -53);
    a2 = al * i128_to_f64(k1, order == 1 ? -53 : -106);
  } else {
    a0 = __longlong_as_double(r[0]);
    a1 = __longlong_as_double(r[1]);
    a2 = __longlong_as_double(r[2]);
  }
  if (order == 1) {
    pt[0] = a1;
    pt[1] = a0 - a1 - a2;
    pt[2] = a2;
  } else {
    pt[0] = 0.5 * (0.25 * a0 - a1 + a2);
    pt[1] = 0.75 * a0 - a2;
    pt[2] = 0.5 * (0.25 * a0 + a1 + a2);
  }
}

// rho_i = (q/dx) (part[i-1][+] + part[i][0] + part[i+1][-]), periodic
__global__ void deposit_combine_kernel(int64_t C, const long long* rec, int order, double q_over_dx,
                                       double* rho) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < C;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t im = (i == 0) ? C - 1 : i - 1;
    const int64_t ip = (i == C - 1) ? 0 : i + 1;
    double pm[3], p0[3], pp[3];
    dep_parts(rec + (size_t)im * kDepWords, order, pm);
    dep_parts(rec + (size_t)i * kDepWords, order, p0);
    dep_parts(rec + (size_t)ip * kDepWords, order, pp);
    rho[i] = q_over_dx * (pm[2] + p0[1] + pp[0]);
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
                           const double* alpha, double dx, double q, int order, void* ws,
                           double* rho, cudaStream_t s) {
  if (C == 0) return cudaSuccess;
  long long* rec = (long long*)ws;
  deposit_partials_kernel<4><<<grid_for((C + 3) / 4, 152 * 16), 128, 0, s>>>(C, cell_off, x, alpha,
                                                                              1.0 / dx, order, rec);
  deposit_combine_kernel<<<grid_for((C + 255) / 256, 1024), 256, 0, s>>>(C, rec, order, q / dx, rho);
  return cudaGetLastError();
}

cudaError_t launch_deposit_combine(int64_t C, double dx, double q, int order, const void* ws,
                                   double* rho, cudaStream_t s) {
  if (C == 0) return cudaSuccess;
  deposit_combine_kernel<<<grid_for((C + 255) / 256, 1024), 256, 0, s>>>(C, (const long long*)ws, order,
                                                                          q / dx, rho);
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
