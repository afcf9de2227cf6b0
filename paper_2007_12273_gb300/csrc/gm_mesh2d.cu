// gm_mesh2d.cu -- the reconstruction on a 2D doubly periodic mesh (Sec. 2.4
// with the tensor-product shape function S(x) S(y), the geometry of the
// 2D-3V Weibel runs of Sec. 3.2).  Cells and nodes are numbered
// j = jy Cx + jx; node (ix, iy) sits at the cell centre.
//
// Sampling, the per-cell velocity sums and the Lemons projection are those
// of the 1D path (recon_sampler.cuh), with one more uniform per particle for
// y.  The mass matrix M_ij = q sum_{p in j} S(x_i - x_p) S(y_i - y_p) has a
// 3 x 3 column per cell.  With the quadratic B-spline it is not diagonally
// dominant in 2D (a uniformly filled cell keeps (2/3)^2 of its weight on
// its own node), so M dA = dx dy (rho' - rho) is solved by defect
// correction with the operator of uniformly filled cells as preconditioner:
// P = (Tx (x) Ty) diag(q N'_j), T the circulant tridiagonal matrix of the
// mean shape weights (e, d0, e) = (1/6, 2/3, 1/6); CIC (1/8, 3/4, 1/8).
// T^-1 is circulant with entries c_k = (r^k + r^(n-k)) / ((1 - r^n) s),
// s = sqrt(d0^2 - 4 e^2), r = (s - d0) / (2 e) (r = -(2 - sqrt 3) for the
// quadratic B-spline: the images of the bi-infinite inverse), so P^-1 is a
// convolution along every row and then every column: all n entries for
// lines of at most 33 cells, else the 33 central ones (the first one left
// out is below 2e-10 of c_0; the residual is always formed with the true M,
// so the preconditioner's truncation changes the rate, not the solution).
// Each iteration is a residual pass, an x pass and a y pass (three
// launches, each a no-op once the residual is below the tolerance).  A cell
// without resampled particles has a unit column: its unknown appears in its
// own row only, so it is left out of the iteration and found afterwards
// from its row.
#include "recon_sampler.cuh"

namespace gmcr {

// shape weights of an in-cell offset s = u - 1/2 on the nodes -1, 0, +1 of
// its cell (the B-spline S(a - s)): quadratic (1/2 - s)^2 / 2, 3/4 - s^2,
// (1/2 + s)^2 / 2; CIC max(-s, 0), 1 - |s|, max(s, 0)
__device__ __forceinline__ void shape3(int order, double s, double (&w)[3]) {
  if (order == 1) {
    w[0] = s < 0.0 ? -s : 0.0;
    w[2] = s > 0.0 ? s : 0.0;
    w[1] = 1.0 - (w[0] + w[2]);
  } else {
    const double a = 0.5 - s, b = 0.5 + s;
    w[0] = 0.5 * a * a;
    w[1] = 0.75 - s * s;
    w[2] = 0.5 * b * b;
  }
}

// part[j][3 (b + 1) + (a + 1)] = sum_{p in j} alpha_p S(x-weight a) S(y-weight b):
// what cell j's particles put on node (jx + a, jy + b).  One warp per cell;
// alpha = NULL means unit weights.
template <int NW>
__global__ void __launch_bounds__(NW * 32) deposit2d_partials_kernel(
    int64_t Cx, int64_t C, const int64_t* cell_off, const double* x, const double* y,
    const double* alpha, double inv_dx, double inv_dy, int order, double* part) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t j = (int64_t)blockIdx.x * NW + wid; j < C; j += (int64_t)gridDim.x * NW) {
    const int64_t jx = j % Cx, jy = j / Cx;
    const int64_t o = cell_off[j], n = cell_off[j + 1] - o;
    double acc[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) acc[t] = 0.0;
    for (int64_t p = lane; p < n; p += 32) {
      double wx[3], wy[3];
      shape3(order, cell_frac(x[o + p], (double)jx, inv_dx) - 0.5, wx);
      shape3(order, cell_frac(y[o + p], (double)jy, inv_dy) - 0.5, wy);
      const double al = alpha ? alpha[o + p] : 1.0;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const double ab = al * wy[b];
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[3 * b + a] = fma(ab, wx[a], acc[3 * b + a]);
      }
    }
#pragma unroll
    for (int t = 0; t < 9; ++t) acc[t] = warp_sum(acc[t]);
    if (lane == 0)
#pragma unroll
      for (int t = 0; t < 9; ++t) part[9 * j + t] = acc[t];
  }
}

// the cell whose entry (a, b) lands on node (ix, iy): (ix - a, iy - b), periodic
__device__ __forceinline__ int64_t src_cell(int64_t ix, int64_t iy, int a, int b, int64_t Cx,
                                            int64_t Cy) {
  int64_t sx = ix - a, sy = iy - b;
  sx = sx < 0 ? sx + Cx : (sx >= Cx ? sx - Cx : sx);
  sy = sy < 0 ? sy + Cy : (sy >= Cy ? sy - Cy : sy);
  return sy * Cx + sx;
}

// rho_i = q / (dx dy) sum over the 3 x 3 cells around node i of their entry on it
__global__ void deposit2d_combine_kernel(int64_t Cx, int64_t Cy, const double* part,
                                         double q_over_dv, double* rho) {
  const int64_t C = Cx * Cy;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < C;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ix = i % Cx, iy = i / Cx;
    double s = 0.0;
    for (int b = -1; b <= 1; ++b)
      for (int a = -1; a <= 1; ++a) s += part[9 * src_cell(ix, iy, a, b, Cx, Cy) + 3 * (b + 1) + (a + 1)];
    rho[i] = q_over_dv * s;
  }
}

// Pass 1, one warp per cell: cstat[j] = [9 unit-weight shape sums (layout of
// part above), sum w (D), sum |w|^2] of the resampled particles
template <int D, int NW>
__global__ void __launch_bounds__(NW * 32) recon2d_stats_kernel(
    int64_t Cx, int64_t C, int Kmax, const int32_t* K, const double* prm, const int64_t* out_off,
    int64_t n_out, uint64_t seed, int order, double* cstat) {
  constexpr int NV = 9 + D + 1;
  __shared__ RecCell<D> rcs[NW];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  RecCell<D>& rc = rcs[wid];
  for (int64_t j = (int64_t)blockIdx.x * NW + wid; j < C; j += (int64_t)gridDim.x * NW) {
    load_cell<D>(rc, j, Kmax, K, prm, lane);
    __syncwarp();
    int64_t o, n;
    out_range(out_off, j, n_out, o, n);
    double acc[NV];
#pragma unroll
    for (int t = 0; t < NV; ++t) acc[t] = 0.0;
    for (int64_t i = lane; i < n; i += 32) {
      uint64_t m0;
      double w[D], wx[3], wy[3];
      sample_particle<D>(rc, j, i, seed, m0, w);
      shape3(order, centred52(m0), wx);
      shape3(order, centred52(sample_y_bits(j, i, seed)), wy);
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[3 * b + a] = fma(wy[b], wx[a], acc[3 * b + a]);
#pragma unroll
      for (int d = 0; d < D; ++d) {
        acc[9 + d] += w[d];
        acc[9 + D] = fma(w[d], w[d], acc[9 + D]);
      }
    }
#pragma unroll
    for (int t = 0; t < NV; ++t) acc[t] = warp_sum(acc[t]);
    if (lane == 0)
#pragma unroll
      for (int t = 0; t < NV; ++t) cstat[(size_t)j * NV + t] = acc[t];
    __syncwarp();
  }
}

// order-preserving bits of a non-negative double (for atomicMax)
__device__ __forceinline__ unsigned long long pos_bits(double v) {
  return (unsigned long long)__double_as_longlong(v);
}

constexpr int kCircTaps = 33;  // entries of T^-1 kept per direction
constexpr int kCircHalf = 16;  // window half-width for lines of more than kCircTaps cells

struct Mesh2dSolve {
  int64_t Cx, Cy;
  const double* cstat;   // [C][NV]
  int nv;                // 9 + D + 1
  const int64_t* out_off;
  int64_t n_out;
  double q;
  double* b;             // [C] right-hand side dx dy (rho' - rho)
  double* dA;            // [C]
  double* r;             // [C] residual
  double* t;             // [C] after the x sweep
  unsigned long long* norm;  // [max_iter + 1] max |r| per iteration (as bits)
  unsigned long long* scale; // [1] max |dx dy rho'| (as bits)
  double tol;
};

// rows of the right-hand side, the iteration's norms cleared, dA = 0
__global__ void assemble2d_kernel(Mesh2dSolve m, const double* W, const double* rho_target,
                                  double dv, int max_iter) {
  const int64_t C = m.Cx * m.Cy;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < C;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ix = i % m.Cx, iy = i / m.Cx;
    double s = 0.0;
    for (int b = -1; b <= 1; ++b)
      for (int a = -1; a <= 1; ++a) {
        const int64_t src = src_cell(ix, iy, a, b, m.Cx, m.Cy);
        const int64_t ns = out_count(m.out_off, src, m.n_out);
        if (ns > 0) s += (W[src] / (double)ns) * m.cstat[(size_t)src * m.nv + 3 * (b + 1) + (a + 1)];
      }
    const double tgt = dv * rho_target[i];
    m.b[i] = tgt - m.q * s;
    m.dA[i] = 0.0;
    atomicMax(m.scale, pos_bits(fabs(tgt)));
    if (i <= max_iter) m.norm[i] = 0ull;
  }
}

// r_i = b_i - (M dA)_i on the rows of cells with particles (empty rows 0);
// block maximum of |r| into norm[it].  A no-op once iteration it - 1 has
// converged.
__global__ void __launch_bounds__(256) mm2d_residual_kernel(Mesh2dSolve m, int it) {
  __shared__ double red[8];
  const double thr = m.tol * __longlong_as_double((long long)*m.scale);
  if (it > 0 && __longlong_as_double((long long)m.norm[it - 1]) <= thr) return;
  const int64_t C = m.Cx * m.Cy;
  double mx = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < C;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ix = i % m.Cx, iy = i / m.Cx;
    double ri = 0.0;
    if (out_count(m.out_off, i, m.n_out) > 0) {
      double s = 0.0;
      for (int b = -1; b <= 1; ++b)
        for (int a = -1; a <= 1; ++a) {
          const int64_t src = src_cell(ix, iy, a, b, m.Cx, m.Cy);
          if (out_count(m.out_off, src, m.n_out) > 0)
            s = fma(m.cstat[(size_t)src * m.nv + 3 * (b + 1) + (a + 1)], m.dA[src], s);
        }
      ri = m.b[i] - m.q * s;
    }
    m.r[i] = ri;
    mx = fmax(mx, fabs(ri));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) mx = fmax(mx, red[q]);
    atomicMax(m.norm + it, pos_bits(mx));
  }
}

// entries of T^-1 along one direction (host-computed, passed by value)
struct CircTaps {
  int full;        // 1: all n entries c_0 .. c_{n-1}; 0: c_0 .. c_16 (window)
  double c[kCircTaps];
};

// (T^-1 line)_i for a line of n values at stride st
__device__ __forceinline__ double circ_apply(const CircTaps& T, const double* line, int64_t n,
                                             int64_t i, int64_t st) {
  double s = 0.0;
  if (T.full) {
#pragma unroll
    for (int k = 0; k < kCircTaps; ++k)
      if (k < n) {
        int64_t j = i - k;
        j = j < 0 ? j + n : j;
        s = fma(T.c[k], line[j * st], s);
      }
    return s;
  }
  s = T.c[0] * line[i * st];
#pragma unroll
  for (int k = 1; k <= kCircHalf; ++k) {
    int64_t jm = i - k, jp = i + k;
    jm = jm < 0 ? jm + n : jm;
    jp = jp >= n ? jp - n : jp;
    s = fma(T.c[k], line[jm * st] + line[jp * st], s);
  }
  return s;
}

// x pass: t = (Tx^-1 along every row) r, one thread per node
__global__ void mm2d_xsweep_kernel(Mesh2dSolve m, int it, CircTaps tx) {
  const double thr = m.tol * __longlong_as_double((long long)*m.scale);
  if (__longlong_as_double((long long)m.norm[it]) <= thr) return;
  const int64_t C = m.Cx * m.Cy;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < C;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ix = i % m.Cx, row = i - ix;
    m.t[i] = circ_apply(tx, m.r + row, m.Cx, ix, 1);
  }
}

// y pass: dA_j += (Ty^-1 along every column of t)_j / (q N'_j) on cells with
// particles, one thread per node
__global__ void mm2d_ysweep_kernel(Mesh2dSolve m, int it, CircTaps ty) {
  const double thr = m.tol * __longlong_as_double((long long)*m.scale);
  if (__longlong_as_double((long long)m.norm[it]) <= thr) return;
  const int64_t C = m.Cx * m.Cy;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < C;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = out_count(m.out_off, i, m.n_out);
    if (n == 0) continue;
    const int64_t ix = i % m.Cx, iy = i / m.Cx;
    m.dA[i] += circ_apply(ty, m.t + ix, m.Cy, iy, m.Cx) / (m.q * (double)n);
  }
}

// the entries of T^-1 for a periodic line of n cells (closed form above)
static CircTaps circ_taps(int64_t n, double e, double d0) {
  CircTaps T;
  const double sq = sqrt(d0 * d0 - 4.0 * e * e), r = (sq - d0) / (2.0 * e);
  const double rn = pow(r, (double)n);
  T.full = n <= kCircTaps ? 1 : 0;
  const int cnt = T.full ? (int)n : kCircHalf + 1;
  for (int k = 0; k < kCircTaps; ++k) T.c[k] = 0.0;
  for (int k = 0; k < cnt; ++k)
    T.c[k] = (pow(r, (double)k) + pow(r, (double)(n - k))) / ((1.0 - rn) * sq);
  return T;
}

// after the iterations: the unknowns of empty cells from their own rows
// (unit diagonal), and the convergence status of the solve
__global__ void mm2d_finish_kernel(Mesh2dSolve m, int max_iter, int* converged) {
  const double thr = m.tol * __longlong_as_double((long long)*m.scale);
  const int64_t C = m.Cx * m.Cy;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < C;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i == 0) {
      int conv = 0;
      for (int k = 0; k <= max_iter; ++k)
        if (__longlong_as_double((long long)m.norm[k]) <= thr) conv = 1;
      *converged = conv;
    }
    if (out_count(m.out_off, i, m.n_out) > 0) continue;
    const int64_t ix = i % m.Cx, iy = i / m.Cx;
    double s = 0.0;
    for (int b = -1; b <= 1; ++b)
      for (int a = -1; a <= 1; ++a) {
        const int64_t src = src_cell(ix, iy, a, b, m.Cx, m.Cy);
        if (out_count(m.out_off, src, m.n_out) > 0)
          s = fma(m.cstat[(size_t)src * m.nv + 3 * (b + 1) + (a + 1)], m.dA[src], s);
      }
    m.dA[i] = m.b[i] - m.q * s;
  }
}

// Pass 2, one warp per cell: projection coefficients and the final particles
template <int D, int NW>
__global__ void __launch_bounds__(NW * 32) recon2d_emit_kernel(
    int64_t Cx, int64_t C, int Kmax, const int32_t* K, const double* prm, const double* W,
    const int64_t* out_off, const double* cstat, const double* dA, const int* converged,
    uint64_t seed, double dx, double dy, int64_t n_out, double* x_out, double* y_out, double* v_out,
    double* alpha_out, uint32_t* status_out) {
  constexpr int NV = 9 + D + 1;
  __shared__ RecCell<D> rcs[NW];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  RecCell<D>& rc = rcs[wid];
  for (int64_t j = (int64_t)blockIdx.x * NW + wid; j < C; j += (int64_t)gridDim.x * NW) {
    const int64_t jx = j % Cx, jy = j / Cx;
    load_cell<D>(rc, j, Kmax, K, prm, lane);
    __syncwarp();
    int64_t o, n;
    const bool in_range = out_range(out_off, j, n_out, o, n);
    if (lane == 0)
      status_out[j] = projection_coeffs<D>(rc, n, W[j], dA[j], cstat + (size_t)j * NV + 9) |
                      (*converged ? 0u : GM_ST_MM_NOT_CONVERGED) | (in_range ? 0u : GM_ST_BAD_RANGE);
    __syncwarp();
    const double aa = rc.a, an = rc.alpha_new;
    const int skip = rc.skip;
    for (int64_t i = lane; i < n; i += 32) {
      uint64_t m0;
      double w[D];
      sample_particle<D>(rc, j, i, seed, m0, w);
      const double u0 = uniform_pos52(m0);
      const double uy =
          uniform_pos52(sample_y_bits(j, i, seed));
      x_out[o + i] = __dmul_rn(__dadd_rn((double)jx, u0), dx);
      y_out[o + i] = __dmul_rn(__dadd_rn((double)jy, uy), dy);
      alpha_out[o + i] = an;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const double vp = skip ? rc.u[d] + w[d] : fma(aa, w[d] + rc.beta[d], rc.u[d]);
        v_out[(int64_t)d * n_out + o + i] = vp;
      }
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
static int grid_cap(int64_t units, int per, int cap) {
  const int64_t g = (units + per - 1) / per;
  return (int)(g < 1 ? 1 : (g < cap ? g : cap));
}

cudaError_t launch_deposit2d(int64_t Cx, int64_t Cy, const int64_t* cell_off, const double* x,
                             const double* y, const double* alpha, double dx, double dy, double q,
                             int order, double* part, double* rho, cudaStream_t s) {
  const int64_t C = Cx * Cy;
  if (C == 0) return cudaSuccess;
  deposit2d_partials_kernel<4><<<grid_cap(C, 4, 152 * 16), 128, 0, s>>>(
      Cx, C, cell_off, x, y, alpha, 1.0 / dx, 1.0 / dy, order, part);
  deposit2d_combine_kernel<<<grid_cap(C, 256, 1024), 256, 0, s>>>(Cx, Cy, part, q / (dx * dy), rho);
  return cudaGetLastError();
}

size_t reconstruct2d_ws_bytes(int D, int64_t Cx, int64_t Cy) {
  const int64_t C = Cx * Cy;
  const size_t dbl = (size_t)(9 + D + 1) * C + 4 * (size_t)C + (kMesh2dMaxIter + 1) + 1;
  return dbl * sizeof(double) + 1024;
}

cudaError_t launch_reconstruct2d(int D, int64_t Cx, int64_t Cy, int Kmax, const int32_t* K,
                                 const double* prm, const double* W, const double* rho_target,
                                 int64_t n_out, const int64_t* out_off, uint64_t seed, double dx,
                                 double dy, double q, int order, double* x_out, double* y_out,
                                 double* v_out, double* alpha_out, uint32_t* status_out,
                                 double* dA_user, void* ws, cudaStream_t s) {
  const int64_t C = Cx * Cy;
  if (C == 0) return cudaSuccess;
  const int NVm = 9 + D + 1;
  double* base = (double*)ws;
  Mesh2dSolve m;
  m.Cx = Cx;
  m.Cy = Cy;
  double* cstat = base;
  m.cstat = cstat;
  m.nv = NVm;
  m.out_off = out_off;
  m.n_out = n_out;
  m.q = q;
  m.b = cstat + (size_t)NVm * C;
  m.dA = m.b + C;
  m.r = m.dA + C;
  m.t = m.r + C;
  m.norm = (unsigned long long*)(m.t + C);
  m.scale = m.norm + kMesh2dMaxIter + 1;
  int* converged = (int*)(m.scale + 1);
  m.tol = kMesh2dTol;
  if (dA_user) m.dA = dA_user;
  const double e = order == 1 ? 0.125 : 1.0 / 6.0;
  const double d0 = order == 1 ? 0.75 : 2.0 / 3.0;
  const CircTaps tx = circ_taps(Cx, e, d0), ty = circ_taps(Cy, e, d0);

  constexpr int NW = 4;
  const int g = grid_cap(C, NW, 152 * 16);
  cudaError_t err = cudaMemsetAsync(m.scale, 0, sizeof(unsigned long long), s);
  if (err != cudaSuccess) return err;
  if (D == 1)
    recon2d_stats_kernel<1, NW><<<g, NW * 32, 0, s>>>(Cx, C, Kmax, K, prm, out_off, n_out, seed, order,
                                                      cstat);
  else
    recon2d_stats_kernel<3, NW><<<g, NW * 32, 0, s>>>(Cx, C, Kmax, K, prm, out_off, n_out, seed, order,
                                                      cstat);
  const int ga = grid_cap(C > kMesh2dMaxIter + 1 ? C : kMesh2dMaxIter + 1, 256, 2048);
  assemble2d_kernel<<<ga, 256, 0, s>>>(m, W, rho_target, dx * dy, kMesh2dMaxIter);
  // norm[i] for i < C is cleared by the grid-stride loop above; meshes with
  // fewer cells than iterations clear the rest here
  if (C <= kMesh2dMaxIter) {
    err = cudaMemsetAsync(m.norm + C, 0, sizeof(unsigned long long) * (kMesh2dMaxIter + 1 - C), s);
    if (err != cudaSuccess) return err;
  }
  const int gr = grid_cap(C, 256, 152 * 4);
  for (int it = 0; it < kMesh2dMaxIter; ++it) {
    mm2d_residual_kernel<<<gr, 256, 0, s>>>(m, it);
    mm2d_xsweep_kernel<<<gr, 256, 0, s>>>(m, it, tx);
    mm2d_ysweep_kernel<<<gr, 256, 0, s>>>(m, it, ty);
  }
  mm2d_residual_kernel<<<gr, 256, 0, s>>>(m, kMesh2dMaxIter);
  mm2d_finish_kernel<<<grid_cap(C, 256, 1024), 256, 0, s>>>(m, kMesh2dMaxIter, converged);
  if (D == 1)
    recon2d_emit_kernel<1, NW><<<g, NW * 32, 0, s>>>(Cx, C, Kmax, K, prm, W, out_off, cstat, m.dA,
                                                      converged, seed, dx, dy, n_out, x_out, y_out,
                                                      v_out, alpha_out, status_out);
  else
    recon2d_emit_kernel<3, NW><<<g, NW * 32, 0, s>>>(Cx, C, Kmax, K, prm, W, out_off, cstat, m.dA,
                                                      converged, seed, dx, dy, n_out, x_out, y_out,
                                                      v_out, alpha_out, status_out);
  return cudaGetLastError();
}

}  // namespace gmcr
