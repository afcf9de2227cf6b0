// gm_reconstruct.cu -- particle reconstruction (Sec. 2.4): ancestral
// sampling, the Gauss'-law mass-matrix weight correction and the Lemons
// moment-matching projection.
//
// The sampler is counter-based, so a particle can be regenerated
// bit-identically from (seed, cell, index).  It keeps FP64 to the position
// and to the velocity's offset from the mixture mean (so that both passes
// see the same w = v - u, which is what makes the projected moments exact);
// the categorical choice is decided on integers and the Gaussian draw is
// FP32 (GB300 runs FP64 at 1/64 of the FP32 rate).  The pipeline never
// writes unprojected particles:
//   pass 0 (one thread per cell) prepares each cell's mixture data;
//   pass 1 (one warp per cell) draws every particle, accumulates the
//     per-cell mass-matrix column and the velocity sums, and stages the
//     draw (20 bytes) in the particle's own output slots;
//   a small FP64 solve gives dA, and one thread per cell the projection
//     coefficients;
//   pass 2 (one warp per cell) reads each staged draw back and writes the
//     final position, projected velocity and corrected weight over it.
// HBM traffic: the staged draws (written once, read once) and the output,
// 8 (x) + 8 D (v) + 8 (alpha) bytes per particle.
#include "recon_sampler.cuh"

namespace gmcr {

// Per-cell sums of the resampled particles, written by pass 1 (raw_words
// doubles per cell).  A one-component cell with at most kFixMaxN particles
// keeps exact 128-bit integer sums (see below), every other cell FP64 sums:
//   integer: words (2t, 2t+1) hold sum t as (low, high) 64-bit halves, t =
//            0, 1 the position sums, 2 .. 1+D the sums of f_d, 2+D .. 1+2D
//            those of f_d^2;
//   FP64:    words 0, 1 the position sums, 2 .. 1+D the sums of f_d (one
//            component) or w_d (otherwise), 2+D the sum of |f|^2 or |w|^2.
// The position sums are S1 = sum s, S2 = sum s^2 (quadratic B-spline) or
// sum max(-s, 0), sum max(s, 0) (CIC), s = xi - 1/2 the particle's offset
// from the cell centre; w = v - u = dz + f with f = L_z xi.
template <int D>
__host__ __device__ constexpr int raw_words() { return 2 * (2 + 2 * D); }
__device__ __forceinline__ bool fixed_sums(int Kj, int64_t n) { return Kj == 1 && n <= kFixMaxN; }
__device__ __forceinline__ __int128 load_i128(const double* p) {
  const longlong2 v = *reinterpret_cast<const longlong2*>(p);
  return ((__int128)v.y << 64) | (__int128)(unsigned long long)v.x;
}
// the exponents eq_d of the fixed-point f_d: |f_d| <= 9 sum_e |L_de|
// (|xi| <= sqrt(-2 ln 2^-53) = 8.6) keeps f_d / 2^eq_d below 2^kFixBits
template <int D>
__device__ __forceinline__ void fix_exponents(const float* L, int (&eq)[D]) {
  float bnd[D];
  if (D == 1) {
    bnd[0] = fabsf(L[0]);
  } else {
    bnd[0] = fabsf(L[0]);
    bnd[1] = fabsf(L[1]) + fabsf(L[2]);
    bnd[D - 1] = fabsf(L[3]) + fabsf(L[4]) + fabsf(L[5]);
  }
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const int eb = (int)((__float_as_uint(9.0f * bnd[d]) >> 23) & 0xFFu);
    eq[d] = (eb ? eb - 127 : -126) + 1 - kFixBits;
  }
}
// Pass 1 stages each particle's draw in the caller's output slots of that
// same particle, and pass 2 reads it back before it overwrites them with
// the final values (one thread reads, then writes, each particle's slots,
// so no other particle's staging is ever touched): x_out[p] holds the
// position integer m0 (52 bits) and the component z (bits 56-63),
// alpha_out[p] the FP32 pair (f_0, f_1), v_out[0][p] (D = 3) the FP32 f_2.
// The second pass then needs neither the Philox draws nor the Box-Muller
// transform of the first.
template <int D>
__device__ __forceinline__ void stage_draw(double* x_out, double* v_out, double* alpha_out,
                                           int64_t p, uint64_t m0, int z, const float (&f)[D]) {
  reinterpret_cast<unsigned long long*>(x_out)[p] = m0 | ((unsigned long long)(z & 0xFF) << 56);
  reinterpret_cast<float2*>(alpha_out)[p] = make_float2(f[0], D == 3 ? f[1] : 0.0f);
  if (D == 3) reinterpret_cast<float2*>(v_out)[p] = make_float2(f[D - 1], 0.0f);
}
template <int D>
__device__ __forceinline__ void load_draw(const double* x_out, const double* v_out,
                                          const double* alpha_out, int64_t p, uint64_t& m0, int& z,
                                          float (&f)[D]) {
  const unsigned long long t = reinterpret_cast<const unsigned long long*>(x_out)[p];
  m0 = t & ((1ull << 52) - 1ull);
  z = (int)(t >> 56);
  const float2 a = reinterpret_cast<const float2*>(alpha_out)[p];
  f[0] = a.x;
  if (D == 3) {
    f[1] = a.y;
    f[D - 1] = reinterpret_cast<const float2*>(v_out)[p].x;
  }
}

// the unit-weight shape sums of a cell's n particles on nodes j-1, j, j+1
// (cs[0], cs[1], cs[2]): c- = (n/4 - S1 + S2) / 2, c+ = (n/4 + S1 + S2) / 2,
// c0 = 3n/4 - S2 for the quadratic B-spline; c- = sum max(-s, 0),
// c+ = sum max(s, 0), c0 = n - c- - c+ for CIC
__device__ __forceinline__ void shape_sums(const double* rw, bool fixed, int order, int64_t n,
                                           double (&cs)[3]) {
  double a0, a1;
  if (fixed) {
    a0 = i128_to_f64(load_i128(rw), -53);
    a1 = i128_to_f64(load_i128(rw + 2), order == 1 ? -53 : -106);
  } else {
    a0 = rw[0];
    a1 = rw[1];
  }
  const double nd = (double)n;
  if (order == 1) {
    cs[0] = a0;
    cs[2] = a1;
    cs[1] = nd - a0 - a1;
  } else {
    cs[0] = 0.5 * (0.25 * nd - a0 + a1);
    cs[2] = 0.5 * (0.25 * nd + a0 + a1);
    cs[1] = 0.75 * nd - a1;
  }
}
// sum w (sw[0 .. D-1]) and sum |w|^2 (sw[D]) of a cell; for one component
// w = dz + f with one dz, so sum w = n dz + sum f and
// sum |w|^2 = n |dz|^2 + 2 dz . sum f + sum |f|^2
template <int D>
__device__ __forceinline__ void velocity_sums(const double* rw, bool fixed, int Kj,
                                              const RecComp<D>& c0, int64_t n, double (&sw)[D + 1]) {
  if (fixed) {
    int eq[D];
    fix_exponents<D>(c0.Lf, eq);
    sw[D] = 0.0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      sw[d] = i128_to_f64(load_i128(rw + 4 + 2 * d), eq[d]);
      sw[D] += i128_to_f64(load_i128(rw + 4 + 2 * (D + d)), 2 * eq[d]);
    }
  } else {
#pragma unroll
    for (int t = 0; t <= D; ++t) sw[t] = rw[2 + t];
  }
  if (Kj == 1) {
    const double nd = (double)n;
    double dzf = 0.0, dz2 = 0.0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const double dz = c0.dz[d];
      dzf = fma(dz, sw[d], dzf);
      dz2 = fma(dz, dz, dz2);
      sw[d] = fma(nd, dz, sw[d]);
    }
    sw[D] = fma(nd, dz2, fma(2.0, dzf, sw[D]));
  }
}

// Pass 0, one thread per cell: each cell's mixture data for the two particle
// passes (prep_cell).
template <int D>
__global__ void recon_prep_kernel(int64_t C, int Kmax, const int32_t* K, const double* prm,
                                  RecHead<D>* head, RecComp<D>* comp) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < C;
       j += (int64_t)gridDim.x * blockDim.x)
    prep_cell<D>(j, Kmax, K, prm, head, comp);
}

// Pass 1, one warp per cell: the position and velocity sums of the cell's
// resampled particles (raw_words layout above).
template <int D, int NW>
__global__ void __launch_bounds__(NW * 32, 6) recon_stats_kernel(int64_t C, int Kmax,
                                                              const RecHead<D>* head,
                                                              const RecComp<D>* comp,
                                                              const int64_t* out_off, int64_t n_out,
                                                              uint64_t seed, int order, double* raw,
                                                              double* x_out, double* v_out,
                                                              double* alpha_out) {
  constexpr int NA = 2 + D + 1;
  constexpr int NS = 2 + 2 * D;
  __shared__ RecCell<D> rcs[NW];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  RecCell<D>& rc = rcs[wid];
  for (int64_t j = (int64_t)blockIdx.x * NW + wid; j < C; j += (int64_t)gridDim.x * NW) {
    load_prepped<D>(rc, j, Kmax, head, comp, lane);
    __syncwarp();
    int64_t o, n;
    out_range(out_off, j, n_out, o, n);
    double* rw = raw + (size_t)j * raw_words<D>();
    if (fixed_sums(rc.K, n)) {
      // one component: all sums on the integer pipe, exactly: the in-cell
      // position offset s = k 2^-53 with the odd integer
      // k = 2 m0 - 2^52 + 1, and f_d taken as an integer multiple of 2^eq_d
      // (exact within 2^-30 of the bound, to 2^-55 of it below)
      int eq[D];
      fix_exponents<D>(rc.Lf[0], eq);
      // a lane sums at most kFixMaxN / 32 = 512 terms, so its sums of
      // k (|k| < 2^52) and of f_d / 2^eq_d (below 0.96 x 2^54: |xi| <= 8.6
      // against the bound's 9) stay below 2^63 and fit in 64 bits; the
      // squares take 128
      __int128 sm[NS];
      long long s0 = 0, sf[D];
#pragma unroll
      for (int t = 0; t < NS; ++t) sm[t] = 0;
#pragma unroll
      for (int d = 0; d < D; ++d) sf[d] = 0;
      for (int64_t i = lane; i < n; i += 32) {
        uint64_t m0;
        int z;
        float f[D];
        sample_f<D>(rc, j, i, seed, m0, z, f);
        stage_draw<D>(x_out, v_out, alpha_out, o + i, m0, z, f);
        const long long k = 2ll * (long long)m0 - (1ll << 52) + 1ll;
        if (order == 1) {
          s0 += k < 0 ? -k : 0;
          sm[1] += (__int128)(k > 0 ? k : 0);
        } else {
          s0 += k;
          sm[1] += (__int128)k * (__int128)k;
        }
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const long long fq = fixq(f[d], eq[d]);
          sf[d] += fq;
          sm[2 + D + d] += (__int128)fq * (__int128)fq;
        }
      }
      sm[0] = (__int128)s0;
#pragma unroll
      for (int d = 0; d < D; ++d) sm[2 + d] = (__int128)sf[d];
      __int128 mine = 0;
#pragma unroll
      for (int t = 0; t < NS; ++t) {
#pragma unroll
        for (int o2 = 16; o2 > 0; o2 >>= 1) sm[t] += shfl_xor_i128(sm[t], o2);
        if (lane == t) mine = sm[t];
      }
      if (lane < NS)
        *reinterpret_cast<longlong2*>(rw + 2 * lane) =
            make_longlong2((long long)(unsigned long long)mine, (long long)(mine >> 64));
    } else {
      double acc[NA];
#pragma unroll
      for (int t = 0; t < NA; ++t) acc[t] = 0.0;
      for (int64_t i = lane; i < n; i += 32) {
        uint64_t m0;
        int z;
        float f[D];
        double w[D];
        sample_f<D>(rc, j, i, seed, m0, z, f);
        stage_draw<D>(x_out, v_out, alpha_out, o + i, m0, z, f);
        if (rc.K == 1) {
          // the f sums (above 2^14 particles)
#pragma unroll
          for (int d = 0; d < D; ++d) w[d] = f2d_exact(f[d]);
        } else {
          draw_offset<D>(rc, z, f, w);
        }
        const double sx = centred52(m0);
        if (order == 1) {
          acc[0] += sx < 0.0 ? -sx : 0.0;
          acc[1] += sx > 0.0 ? sx : 0.0;
        } else {
          acc[0] += sx;
          acc[1] = fma(sx, sx, acc[1]);
        }
#pragma unroll
        for (int d = 0; d < D; ++d) {
          acc[2 + d] += w[d];
          acc[2 + D] = fma(w[d], w[d], acc[2 + D]);
        }
      }
#pragma unroll
      for (int t = 0; t < NA; ++t) acc[t] = warp_sum(acc[t]);
      if (lane == 0)
        for (int t = 0; t < NA; ++t) rw[t] = acc[t];
    }
    __syncwarp();
  }
}

// Mass matrix rows (eq. below new-p-weight): row i couples dA_{i-1}, dA_i,
// dA_{i+1}; M(i,j) = q * (shape sum of cell j's particles on node i).
// rhs_i = dx (rho'_i - rho_i), rho_i dx = q sum_j alpha_j (shape sum).
template <int D>
__global__ void assemble_kernel(int64_t C, const RecHead<D>* head, const double* raw,
                                const double* W, const int64_t* out_off, int64_t n_out,
                                const double* rho_target, double dx, double q, int order, double* A,
                                double* B, double* Cc, double* Dd) {
  constexpr int RW = raw_words<D>();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < C;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t im = (i == 0) ? C - 1 : i - 1;
    const int64_t ip = (i == C - 1) ? 0 : i + 1;
    const int64_t nm = out_count(out_off, im, n_out);
    const int64_t n0 = out_count(out_off, i, n_out);
    const int64_t np = out_count(out_off, ip, n_out);
    const double am = nm > 0 ? W[im] / (double)nm : 0.0;
    const double a0 = n0 > 0 ? W[i] / (double)n0 : 0.0;
    const double ap = np > 0 ? W[ip] / (double)np : 0.0;
    double sm[3], s0[3], sp[3];
    shape_sums(raw + (size_t)im * RW, fixed_sums(head[im].K, nm), order, nm, sm);
    shape_sums(raw + (size_t)i * RW, fixed_sums(head[i].K, n0), order, n0, s0);
    shape_sums(raw + (size_t)ip * RW, fixed_sums(head[ip].K, np), order, np, sp);
    const double cm = sm[2];  // cell i-1 on node i
    const double c0 = s0[1];
    const double cp = sp[0];  // cell i+1 on node i
    A[i] = q * cm;
    B[i] = n0 > 0 ? q * c0 : 1.0;  // empty column: unit diagonal
    Cc[i] = q * cp;
    Dd[i] = dx * rho_target[i] - q * (am * cm + a0 * c0 + ap * cp);
  }
}

// Sequential cyclic tridiagonal solve (Thomas elimination and a rank-one
// Sherman-Morrison correction for the corners), one thread, n >= 3.
// Row r: a_r x_{r-1} + b_r x_r + c_r x_{r+1} = d_r (indices mod n).
__device__ void cyclic_thomas_seq(int64_t n, const double* a, const double* b, const double* c,
                                  const double* d, double* x, double* cp, double* y, double* z) {
  const double g = -b[0];
  const double corner = a[0] / g;
  // forward elimination with two right-hand sides: d and u = (g, 0..0, c_{n-1})
  double bb = b[0] - g;
  double r = 1.0 / bb;
  cp[0] = c[0] * r;
  y[0] = d[0] * r;
  z[0] = g * r;
  for (int64_t i = 1; i < n; ++i) {
    double bi = b[i];
    if (i == n - 1) bi -= c[n - 1] * corner;
    const double m = bi - a[i] * cp[i - 1];
    r = 1.0 / m;
    cp[i] = c[i] * r;
    const double ui = (i == n - 1) ? c[n - 1] : 0.0;
    y[i] = (d[i] - a[i] * y[i - 1]) * r;
    z[i] = (ui - a[i] * z[i - 1]) * r;
  }
  for (int64_t i = n - 2; i >= 0; --i) {
    y[i] -= cp[i] * y[i + 1];
    z[i] -= cp[i] * z[i + 1];
  }
  const double vy = y[0] + corner * y[n - 1];
  const double vz = z[0] + corner * z[n - 1];
  const double f = vy / (1.0 + vz);
  for (int64_t i = 0; i < n; ++i) x[i] = y[i] - f * z[i];
}

// Mass-matrix solve M dA = rhs on one CTA.
// n <= 2: dense; n < 64: sequential; otherwise a partition method: P blocks
// of contiguous rows, each thread eliminates its block with three
// right-hand sides (rhs, the coupling to the previous block's last unknown,
// the coupling to the next block's first unknown); the 2P interface
// unknowns satisfy a cyclic tridiagonal system (after the row combinations
// that eliminate the outer coupling of each block's first / last equation)
// solved by one thread; the blocks then reconstruct their interiors.
struct SolveWs {
  double *y, *v, *w, *cp;      // [n]
  double *ra, *rb, *rc, *rd;   // [2P]
  double *rz, *rcp, *ry, *rzz; // [2P]
};

// block t of P (rows r0 .. r1-1): forward elimination of the local
// tridiagonal system (no outer couplings) with three right-hand sides, back
// substitution, and the block's two interface rows
__device__ __forceinline__ void block_eliminate(int64_t n, const double* __restrict__ a,
                                                const double* __restrict__ b,
                                                const double* __restrict__ c,
                                                const double* __restrict__ d, const SolveWs& ws,
                                                int P, int t) {
  const int64_t r0 = (int64_t)t * n / P, r1 = (int64_t)(t + 1) * n / P;
  double r = 1.0 / b[r0];
  ws.cp[r0] = c[r0] * r;
  ws.y[r0] = d[r0] * r;
  ws.v[r0] = a[r0] * r;
  ws.w[r0] = (r1 - 1 == r0) ? c[r0] * r : 0.0;
  for (int64_t i = r0 + 1; i < r1; ++i) {
    const double m = b[i] - a[i] * ws.cp[i - 1];
    r = 1.0 / m;
    ws.cp[i] = c[i] * r;
    ws.y[i] = (d[i] - a[i] * ws.y[i - 1]) * r;
    ws.v[i] = (-a[i] * ws.v[i - 1]) * r;
    ws.w[i] = ((i == r1 - 1 ? c[i] : 0.0) - a[i] * ws.w[i - 1]) * r;
  }
  for (int64_t i = r1 - 2; i >= r0; --i) {
    ws.y[i] -= ws.cp[i] * ws.y[i + 1];
    ws.v[i] -= ws.cp[i] * ws.v[i + 1];
    ws.w[i] -= ws.cp[i] * ws.w[i + 1];
  }
  const double yF = ws.y[r0], vF = ws.v[r0], wF = ws.w[r0];
  const double yL = ws.y[r1 - 1], vL = ws.v[r1 - 1], wL = ws.w[r1 - 1];
  // interface rows: 2t (eliminates X_{t+1}^F), 2t+1 (eliminates X_{t-1}^L)
  ws.ra[2 * t] = wL * vF - wF * vL;
  ws.rb[2 * t] = wL;
  ws.rc[2 * t] = -wF;
  ws.rd[2 * t] = wL * yF - wF * yL;
  ws.ra[2 * t + 1] = vL;
  ws.rb[2 * t + 1] = -vF;
  ws.rc[2 * t + 1] = vL * wF - vF * wL;
  ws.rd[2 * t + 1] = vL * yF - vF * yL;
}

// block t's interior from the interface solution ws.rz
__device__ __forceinline__ void block_reconstruct(int64_t n, const SolveWs& ws, int P, int t,
                                                  double* x) {
  const int64_t r0 = (int64_t)t * n / P, r1 = (int64_t)(t + 1) * n / P;
  const double Xl = ws.rz[(2 * t - 1 + 2 * P) % (2 * P)];  // last unknown of block t-1
  const double Xf = ws.rz[(2 * t + 2) % (2 * P)];          // first unknown of block t+1
  for (int64_t i = r0; i < r1; ++i) x[i] = ws.y[i] - ws.v[i] * Xl - ws.w[i] * Xf;
}

__global__ void __launch_bounds__(1024) mass_solve_kernel(int64_t n, const double* a,
                                                          const double* b, const double* c,
                                                          const double* d, double* x, SolveWs ws,
                                                          int P) {
  const int t = threadIdx.x;
  if (n <= 2) {
    if (t == 0) {
      if (n == 1) {
        x[0] = d[0] / (a[0] + b[0] + c[0]);
      } else {
        // rows: b0 x0 + (a0 + c0) x1 = d0 ; (a1 + c1) x0 + b1 x1 = d1
        const double m00 = b[0], m01 = a[0] + c[0], m10 = a[1] + c[1], m11 = b[1];
        const double det = m00 * m11 - m01 * m10;
        x[0] = (d[0] * m11 - m01 * d[1]) / det;
        x[1] = (m00 * d[1] - m10 * d[0]) / det;
      }
    }
    return;
  }
  if (n < 64 || P < 2) {
    if (t == 0) cyclic_thomas_seq(n, a, b, c, d, x, ws.cp, ws.y, ws.v);
    return;
  }
  if (t < P) block_eliminate(n, a, b, c, d, ws, P, t);
  __syncthreads();
  if (t == 0) cyclic_thomas_seq(2 * P, ws.ra, ws.rb, ws.rc, ws.rd, ws.rz, ws.rcp, ws.ry, ws.rzz);
  __syncthreads();
  if (t < P) block_reconstruct(n, ws, P, t, x);
}

// The same partition method across the GPU for large meshes: the blocks
// are eliminated by one thread each over many CTAs (the FP64 work of a
// large mesh would otherwise run at one SM's FP64 rate), the 2P interface
// unknowns are solved by mass_solve_kernel, and the blocks reconstructed.
__global__ void mm_eliminate_kernel(int64_t n, const double* a, const double* b, const double* c,
                                    const double* d, SolveWs ws, int P) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < P) block_eliminate(n, a, b, c, d, ws, P, t);
}
__global__ void mm_reconstruct_kernel(int64_t n, SolveWs ws, int P, double* x) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < P) block_reconstruct(n, ws, P, t, x);
}

// After the mass-matrix solve, one thread per cell: the Lemons projection
// coefficients (proj_coeffs) from the cell's velocity sums and dA, and the
// cell's status.  For one component also cv = u + a (dz + beta), so that
// the particle pass writes v = cv + a f.
template <int D>
struct RecCoef {
  double a, beta[D], alpha_new, cv[D];
  int skip;
  int pad;
};
template <int D>
__global__ void recon_coeffs_kernel(int64_t C, int Kmax, const RecHead<D>* head,
                                    const RecComp<D>* comp, const double* raw,
                                    const int64_t* out_off, int64_t n_out, const double* W,
                                    const double* dA, RecCoef<D>* coef, uint32_t* status_out) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < C;
       j += (int64_t)gridDim.x * blockDim.x) {
    int64_t o, n;
    const bool in_range = out_range(out_off, j, n_out, o, n);
    const RecHead<D> h = head[j];
    const RecComp<D>& c0 = comp[(size_t)j * Kmax];
    double sw[D + 1];
    velocity_sums<D>(raw + (size_t)j * raw_words<D>(), fixed_sums(h.K, n), h.K, c0, n, sw);
    const ProjCoef<D> pc = proj_coeffs<D>(h.K, h.u, h.theta, n, W[j], dA[j], sw);
    RecCoef<D> cf;
    cf.a = pc.a;
    cf.alpha_new = pc.alpha_new;
    cf.skip = pc.skip;
    cf.pad = 0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      cf.beta[d] = pc.beta[d];
      // one component: v = u + a (dz + f + beta) = cv + a f (a = 1, beta = 0
      // when skipped)
      cf.cv[d] = h.K == 1 ? fma(pc.a, c0.dz[d] + pc.beta[d], h.u[d]) : 0.0;
    }
    coef[j] = cf;
    status_out[j] = pc.status | (in_range ? 0u : GM_ST_BAD_RANGE);
  }
}

// Pass 2, one warp per cell: the final particles (positions, projected
// velocities, corrected weights) from the draws that pass 1 staged.
template <int D, int NW>
__global__ void __launch_bounds__(NW * 32) recon_emit_kernel(
    int64_t C, int Kmax, const RecHead<D>* head, const RecComp<D>* comp, const RecCoef<D>* coef,
    const int64_t* out_off, double dx, int64_t n_out, double* x_out, double* v_out,
    double* alpha_out) {
  __shared__ RecCell<D> rcs[NW];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  RecCell<D>& rc = rcs[wid];
  for (int64_t j = (int64_t)blockIdx.x * NW + wid; j < C; j += (int64_t)gridDim.x * NW) {
    load_prepped<D>(rc, j, Kmax, head, comp, lane);
    const RecCoef<D> cf = coef[j];
    __syncwarp();
    int64_t o, n;
    out_range(out_off, j, n_out, o, n);
    const double aa = cf.a, an = cf.alpha_new;
    if (rc.K == 1) {
      // four particles per lane per step: their staged draws are all loaded
      // before any of their slots is overwritten, so the loads of a step
      // are in flight together
      constexpr int U = 4;
      int64_t i = lane;
      for (; i + 32 * (U - 1) < n; i += 32 * U) {
        uint64_t m0[U];
        int z[U];
        float f[U][D];
#pragma unroll
        for (int u = 0; u < U; ++u) load_draw<D>(x_out, v_out, alpha_out, o + i + 32 * u, m0[u], z[u], f[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t p = o + i + 32 * u;
          x_out[p] = __dmul_rn(cell_plus_u0((uint64_t)j, m0[u]), dx);
          alpha_out[p] = an;
#pragma unroll
          for (int d = 0; d < D; ++d) v_out[(int64_t)d * n_out + p] = fma(aa, f2d_exact(f[u][d]), cf.cv[d]);
        }
      }
      for (; i < n; i += 32) {
        uint64_t m0;
        int z;
        float f[D];
        load_draw<D>(x_out, v_out, alpha_out, o + i, m0, z, f);
        x_out[o + i] = __dmul_rn(cell_plus_u0((uint64_t)j, m0), dx);
        alpha_out[o + i] = an;
#pragma unroll
        for (int d = 0; d < D; ++d) v_out[(int64_t)d * n_out + o + i] = fma(aa, f2d_exact(f[d]), cf.cv[d]);
      }
    } else {
      for (int64_t i = lane; i < n; i += 32) {
        uint64_t m0;
        int z;
        float f[D];
        double w[D];
        load_draw<D>(x_out, v_out, alpha_out, o + i, m0, z, f);
        draw_offset<D>(rc, z, f, w);
        x_out[o + i] = __dmul_rn(cell_plus_u0((uint64_t)j, m0), dx);
        alpha_out[o + i] = an;
#pragma unroll
        for (int d = 0; d < D; ++d) {
          // v = u + w; projected: u + a (w + beta) (eqs. alpha, beta)
          const double vp = cf.skip ? rc.u[d] + w[d] : fma(aa, w[d] + cf.beta[d], rc.u[d]);
          v_out[(int64_t)d * n_out + o + i] = vp;
        }
      }
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
int solve_blocks(int64_t C) {
  if (C < 64) return 1;
  int P = (int)sqrt((double)C / 2.0);
  if (P > 1024) P = 1024;
  if (P < 2) P = 2;
  return P;
}

// Mass-matrix solve plan.  A mesh below kMultiRows cells is solved on one
// CTA (mass_solve_kernel, solve_blocks(n) blocks).  A larger one by the same
// partition method applied level by level across the GPU: level l splits
// its n_l rows into P_l blocks of about kLevelRows rows, one thread each
// (mm_eliminate_kernel), and the blocks' 2 P_l interface rows are level
// l + 1's cyclic tridiagonal system; the first level below kMultiRows rows
// goes to one CTA, and the levels are then reconstructed in reverse order
// (mm_reconstruct_kernel).  Short blocks keep each thread's sequential
// FP64 elimination short; 262144 cells take three levels (16384, 2048 and
// 256 blocks) and a 512-row system on one CTA.
constexpr int64_t kMultiRows = 2048;
constexpr int64_t kLevelRows = 16;
constexpr int kMaxLevels = 12;
struct SolvePlan {
  int L;                      // multi-CTA levels (0: the whole system on one CTA)
  int64_t n[kMaxLevels + 1];  // rows of level l; n[L] the one-CTA system
  int P[kMaxLevels];          // blocks of the multi-CTA levels
  int Pf;                     // blocks of the one-CTA system
};
static SolvePlan plan_solve(int64_t C) {
  SolvePlan pl;
  pl.L = 0;
  pl.n[0] = C;
  while (pl.n[pl.L] >= kMultiRows && pl.L < kMaxLevels) {
    pl.P[pl.L] = (int)(pl.n[pl.L] / kLevelRows);
    pl.n[pl.L + 1] = 2 * (int64_t)pl.P[pl.L];
    ++pl.L;
  }
  pl.Pf = solve_blocks(pl.n[pl.L]);
  return pl;
}
// doubles of one level's SolveWs: y, v, w, cp over its n rows and the eight
// interface arrays over 2 P + 2
static size_t level_doubles(int64_t n, int P) { return 4 * (size_t)n + 8 * (size_t)(2 * (int64_t)P + 2); }
static SolveWs level_ws(double* base, int64_t n, int P) {
  SolveWs w;
  w.y = base; w.v = base + n; w.w = base + 2 * n; w.cp = base + 3 * n;
  double* r = base + 4 * n;
  const int64_t R2 = 2 * (int64_t)P + 2;
  w.ra = r; w.rb = r + R2; w.rc = r + 2 * R2; w.rd = r + 3 * R2;
  w.rz = r + 4 * R2; w.rcp = r + 5 * R2; w.ry = r + 6 * R2; w.rzz = r + 7 * R2;
  return w;
}
static size_t solve_doubles(const SolvePlan& pl) {
  size_t d = 0;
  for (int l = 0; l < pl.L; ++l) d += level_doubles(pl.n[l], pl.P[l]);
  return d + level_doubles(pl.n[pl.L], pl.Pf);
}

// workspace: the raw sums, the mixture heads and component records, the
// projection coefficients, then the FP64 arrays of the mass-matrix solve
static size_t rec_bytes(int D, int64_t C, int Kmax, size_t* off_head, size_t* off_coef,
                        size_t* off_comp) {
  const size_t raw = (size_t)C * (D == 1 ? raw_words<1>() : raw_words<3>()) * sizeof(double);
  const size_t hd = (size_t)C * (D == 1 ? sizeof(RecHead<1>) : sizeof(RecHead<3>));
  const size_t cf = (size_t)C * (D == 1 ? sizeof(RecCoef<1>) : sizeof(RecCoef<3>));
  const size_t cp = (size_t)C * Kmax * (D == 1 ? sizeof(RecComp<1>) : sizeof(RecComp<3>));
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  if (off_head) *off_head = up(raw);
  if (off_coef) *off_coef = up(raw) + up(hd);
  if (off_comp) *off_comp = up(raw) + up(hd) + up(cf);
  return up(raw) + up(hd) + up(cf) + up(cp);
}

size_t reconstruct_ws_bytes(int D, int64_t C, int Kmax) {
  const SolvePlan pl = plan_solve(C);
  const size_t dbl = 5 * (size_t)C /*a b c d, dA*/ + solve_doubles(pl);
  return rec_bytes(D, C, Kmax, nullptr, nullptr, nullptr) + dbl * sizeof(double) + 1024;
}

template <int D>
static void launch_passes(int64_t C, int Kmax, const int32_t* K, const double* prm, const double* W,
                          const double* rho_target, int64_t n_out, const int64_t* out_off,
                          uint64_t seed, double dx, double q, int order, double* x_out,
                          double* v_out, double* alpha_out, uint32_t* status_out, double* dA,
                          unsigned char* recs, double* A, double* B, double* Cc, double* Dd,
                          const SolvePlan& pl, const SolveWs* lws, cudaStream_t s) {
  size_t oh, oc, op;
  rec_bytes(D, C, Kmax, &oh, &oc, &op);
  double* raw = (double*)recs;
  RecHead<D>* head = (RecHead<D>*)(recs + oh);
  RecCoef<D>* coef = (RecCoef<D>*)(recs + oc);
  RecComp<D>* comp = (RecComp<D>*)(recs + op);
  trace_mark(nullptr, s);
  const int ga = (int)((C + 255) / 256 < 4096 ? (C + 255) / 256 : 4096);
  recon_prep_kernel<D><<<ga, 256, 0, s>>>(C, Kmax, K, prm, head, comp);
  trace_mark("recon_prep_kernel", s);
  // one warp per cell, 4 cells per CTA, at most 16 CTAs per SM resident
  constexpr int NW = 4;
  const int64_t ncta = (C + NW - 1) / NW;
  const int g = (int)(ncta < 152 * 16 ? ncta : 152 * 16);
  recon_stats_kernel<D, NW><<<g, NW * 32, 0, s>>>(C, Kmax, head, comp, out_off, n_out, seed, order,
                                                  raw, x_out, v_out, alpha_out);
  trace_mark("recon_stats_kernel", s);
  assemble_kernel<D><<<ga, 256, 0, s>>>(C, head, raw, W, out_off, n_out, rho_target, dx, q, order,
                                        A, B, Cc, Dd);
  trace_mark("assemble_kernel", s);
  {
    // level l's system: (A, B, Cc, Dd) for l = 0, else level l - 1's
    // interface rows; its solution: dA for l = 0, else level l - 1's rz
    const double *sa = A, *sb = B, *sc = Cc, *sd = Dd;
    for (int l = 0; l < pl.L; ++l) {
      // 32-thread CTAs spread a level's blocks over the SMs (each thread's
      // elimination is a latency-bound FP64 chain)
      mm_eliminate_kernel<<<(pl.P[l] + 31) / 32, 32, 0, s>>>(pl.n[l], sa, sb, sc, sd, lws[l], pl.P[l]);
      sa = lws[l].ra; sb = lws[l].rb; sc = lws[l].rc; sd = lws[l].rd;
    }
    const int Pf = pl.Pf;
    double* xf = pl.L > 0 ? lws[pl.L - 1].rz : dA;
    mass_solve_kernel<<<1, Pf < 32 ? 32 : ((Pf + 31) / 32) * 32, 0, s>>>(pl.n[pl.L], sa, sb, sc, sd, xf,
                                                                         lws[pl.L], Pf);
    for (int l = pl.L - 1; l >= 0; --l)
      mm_reconstruct_kernel<<<(pl.P[l] + 31) / 32, 32, 0, s>>>(pl.n[l], lws[l], pl.P[l],
                                                                  l > 0 ? lws[l - 1].rz : dA);
  }
  trace_mark("mass-matrix solve (mass_solve_kernel and the blocked kernels)", s);
  recon_coeffs_kernel<D><<<ga, 256, 0, s>>>(C, Kmax, head, comp, raw, out_off, n_out, W, dA, coef,
                                            status_out);
  trace_mark("recon_coeffs_kernel", s);
  recon_emit_kernel<D, NW><<<g, NW * 32, 0, s>>>(C, Kmax, head, comp, coef, out_off, dx, n_out,
                                                 x_out, v_out, alpha_out);
  trace_mark("recon_emit_kernel", s);
}

cudaError_t launch_reconstruct(int D, int64_t C, int Kmax, const int32_t* K, const double* prm,
                               const double* W, const double* rho_target, int64_t n_out,
                               const int64_t* out_off, uint64_t seed, double dx, double q,
                               int order, double* x_out, double* v_out, double* alpha_out,
                               uint32_t* status_out, double* dA_user, void* ws, cudaStream_t s) {
  if (C == 0) return cudaSuccess;
  const SolvePlan pl = plan_solve(C);
  unsigned char* recs = (unsigned char*)ws;
  double* A = (double*)(recs + rec_bytes(D, C, Kmax, nullptr, nullptr, nullptr));
  double* B = A + C;
  double* Cc = B + C;
  double* Dd = Cc + C;
  double* dA = Dd + C;
  SolveWs lws[kMaxLevels + 1];
  double* base = dA + C;
  for (int l = 0; l < pl.L; ++l) {
    lws[l] = level_ws(base, pl.n[l], pl.P[l]);
    base += level_doubles(pl.n[l], pl.P[l]);
  }
  lws[pl.L] = level_ws(base, pl.n[pl.L], pl.Pf);
  if (dA_user) dA = dA_user;
  if (D == 1)
    launch_passes<1>(C, Kmax, K, prm, W, rho_target, n_out, out_off, seed, dx, q, order, x_out,
                     v_out, alpha_out, status_out, dA, recs, A, B, Cc, Dd, pl, lws, s);
  else
    launch_passes<3>(C, Kmax, K, prm, W, rho_target, n_out, out_off, seed, dx, q, order, x_out,
                     v_out, alpha_out, status_out, dA, recs, A, B, Cc, Dd, pl, lws, s);
  return cudaGetLastError();
}

}  // namespace gmcr
