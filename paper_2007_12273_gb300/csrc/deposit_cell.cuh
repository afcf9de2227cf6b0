// deposit_cell.cuh -- one cell's charge-deposit sums (Sec. 2.4.1), computed
// by one warp: the record that deposit_combine_kernel turns into rho.  Used
// by the deposit kernel and, fused with the closed-form pre-pass of
// gm_compress_from, by em_k1_kernel (both read the cell's weights).
//
// Per cell, the partial deposits on nodes j-1, j, j+1 follow from
// A0 = sum alpha, A1 = sum alpha s, A2 = sum alpha s^2 (quadratic
// B-spline) or the CIC parts sum alpha max(-s, 0), sum alpha max(s, 0),
// with s = xi - 1/2 the particle's offset from the cell centre.  Record of
// kDepWords 64-bit words:
//   equal weights: [k0 (low, high), k1 (low, high), alpha bits, n], the
//     exact 128-bit sums of k and k^2 (or of the CIC parts) with
//     s = k 2^-53;
//   otherwise: [A0, A1, A2 (FP64 bits), -, -, -1].
#pragma once

#include "gm_common.cuh"

namespace gmcr {

constexpr int kDepWords = 6;

// the weights of a cell's n particles equal bit for bit (every lane gets the
// answer; alpha = NULL means unit weights)
__device__ __forceinline__ bool equal_weights(const double* alpha, int64_t o, int64_t n, int lane) {
  if (!alpha) return true;
  const long long wb = __double_as_longlong(alpha[o]);
  bool same = true;
#pragma unroll 4
  for (int64_t p = lane; p < n; p += 32) same &= (__double_as_longlong(alpha[o + p]) == wb);
  return __all_sync(0xffffffffu, same);
}

// cell j's record r; same = equal_weights(...) for 0 < n <= kFixMaxN
__device__ __forceinline__ void deposit_cell(int64_t j, int64_t o, int64_t n, const double* x,
                                             const double* alpha, double inv_dx, int order,
                                             long long* r, int lane, bool same) {
  const double jd = (double)j;
  // equal weights (bit for bit) and at most 2^14 particles: the sums of s
  // and s^2 (or of the CIC parts) exactly on the integer pipe, s = k 2^-53
  // with k = round(xi 2^53) - 2^52 from the bits of the FP64 in-cell
  // position xi in [0, 1); the weight multiplies the sums once
  if (n > 0 && n <= kFixMaxN && same) {
    const long long wb = alpha ? __double_as_longlong(alpha[o]) : __double_as_longlong(1.0);
    // a lane sums at most kFixMaxN / 32 = 512 values of |k| <= 2^52: the
    // linear sum fits in 64 bits, the squares take 128
    long long k0l = 0;
    __int128 k1 = 0;
#pragma unroll 2
    for (int64_t p = lane; p < n; p += 32) {
      const double xi = cell_frac(x[o + p], jd, inv_dx);
      // xi = m 2^(e - 1075) (m with its implicit bit), k = round(xi 2^53) - 2^52
      const unsigned long long u = (unsigned long long)__double_as_longlong(xi);
      const int e = (int)((u >> 52) & 0x7FFull);
      const long long m = (long long)((u & ((1ull << 52) - 1ull)) | (e ? (1ull << 52) : 0ull));
      const int sh = (e ? e : 1) - 1022;  // xi 2^53 = m 2^sh, sh <= 0
      long long rr = 0;
      if (sh == 0) rr = m;
      else if (sh > -60) rr = (m + (1ll << (-sh - 1))) >> (-sh);
      const long long k = rr - (1ll << 52);
      if (order == 1) {
        k0l += k < 0 ? -k : 0;
        k1 += (__int128)(k > 0 ? k : 0);
      } else {
        k0l += k;
        k1 += (__int128)k * (__int128)k;
      }
    }
    __int128 k0 = (__int128)k0l;
#pragma unroll
    for (int q = 16; q > 0; q >>= 1) {
      k0 += shfl_xor_i128(k0, q);
      k1 += shfl_xor_i128(k1, q);
    }
    // lanes 0-5 write the record's words
    long long wv = (long long)(unsigned long long)k0;
    wv = lane == 1 ? (long long)(k0 >> 64) : wv;
    wv = lane == 2 ? (long long)(unsigned long long)k1 : wv;
    wv = lane == 3 ? (long long)(k1 >> 64) : wv;
    wv = lane == 4 ? wb : wv;
    wv = lane == 5 ? (long long)n : wv;
    if (lane < kDepWords) r[lane] = wv;
    return;
  }
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (int64_t p = lane; p < n; p += 32) {
    const double sx = cell_frac(x[o + p], jd, inv_dx) - 0.5;
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
  long long wv = __double_as_longlong(a0);
  wv = lane == 1 ? __double_as_longlong(a1) : wv;
  wv = lane == 2 ? __double_as_longlong(a2) : wv;
  wv = lane == 5 ? -1ll : wv;
  if (lane < kDepWords) r[lane] = wv;
}

}  // namespace gmcr
