// gm_common.cuh -- shared device helpers of the GB300 GM checkpoint-restart
// kernels: the Philox4x32-10 generator, the 52-bit uniform map, warp
// reductions and the per-cell status bits.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gm.h"

namespace gmcr {

constexpr int kMaxK = 16;
constexpr int kWarp = 32;

__host__ __device__ constexpr int T_of(int D) { return D * (D + 3) / 2; }         // App. A
__host__ __device__ constexpr int P_of(int D) { return 1 + D + D * (D + 1) / 2; }  // record size
__host__ __device__ constexpr int NM_of(int D) { return D * (D + 1) / 2; }         // covariance entries

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds, each two
// 32x32 -> 64-bit products of counter words with the round multipliers,
// an xor/permute with the key, and the key advanced by the Weyl increments
// between rounds.
struct u32x4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = u32x4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// uniform in (0,1): the 52 leading bits m of (hi, lo), u = (m + 1/2) 2^-52
__device__ __forceinline__ double uniform52(uint32_t hi, uint32_t lo) {
  const uint64_t m = ((uint64_t)hi << 20) | (uint64_t)(lo >> 12);
  return __dmul_rn(__dadd_rn((double)m, 0.5), 2.220446049250313080847263336181640625e-16);
}

constexpr uint32_t kTagInit = 0x494E4954u;
constexpr uint32_t kTagSample = 0x53000000u;

__device__ __forceinline__ u32x4 philox_draw(uint64_t seed, uint32_t c0, uint32_t c1, int64_t cell) {
  return philox4x32_10(u32x4{c0, c1, (uint32_t)((uint64_t)cell), (uint32_t)((uint64_t)cell >> 32)},
                       (uint32_t)seed, (uint32_t)(seed >> 32));
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Conversions on the integer pipe.  GB300's FP64 pipe runs at 1/64 of the
// FP32 rate and a conversion to or from FP64 occupies it like an FP64
// operation; these build the result from the bit patterns with integer
// operations and selects only (no hardware conversion on any path).
// f2d_exact: FP32 -> FP64, exact for every finite input (normal, subnormal,
// signed zero); infinities map to infinities, a NaN to a quiet NaN.
__device__ __forceinline__ double f2d_exact(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  const unsigned long long sgn = (unsigned long long)(u >> 31) << 63;
  // normal: rebias the exponent, widen the mantissa
  unsigned long long r = sgn | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)m << 29);
  // subnormal m 2^-149 (m != 0): leading bit b of m, value 2^(b - 149) (m / 2^b)
  const int b = 31 - __clz((int)m);
  const unsigned long long rs = sgn | ((unsigned long long)(b + 874) << 52) |
                                (((unsigned long long)m << (52 - b)) & ((1ull << 52) - 1ull));
  // infinity / NaN (the quiet bit set)
  const unsigned long long ri = sgn | (0x7FFull << 52) | ((unsigned long long)m << 29) |
                                (m ? (1ull << 51) : 0ull);
  r = e == 0xFFu ? ri : r;
  r = e == 0u ? (m ? rs : sgn) : r;
  return __longlong_as_double((long long)r);
}
template <typename VT>
__device__ __forceinline__ double to_f64(VT v) {
  if constexpr (sizeof(VT) == 4) return f2d_exact(v);
  else return (double)v;
}
// d2f_trunc: FP64 -> FP32 with the mantissa truncated (toward zero,
// relative error below 2^-23 in FP32's normal range); below it the value
// truncates to an FP32 subnormal or a signed zero, from 2^128 up (and
// infinities) to a signed infinity, a NaN to a quiet NaN
__device__ __forceinline__ float d2f_trunc(double d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const uint32_t sgn = (uint32_t)(u >> 32) & 0x80000000u;
  const int ed = (int)((u >> 52) & 0x7FFull);
  const int e = ed - 896;
  const unsigned long long mant = u & ((1ull << 52) - 1ull);
  uint32_t r = sgn | ((uint32_t)(e > 0 ? e : 0) << 23) | (uint32_t)(mant >> 29);
  // below the normal range: |d| = (2^52 + mant) 2^(ed - 1075), as a multiple
  // of 2^-149 truncated (zero for ed <= 873 and for double subnormals)
  const int sh = 926 - ed < 30 ? 30 : 926 - ed;  // 926 - ed >= 30 wherever sub is used
  const uint32_t sub = (ed > 0 && sh < 64) ? (uint32_t)(((1ull << 52) | mant) >> sh) : 0u;
  r = e <= 0 ? (sgn | sub) : r;
  // overflow, infinity, NaN
  const uint32_t big = sgn | 0x7F800000u | ((ed == 0x7FF && mant) ? 0x400000u : 0u);
  r = e >= 255 ? big : r;
  return __uint_as_float(r);
}
// k 2^-53 for an odd integer 1 <= k < 2^53 (exact), negated if neg: the
// double built from k's leading bit position and the bits below it
__device__ __forceinline__ double odd_2m53(unsigned long long k, bool neg) {
  const int b = 63 - __clzll((long long)k);  // leading bit, 0 .. 52
  const unsigned long long mant = (k << (52 - b)) & ((1ull << 52) - 1ull);
  const unsigned long long ex = (unsigned long long)(970 + b) << 52;  // 1023 + b - 53
  return __longlong_as_double((long long)(ex | mant | (neg ? (1ull << 63) : 0ull)));
}

// Fixed-point sums on the integer pipe: a value v is taken as the integer
// round(v / 2^eq), sums of such integers and of their products are exact in
// 128 bits, and one conversion to FP64 per sum replaces a per-element FP64
// accumulation.  kFixBits bounds |v| / 2^eq below 2^kFixBits, kFixMaxN the
// count of summed products (2 kFixBits + 2 + log2 kFixMaxN < 127).
constexpr int kFixBits = 54;
constexpr int kFixMaxN = 1 << 14;

// v / 2^eq rounded to the nearest integer (ties away from zero), from the
// bit pattern of an FP32 v with |v| < 2^(eq + kFixBits)
__device__ __forceinline__ long long fixq(float v, int eq) {
  const uint32_t u = __float_as_uint(v);
  const int eb = (int)((u >> 23) & 0xFFu);
  const long long m = (long long)((u & 0x7FFFFFu) | (eb ? 0x800000u : 0u));
  const int sh = (eb ? eb - 150 : -149) - eq;  // v = m 2^(eb - 150) (subnormal: 2^-149)
  long long r = 0;
  if (sh >= 0) r = m << sh;
  else if (sh > -40) r = (m + (1ll << (-sh - 1))) >> (-sh);
  return (u >> 31) ? -r : r;
}

__device__ __forceinline__ __int128 shfl_xor_i128(__int128 x, int b) {
  const long long lo = __shfl_xor_sync(0xffffffffu, (long long)(unsigned long long)x, b);
  const long long hi = __shfl_xor_sync(0xffffffffu, (long long)(x >> 64), b);
  return ((__int128)hi << 64) | (__int128)(unsigned long long)lo;
}

// a 128-bit integer times 2^e as the nearest-ish double (two roundings)
__device__ __forceinline__ double i128_to_f64(__int128 x, int e) {
  const long long hi = (long long)(x >> 64);
  const unsigned long long lo = (unsigned long long)x;
  return ldexp(fma((double)hi, 18446744073709551616.0, (double)lo), e);
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// hardware base-2 exponential / logarithm (PTX ex2.approx / lg2.approx,
// relative error about 2^-22)
__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Shape-function weights of a particle at fractional cell position
// xi in [0,1) on the nodes j-1, j, j+1 (B-splines of order 1 or 2 centred
// on the nodes at (i + 1/2) dx).
__device__ __forceinline__ void shape3(int order, double xi, double& wm, double& w0, double& wp) {
  const double s = xi - 0.5;
  if (order == 1) {
    wm = s < 0.0 ? -s : 0.0;
    wp = s > 0.0 ? s : 0.0;
    w0 = 1.0 - (s < 0.0 ? -s : s);
  } else {
    const double a = 0.5 - s, b = 0.5 + s;
    wm = 0.5 * a * a;
    wp = 0.5 * b * b;
    w0 = 0.75 - s * s;
  }
}

// fractional position of x inside cell j, clamped to [0, 1): below 0 (and
// -inf) to 0, from 1 up (+inf, NaN) to 1 - 2^-53.  One FP64 operation; the
// clamp compares the bit pattern on the integer pipe (the sign bit, then
// the magnitude against those of 1.0 and of the infinities).
__device__ __forceinline__ double cell_frac(double x, double jd, double inv_dx) {
  const double xi = x * inv_dx - jd;  // jd = (double)j, converted once per cell by the caller
  const long long b = __double_as_longlong(xi);
  const unsigned long long mag = (unsigned long long)b & 0x7FFFFFFFFFFFFFFFull;
  if (mag > 0x7FF0000000000000ull || (b >= 0 && mag >= 0x3FF0000000000000ull)) return 0.99999999999999989;
  return b < 0 ? 0.0 : xi;
}

}  // namespace gmcr

namespace gmcr {

// Two FP32 values in one 64-bit register, operated on by Blackwell's packed
// FP32 instructions (add/mul/fma .f32x2): two particles per instruction.
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pk2(float lo, float hi) {
  f32x2 r;
  asm("mov.b64 %0, {%1,%2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void upk2(f32x2 v, float& lo, float& hi) {
  asm("mov.b64 {%0,%1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 bc2(float x) { return pk2(x, x); }
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
// hardware reciprocal (PTX rcp.approx, relative error about 2^-23)
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// maximum of three (one three-input max instruction on sm_100 and later)
__device__ __forceinline__ float max3f(float a, float b, float c) {
  float y;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(y) : "f"(a), "f"(b), "f"(c));
  return y;
}

}  // namespace gmcr
