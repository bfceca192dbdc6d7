// FP64 <-> FP32-pair conversions by integer bit manipulation, and double-float (df64)
// arithmetic on FP32 units.
//
// On GB300 an FP64 arithmetic instruction and an F2F conversion both issue at about two per
// clock per SM, against 128 FP32 and 64 integer operations, so the FP32-refined solve keeps
// every per-point operation off the FP64 pipe:
//  * f64_to_f32_trunc / f64_split: a double's sign, exponent and top 24 significand bits give
//    hi; the remaining 29 bits, converted by I2F and scaled by a power of two built in the
//    exponent field, give lo, so hi + lo equals x to about 2^-47 relative.  Zeros, values below
//    the FP32 normal range (flushed to zero) and values above it (to +-inf) are handled.
//  * f32_pair_to_f64: a + b as a double, computed exactly in a 64-bit integer (the two
//    significands aligned to the larger exponent) and rounded once to 53 bits.
//  * two_sum / two_diff (Knuth), two_prod (by FMA), df_add, df_mul: the classical
//    double-float algorithms (Dekker 1971, Knuth TAOCP vol. 2), accurate to about 2^-47.
// Everything is __host__ __device__ so that the host test suite can check it bit for bit.
#pragma once

#include <math.h>
#include <stdint.h>
#include <string.h>

#ifndef __CUDACC__
#define __host__
#define __device__
#define __forceinline__ inline
#endif

namespace pp {

__host__ __device__ __forceinline__ uint64_t bits_of(double x) {
  uint64_t u;
  memcpy(&u, &x, 8);
  return u;
}
__host__ __device__ __forceinline__ double double_of(uint64_t u) {
  double x;
  memcpy(&x, &u, 8);
  return x;
}
__host__ __device__ __forceinline__ uint32_t bits_of(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  return u;
}
__host__ __device__ __forceinline__ float float_of(uint32_t u) {
  float x;
  memcpy(&x, &u, 4);
  return x;
}
__host__ __device__ __forceinline__ int clz64(uint64_t u) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)u);
#else
  return u ? __builtin_clzll(u) : 64;
#endif
}

// x truncated toward zero to FP32 (flush below the normal range, +-inf above it).
__host__ __device__ __forceinline__ float f64_to_f32_trunc(double x) {
  const uint64_t u = bits_of(x);
  const uint32_t sign = (uint32_t)(u >> 63) << 31;
  const int e = (int)((u >> 52) & 0x7ff);
  if (e == 0x7ff) return float_of(sign | 0x7f800000u | ((u & 0xfffffffffffffull) ? 0x400000u : 0u));
  const int fe = e - 1023 + 127;
  if (fe <= 0) return float_of(sign);
  if (fe >= 255) return float_of(sign | 0x7f800000u);
  return float_of(sign | ((uint32_t)fe << 23) | (uint32_t)((u >> 29) & 0x7fffffu));
}

// hi = f64_to_f32_trunc(x), lo ~= x - hi (the remaining 29 significand bits, rounded to 24).
__host__ __device__ __forceinline__ void f64_split(double x, float& hi, float& lo) {
  hi = f64_to_f32_trunc(x);
  const uint64_t u = bits_of(x);
  const int e = (int)((u >> 52) & 0x7ff);
  const int se = e - 1075 + 127;   // exponent of one unit of the remainder
  const int fe = e - 1023 + 127;
  if (fe <= 0 || fe >= 255 || se <= 0) {
    lo = 0.0f;
    return;
  }
  const uint32_t rem = (uint32_t)(u & 0x1fffffffull);   // low 29 bits
  const float mag = (float)rem * float_of((uint32_t)se << 23);
  lo = (u >> 63) ? -mag : mag;
}

// a + b as a double, exact up to one final rounding to 53 bits (round half up on the
// magnitude).  FP32 subnormals are treated as zero.
__host__ __device__ __forceinline__ double f32_pair_to_f64(float a, float b) {
  const uint32_t ua = bits_of(a), ub = bits_of(b);
  const int ea = (int)((ua >> 23) & 0xff), eb = (int)((ub >> 23) & 0xff);
  const bool za = ea == 0, zb = eb == 0;
  if (za && zb) return 0.0;
  if (zb || za) {   // one term is zero: widen the other exactly
    const uint32_t v = zb ? ua : ub;
    const int ev = zb ? ea : eb;
    const uint64_t s = (uint64_t)(v >> 31) << 63;
    return double_of(s | ((uint64_t)(ev + 896) << 52) | ((uint64_t)(v & 0x7fffffu) << 29));
  }
  const int E = ea > eb ? ea : eb;
  // significands (with the implicit bit) in fixed point: leading bit of the larger at bit 61
  const int sha = 38 - (E - ea), shb = 38 - (E - eb);
  int64_t A = sha >= 0 ? (int64_t)((uint64_t)((ua & 0x7fffffu) | 0x800000u) << sha) : 0;
  int64_t B = 0;
  if (shb >= 0) B = (int64_t)((uint64_t)((ub & 0x7fffffu) | 0x800000u) << shb);
  else if (shb > -24) B = (int64_t)(((ub & 0x7fffffu) | 0x800000u) >> (-shb));
  if (ua >> 31) A = -A;
  if (ub >> 31) B = -B;
  const int64_t S = A + B;
  if (S == 0) return 0.0;
  const uint64_t sign = S < 0 ? (1ull << 63) : 0ull;
  uint64_t U = S < 0 ? (uint64_t)(-S) : (uint64_t)S;
  const int lz = clz64(U);
  U <<= lz;   // leading one at bit 63;  |a + b| = U * 2^(E - 188 - lz)
  const uint64_t frac = (U >> 11) & 0xfffffffffffffull;
  const uint64_t round = (U >> 10) & 1ull;
  const int64_t dexp = (int64_t)E + 898 - lz;   // biased FP64 exponent of the leading one
  if (dexp <= 0) return double_of(sign);
  const uint64_t mag = ((uint64_t)dexp << 52) + frac + round;   // a carry rolls into the exponent
  return double_of(sign | mag);
}

// ---- double-float arithmetic (value = hi + lo) ----------------------------------------------
struct df { float hi, lo; };

__host__ __device__ __forceinline__ df two_sum_df(float a, float b) {
  const float s = a + b;
  const float bp = s - a;
  return df{s, (a - (s - bp)) + (b - bp)};
}
__host__ __device__ __forceinline__ df two_diff_df(float a, float b) {
  const float s = a - b;
  const float bp = s - a;
  return df{s, (a - (s - bp)) - (b + bp)};
}
__host__ __device__ __forceinline__ df quick_two_sum_df(float a, float b) {
  const float s = a + b;
  return df{s, b - (s - a)};
}
__host__ __device__ __forceinline__ df df_add(df a, df b) {
  const df s = two_sum_df(a.hi, b.hi);
  return quick_two_sum_df(s.hi, s.lo + (a.lo + b.lo));
}
__host__ __device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }
// a * b with the rounding error of hi * hi recovered by an FMA; the lo * lo term is dropped.
__host__ __device__ __forceinline__ df df_mul(df a, df b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df{p, e};
}

}  // namespace pp
