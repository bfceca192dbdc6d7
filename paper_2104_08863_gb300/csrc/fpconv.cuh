// FP64 <-> FP32-pair conversions by integer bit manipulation, and double-float (df64)
// arithmetic on FP32 units.
//
// On GB300 an FP64 arithmetic instruction and an F2F conversion both issue at about two per
// clock per SM, against 128 FP32 and 64 integer operations, so the FP32-refined solve keeps the
// per-point work on the FP32 and integer pipes, with at most one FP64 addition per output value:
//  * f64_to_f32_trunc / f64_split: a double's sign, exponent and top 24 significand bits give
//    hi; the remaining 29 bits, converted by I2F and scaled by a power of two built in the
//    exponent field, give lo, so hi + lo equals x to about 2^-47 relative.  Zeros, values below
//    the FP32 normal range (flushed to zero) and values above it (to +-inf) are handled.
//  * f32_to_f64_exact / f32_add_to_f64: an FP32 value widened to FP64 by integer operations
//    (exact), and a + b as one correctly rounded FP64 addition of two such widenings (exact for
//    the two parts of a normalised pair).
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

// Normal range of the fast paths: biased FP64 exponent e with e - 896 a normal FP32 exponent
// (truncation), and in addition e - 948 one (the scale of the split's low part).  There the FP32
// bits are the top 32 bits of u << 3 with the exponent field rebiased by -896 (mod 512, which the
// 9-bit field after the shift absorbs) and the sign put back.
__host__ __device__ __forceinline__ float f64_hi_fast(uint32_t h, uint32_t l) {
  const uint32_t t = ((h << 3) | (l >> 29)) - (384u << 23);
  return float_of((t & 0x7fffffffu) | (h & 0x80000000u));
}

// x truncated toward zero to FP32 (flush below the normal range, +-inf above it).
__host__ __device__ __forceinline__ float f64_to_f32_trunc(double x) {
  const uint64_t u = bits_of(x);
  const uint32_t h = (uint32_t)(u >> 32);
  if (((h >> 20) & 0x7ffu) - 897u <= 1150u - 897u) return f64_hi_fast(h, (uint32_t)u);
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
  const uint64_t u = bits_of(x);
  {
    const uint32_t h = (uint32_t)(u >> 32), l = (uint32_t)u;
    const uint32_t e = (h >> 20) & 0x7ffu;
    if (e - 949u <= 1150u - 949u) {
      hi = f64_hi_fast(h, l);
      const float mag = (float)(l & 0x1fffffffu) * float_of((e - 948u) << 23);
      lo = float_of(bits_of(mag) | (h & 0x80000000u));
      return;
    }
  }
  hi = f64_to_f32_trunc(x);
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

// x widened to FP64 exactly, by integer operations (an F2F conversion would run on the FP64
// pipe): sign, exponent rebiased by +896 (255 -> 2047 for infinities and NaNs), the 23 fraction
// bits at the top of the 52.  FP32 subnormals become zeros of the same sign.
__host__ __device__ __forceinline__ double f32_to_f64_exact(float x) {
  const uint32_t u = bits_of(x);
  const uint32_t e = (u >> 23) & 0xffu;
  const uint32_t sign = u & 0x80000000u;
  if (e == 0u) return double_of((uint64_t)sign << 32);
  const uint32_t ee = e == 0xffu ? 0x7ffu : e + 896u;
  const uint32_t h = sign | (ee << 20) | ((u >> 3) & 0xfffffu);
  return double_of(((uint64_t)h << 32) | (uint64_t)(u << 29));
}

// a + b as a double: one correctly rounded FP64 addition of the exact widenings, the only FP64
// instruction of the conversion.  Exact when b lies within 29 bits below a, as the low part of a
// normalised pair does.
__host__ __device__ __forceinline__ double f32_add_to_f64(float a, float b) {
  return f32_to_f64_exact(a) + f32_to_f64_exact(b);
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
