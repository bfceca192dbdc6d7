// Double-float arithmetic in packed FP32x2 operations: each instruction performs the same
// correctly rounded operation on both lanes, so the algorithms (TwoSum, TwoDiff, the FMA split of
// a product, compensated sums) run on two independent values at half the issued instructions,
// giving lane by lane the results of the scalar forms in fpconv.cuh.  The *_rn
// intrinsics are never fused into FMAs by the compiler, which the error-free transformations rely
// on.
#pragma once

#include <cuda_runtime.h>

namespace pp {

struct df2 { float2 hi, lo; };

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as one FMA with the multiplier -1 (exact product, one rounding: the correctly rounded
// difference)
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// TwoSum / TwoDiff (Knuth) lane by lane: hi + lo == a +- b exactly.
__device__ __forceinline__ df2 two_sum2(float2 a, float2 b) {
  const float2 s = f2add(a, b);
  const float2 bp = f2sub(s, a);
  return df2{s, f2add(f2sub(a, f2sub(s, bp)), f2sub(b, bp))};
}
__device__ __forceinline__ df2 two_diff2(float2 a, float2 b) {
  const float2 s = f2sub(a, b);
  const float2 bp = f2sub(s, a);
  return df2{s, f2sub(f2sub(a, f2sub(s, bp)), f2add(b, bp))};
}

}  // namespace pp
