// Shared device types and helpers for the sm_103a pressure-Poisson kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pp {

template <typename T> struct cplx { T x, y; };

template <typename T> struct vec2;
template <> struct vec2<float> { typedef float2 type; };
template <> struct vec2<double> { typedef double2 type; };

template <typename T> __device__ __forceinline__ cplx<T> mk(T a, T b) { cplx<T> r; r.x = a; r.y = b; return r; }
template <typename T> __device__ __forceinline__ cplx<T> operator+(cplx<T> a, cplx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ cplx<T> operator-(cplx<T> a, cplx<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename T> __device__ __forceinline__ cplx<T> cmulc(cplx<T> a, cplx<T> b) {
  return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename T> __device__ __forceinline__ cplx<T> conj(cplx<T> a) { return mk(a.x, -a.y); }
template <typename T> __device__ __forceinline__ cplx<T> scale(cplx<T> a, T s) { return mk(a.x * s, a.y * s); }
// multiply by +i (s = +1) or -i (s = -1)
template <typename T> __device__ __forceinline__ cplx<T> mul_i(cplx<T> a, int s) {
  return s > 0 ? mk(-a.y, a.x) : mk(a.y, -a.x);
}

template <typename T> __device__ __forceinline__ cplx<T> ldg_c(const cplx<T>* p) {
  typename vec2<T>::type v = __ldg(reinterpret_cast<const typename vec2<T>::type*>(p));
  return mk<T>(v.x, v.y);
}
template <typename T> __device__ __forceinline__ cplx<T> ld_c(const cplx<T>* p) {
  typename vec2<T>::type v = *reinterpret_cast<const typename vec2<T>::type*>(p);
  return mk<T>(v.x, v.y);
}
// A load that is coherent with stores made by other CTAs earlier in the same launch (through L2;
// never the read-only path).
template <typename T> __device__ __forceinline__ cplx<T> ld_c_cg(const cplx<T>* p) {
  const typename vec2<T>::type v = __ldcg(reinterpret_cast<const typename vec2<T>::type*>(p));
  return mk<T>(v.x, v.y);
}

template <typename T> __device__ __forceinline__ void st_c(cplx<T>* p, cplx<T> a) {
  typename vec2<T>::type v; v.x = a.x; v.y = a.y;
  *reinterpret_cast<typename vec2<T>::type*>(p) = v;
}

// Device status word codes (mirror poisson_status).
enum : int { DEV_OK = 0, DEV_TIMEOUT = 5, DEV_NONFINITE = 6 };

}  // namespace pp
