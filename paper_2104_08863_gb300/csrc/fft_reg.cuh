// In-register FFTs: a thread holds one short transform (N <= 32 complex values, N of the form
// 2^a 3^b) in registers and transforms it in place by decimation in frequency, with the
// twiddles of its internal stages as compile-time constants.  Used by the two-pass z-transform
// (a length-Nz transform as N1 x N2: an N2-point transform per thread, one shared-memory
// transpose with the inter-pass twiddles, an N1-point transform per thread).
#pragma once

#include <type_traits>

#include "fft_static.cuh"

namespace pp {

// ---- compile-time unit roots -----------------------------------------------------------------
// cos and sin of 2 pi num / den in double, evaluated by the compiler: the angle is reduced to an
// octant ((pi/4) (q + r/den)), reflected into [0, pi/4] when q is odd, where the Taylor series
// of cos and sin converge to double precision, and rotated back by a multiple of pi/2 (exact).
struct CS { double c, s; };
constexpr double kPiD = 3.14159265358979323846264338327950288;
constexpr double taylor_cos(double x) {
  double t = 1.0, s = 1.0;
  for (int k = 1; k < 16; ++k) {
    t *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
    s += t;
  }
  return s;
}
constexpr double taylor_sin(double x) {
  double t = x, s = x;
  for (int k = 1; k < 16; ++k) {
    t *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
    s += t;
  }
  return s;
}
constexpr CS unit_root(long long num, long long den) {
  const long long m = ((num % den) + den) % den;   // angle 2 pi m / den = (pi/4) 8m/den
  const long long q = (8 * m) / den, r = 8 * m - q * den;
  double c = 0.0, s = 0.0;
  long long quarter = 0;   // rotation by quarter * pi/2 applied last
  if (q % 2 == 0) {        // (pi/4) q + phi, phi = (pi/4) r/den in [0, pi/4)
    const double phi = (kPiD / 4.0) * (double)r / (double)den;
    c = taylor_cos(phi);
    s = taylor_sin(phi);
    quarter = q / 2;
  } else {                 // (pi/4)(q + 1) - phi', phi' = (pi/4)(den - r)/den in (0, pi/4]
    const double phi = (kPiD / 4.0) * (double)(den - r) / (double)den;
    c = taylor_cos(phi);
    s = -taylor_sin(phi);
    quarter = (q + 1) / 2;
  }
  for (long long k = 0; k < quarter % 4; ++k) {   // multiply by i
    const double t = c;
    c = -s;
    s = t;
  }
  return CS{c, s};
}

// ---- compile-time loops ----------------------------------------------------------------------
template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// ---- register DFT ------------------------------------------------------------------------------
__host__ __device__ constexpr bool reg_base(int n) { return n == 2 || n == 3 || n == 4 || n == 8 || n == 16; }
__host__ __device__ constexpr int reg_radix(int n) {
  return reg_base(n) ? n : (n % 8 == 0 ? 8 : (n % 4 == 0 ? 4 : (n % 2 == 0 ? 2 : 3)));
}
// Frequency held by slot s of an n-point register DFT after reg_dft (decimation in frequency
// leaves the outputs in digit-reversed order; the callers index by this map at compile time).
__host__ __device__ constexpr int reg_freq(int n, int s) {
  if (n == 1 || reg_base(n)) return s;
  const int R = reg_radix(n), np = n / R;
  return R * reg_freq(np, s % np) + s / np;
}

// a * e^{SIGN 2 pi i k / N} for compile-time k, N (trivial factors cost no multiply).
template <typename T, int SIGN, int K, int N>
__device__ __forceinline__ cplx<T> twiddle_c(cplx<T> a) {
  constexpr int k = ((K % N) + N) % N;
  if constexpr (k == 0) {
    return a;
  } else if constexpr (4 * k == N) {
    return mul_i(a, SIGN);
  } else if constexpr (2 * k == N) {
    return mk<T>(-a.x, -a.y);
  } else if constexpr (4 * k == 3 * N) {
    return mul_i(a, -SIGN);
  } else {
    constexpr CS w = unit_root((long long)SIGN * k, N);
    return cmul(a, mk<T>(T(w.c), T(w.s)));
  }
}

// In-place N-point DFT (e^{SIGN 2 pi i n k / N}) of v[0..N-1]; slot s ends up holding frequency
// reg_freq(N, s).  x[n1 + NP n2] (NP = N/R) -> R-point DFTs over n2, twiddles W_N^{n1 k2},
// NP-point DFTs over n1 on the contiguous slices v[NP k2 ..].
template <typename T, int N, int SIGN>
__device__ __forceinline__ void reg_dft(cplx<T>* v) {
  if constexpr (N == 1) {
    return;
  } else if constexpr (reg_base(N)) {
    dft_r<T, N, SIGN>(v);
  } else {
    constexpr int R = reg_radix(N), NP = N / R;
    static_for<0, NP>([&](auto n1c) {
      constexpr int n1 = decltype(n1c)::value;
      cplx<T> t[R];
#pragma unroll
      for (int r = 0; r < R; ++r) t[r] = v[n1 + NP * r];
      dft_r<T, R, SIGN>(t);
      static_for<0, R>([&](auto k2c) {
        constexpr int k2 = decltype(k2c)::value;
        v[n1 + NP * k2] = twiddle_c<T, SIGN, n1 * k2, N>(t[k2]);
      });
    });
    static_for<0, R>([&](auto k2c) { reg_dft<T, NP, SIGN>(v + NP * decltype(k2c)::value); });
  }
}

// Split n = n1 * n2 with n1 >= n2 (n1 the smallest divisor >= sqrt(n)); both <= 32 for n <= 1024.
__host__ __device__ constexpr int split_n1(int n) {
  int d = 1;
  while (d * d < n) ++d;
  while (n % d) ++d;
  return d;
}

}  // namespace pp
