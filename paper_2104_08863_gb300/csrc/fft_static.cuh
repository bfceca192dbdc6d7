// Compile-time specialised batched Stockham FFT (radix 16, 8, 4, 3, 2) in shared memory.
//
// Same self-sorting Stockham recurrence as fft.cuh (butterfly j of a radix-R stage with span
// Ns reads j + r L/R, is twiddled by W_L^{r (j mod Ns) L/(Ns R)} and writes
// (j div Ns) Ns R + (j mod Ns) + r Ns), but with the length, the radix sequence, the batch and
// the thread count fixed at compile time: every index is constant-folded, each thread's
// butterflies are unrolled, and a stage runs IN PLACE on one buffer by staging the thread's
// inputs in registers between two barriers.  Larger radices (16 = 4 x 4) mean fewer passes
// through shared memory, which bounds these kernels once HBM traffic is minimal.
#pragma once

#include "fft.cuh"

namespace pp {

struct Radix { int n; int r[8]; };

// Factorisation preferring radix 16 (when maxr allows), then 8, 4, 2, with the factors of 3
// last.  FP64 kernels cap the radix at 8: a radix-16 butterfly stages 32 doubles per thread,
// which halves their occupancy.
__host__ __device__ constexpr Radix factorize(int L, int maxr = 16) {
  Radix f{0, {0, 0, 0, 0, 0, 0, 0, 0}};
  int x = L;
  while (maxr >= 16 && x % 16 == 0 && x > 8) { f.r[f.n++] = 16; x /= 16; }
  while (x % 8 == 0) { f.r[f.n++] = 8; x /= 8; }
  while (x % 4 == 0) { f.r[f.n++] = 4; x /= 4; }
  while (x % 2 == 0) { f.r[f.n++] = 2; x /= 2; }
  while (x % 3 == 0) { f.r[f.n++] = 3; x /= 3; }
  return f;
}
__host__ __device__ constexpr bool factorizable(int L) {
  int x = L;
  while (x % 2 == 0) x /= 2;
  while (x % 3 == 0) x /= 3;
  return x == 1 && L > 1;
}
template <typename T> __host__ __device__ constexpr int max_radix() { return sizeof(T) == 4 ? 16 : 8; }

__host__ __device__ constexpr int span_before(int L, int s, int maxr) {
  int ns = 1;
  const Radix f = factorize(L, maxr);
  for (int i = 0; i < s; ++i) ns *= f.r[i];
  return ns;
}

// 16-point DFT as 4 x 4 with internal twiddles W16^{n2 k1}.
template <typename T, int SIGN>
__device__ __forceinline__ void dft16(cplx<T>* v) {
  const T c1 = T(0.92387953251128675613), s1 = T(0.38268343236508977173), r = T(0.70710678118654752440);
  cplx<T> a[4][4];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    cplx<T> q[4] = {v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]};
    dft4<T, SIGN>(q);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) a[n2][k1] = q[k1];
  }
  // twiddles W16^{n2 k1}, exponent in {0, 1, 2, 3, 4, 6, 9}; W = cos + SIGN i sin
  const T sg = T(SIGN);
  a[1][1] = cmul(a[1][1], mk<T>(c1, sg * s1));
  a[1][2] = cmul(a[1][2], mk<T>(r, sg * r));
  a[1][3] = cmul(a[1][3], mk<T>(s1, sg * c1));
  a[2][1] = cmul(a[2][1], mk<T>(r, sg * r));
  a[2][2] = mul_i(a[2][2], SIGN);
  a[2][3] = cmul(a[2][3], mk<T>(-r, sg * r));
  a[3][1] = cmul(a[3][1], mk<T>(s1, sg * c1));
  a[3][2] = cmul(a[3][2], mk<T>(-r, sg * r));
  a[3][3] = cmul(a[3][3], mk<T>(-c1, -sg * s1));
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    cplx<T> q[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
    dft4<T, SIGN>(q);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = q[k2];
  }
}

template <typename T, int R, int SIGN>
__device__ __forceinline__ void dft_r(cplx<T>* v) {
  if constexpr (R == 2) dft2<T, SIGN>(v);
  if constexpr (R == 3) dft3<T, SIGN>(v);
  if constexpr (R == 4) dft4<T, SIGN>(v);
  if constexpr (R == 8) dft8<T, SIGN>(v);
  if constexpr (R == 16) dft16<T, SIGN>(v);
}

// Shared-memory padding: logical element i lives at i + (i >> P), one pad slot per 2^P
// elements (128 bytes of data), which spreads the strided Stockham writes over the banks.
template <typename T> struct SmemPad { static constexpr int shift = sizeof(T) == 4 ? 4 : 3; };
template <typename T> __device__ __forceinline__ int padi(int i) { return i + (i >> SmemPad<T>::shift); }
template <typename T> __host__ __device__ constexpr int padded_size(int n) { return n + (n >> SmemPad<T>::shift) + 1; }

// One in-place stage.  Element n of transform t lives at buf[padi(t*BS + n*ES)]; B transforms.
// MAPB: consecutive threads take consecutive transforms (column tiles) instead of
// consecutive butterflies (rows).
template <typename T, int L, int S, int SIGN, int B, int THREADS, int ES, int BS, bool MAPB, int MAXR>
__device__ __forceinline__ void stage_inplace(cplx<T>* buf, const cplx<T>* __restrict__ tw) {
  constexpr Radix F = factorize(L, MAXR);
  constexpr int R = F.r[S];
  constexpr int Ns = span_before(L, S, MAXR);
  constexpr int NBF = L / R;
  constexpr int TOTAL = NBF * B;
  constexpr int PER = (TOTAL + THREADS - 1) / THREADS;
  constexpr int TSTRIDE = L / (Ns * R);
  cplx<T> v[PER][R];
  int jj[PER], tt[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int idx = threadIdx.x + q * THREADS;
    int t, j;
    if (MAPB) { t = idx % B; j = idx / B; } else { j = idx % NBF; t = idx / NBF; }
    jj[q] = j;
    tt[q] = t;
    if (TOTAL % THREADS == 0 || idx < TOTAL) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = buf[padi<T>(t * BS + (j + r * NBF) * ES)];
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int idx = threadIdx.x + q * THREADS;
    if (TOTAL % THREADS == 0 || idx < TOTAL) {
      const int j = jj[q], t = tt[q];
      const int k = j % Ns;
      if (Ns > 1 && k != 0) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          const cplx<T> w = ldg_c(tw + r * k * TSTRIDE);
          v[q][r] = SIGN < 0 ? cmul(v[q][r], w) : cmulc(v[q][r], w);
        }
      }
      dft_r<T, R, SIGN>(v[q]);
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[padi<T>(t * BS + (base + r * Ns) * ES)] = v[q][r];
    }
  }
  __syncthreads();
}

// The first stage (span 1, no twiddles) with its inputs taken from load(t, n), element n of
// transform t, instead of buf: the callers read a staged copy of the raw input and pack or
// convert it on the way in, which saves one pass through shared memory.
template <typename T, int L, int SIGN, int B, int THREADS, int ES, int BS, bool MAPB, int MAXR, typename Load>
__device__ __forceinline__ void stage_first(cplx<T>* buf, Load load) {
  constexpr Radix F = factorize(L, MAXR);
  constexpr int R = F.r[0];
  constexpr int NBF = L / R;
  constexpr int TOTAL = NBF * B;
  constexpr int PER = (TOTAL + THREADS - 1) / THREADS;
  cplx<T> v[PER][R];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int idx = threadIdx.x + q * THREADS;
    const int t = MAPB ? idx % B : idx / NBF, j = MAPB ? idx / B : idx % NBF;
    if (TOTAL % THREADS == 0 || idx < TOTAL) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = load(t, j + r * NBF);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int idx = threadIdx.x + q * THREADS;
    const int t = MAPB ? idx % B : idx / NBF, j = MAPB ? idx / B : idx % NBF;
    if (TOTAL % THREADS == 0 || idx < TOTAL) {
      dft_r<T, R, SIGN>(v[q]);
#pragma unroll
      for (int r = 0; r < R; ++r) buf[padi<T>(t * BS + (j * R + r) * ES)] = v[q][r];
    }
  }
  __syncthreads();
}

template <typename T, int L, int S, int SIGN, int B, int THREADS, int ES, int BS, bool MAPB, int MAXR>
__device__ __forceinline__ void stages_from(cplx<T>* buf, const cplx<T>* __restrict__ tw) {
  constexpr Radix F = factorize(L, MAXR);
  if constexpr (S < F.n) {
    stage_inplace<T, L, S, SIGN, B, THREADS, ES, BS, MAPB, MAXR>(buf, tw);
    stages_from<T, L, S + 1, SIGN, B, THREADS, ES, BS, MAPB, MAXR>(buf, tw);
  }
}

// Full transform, in place on buf (callers sync before: the first stage reads buf).  MAXR caps
// the radix (and so the values a thread stages per butterfly).
template <typename T, int L, int SIGN, int B, int THREADS, int ES, int BS, bool MAPB, int MAXR = max_radix<T>()>
__device__ __forceinline__ void fft_static(cplx<T>* buf, const cplx<T>* __restrict__ tw) {
  static_assert(factorizable(L), "FFT length must be 2^a 3^b");
  stages_from<T, L, 0, SIGN, B, THREADS, ES, BS, MAPB, MAXR>(buf, tw);
}

// Full transform whose input is read by load(t, n) (see stage_first); `after_first()` runs once
// every thread has finished reading the input (the staging it came from may then be refilled).
template <typename T, int L, int SIGN, int B, int THREADS, int ES, int BS, bool MAPB, int MAXR, typename Load,
          typename Hook>
__device__ __forceinline__ void fft_static_from(cplx<T>* buf, const cplx<T>* __restrict__ tw, Load load,
                                                Hook after_first) {
  static_assert(factorizable(L), "FFT length must be 2^a 3^b");
  stage_first<T, L, SIGN, B, THREADS, ES, BS, MAPB, MAXR>(buf, load);
  after_first();
  stages_from<T, L, 1, SIGN, B, THREADS, ES, BS, MAPB, MAXR>(buf, tw);
}

}  // namespace pp
