// Batched mixed-radix (2, 3, 4, 8) Stockham FFT over shared memory.
//
// The transforms in the periodic directions (x and z) of Eq. 9 are complex-exponential DFTs;
// this header computes a batch of them on data staged in shared memory.  The self-sorting
// Stockham formulation (published by Stockham, 1966; GPU form of Govindaraju et al., SC'08)
// needs no bit reversal: at a stage of radix R with already-combined span Ns, butterfly j of
// a length-L transform reads elements j + r L/R (r < R), multiplies element r by
// W_L^{r (j mod Ns) L/(Ns R)}, takes an R-point DFT and writes element r to
// (j div Ns) Ns R + (j mod Ns) + r Ns of the other buffer.
//
// Element n of transform t lives at buf[t*bs + n*es].  SIGN = -1 is the forward transform
// (e^{-2 pi i nk/L}), SIGN = +1 the unnormalised inverse.  The twiddle table tw[t] holds
// e^{-2 pi i t/L} (t < L) in global memory; the inverse uses its conjugate.
#pragma once

#include "common.cuh"

namespace pp {

struct FftFactors {
  int L;        // transform length
  int nst;      // number of stages
  int rad[12];  // radix of each stage (2, 3, 4 or 8)
};

template <typename T, int SIGN>
__device__ __forceinline__ void dft2(cplx<T>* v) {
  cplx<T> a = v[0], b = v[1];
  v[0] = a + b;
  v[1] = a - b;
}

template <typename T, int SIGN>
__device__ __forceinline__ void dft4(cplx<T>* v) {
  cplx<T> a = v[0] + v[2], b = v[0] - v[2];
  cplx<T> c = v[1] + v[3], d = mul_i(v[1] - v[3], SIGN);
  v[0] = a + c;
  v[2] = a - c;
  v[1] = b + d;
  v[3] = b - d;
}

template <typename T, int SIGN>
__device__ __forceinline__ void dft3(cplx<T>* v) {
  const T h = T(0.86602540378443864676372317075294);  // sqrt(3)/2
  cplx<T> t1 = v[1] + v[2], t2 = v[1] - v[2];
  cplx<T> x0 = v[0] + t1;
  cplx<T> m1 = mk<T>(v[0].x - T(0.5) * t1.x, v[0].y - T(0.5) * t1.y);
  cplx<T> m2 = mul_i(scale(t2, h), SIGN);
  v[0] = x0;
  v[1] = m1 + m2;
  v[2] = m1 - m2;
}

// multiply by e^{SIGN 2 pi i / 8} = (1 + SIGN i)/sqrt(2)
template <typename T, int SIGN>
__device__ __forceinline__ cplx<T> w8(cplx<T> a) {
  const T r = T(0.70710678118654752440084436210485);
  return SIGN < 0 ? mk<T>((a.x + a.y) * r, (a.y - a.x) * r) : mk<T>((a.x - a.y) * r, (a.y + a.x) * r);
}

template <typename T, int SIGN>
__device__ __forceinline__ void dft8(cplx<T>* v) {
  cplx<T> e[4] = {v[0], v[2], v[4], v[6]};
  cplx<T> o[4] = {v[1], v[3], v[5], v[7]};
  dft4<T, SIGN>(e);
  dft4<T, SIGN>(o);
  o[1] = w8<T, SIGN>(o[1]);
  o[2] = mul_i(o[2], SIGN);
  o[3] = mul_i(w8<T, SIGN>(o[3]), SIGN);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[k] = e[k] + o[k];
    v[k + 4] = e[k] - o[k];
  }
}

template <typename T, int R, int SIGN>
__device__ __forceinline__ void butterfly(const cplx<T>* __restrict__ sp, cplx<T>* __restrict__ dp, int j,
                                          int nbf, int Ns, int tstride, int es,
                                          const cplx<T>* __restrict__ tw) {
  cplx<T> v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = sp[(j + r * nbf) * es];
  const int k = j % Ns;
  if (k != 0) {
#pragma unroll
    for (int r = 1; r < R; ++r) {
      cplx<T> w = ldg_c(tw + r * k * tstride);
      v[r] = SIGN < 0 ? cmul(v[r], w) : cmulc(v[r], w);
    }
  }
  if (R == 2) dft2<T, SIGN>(v);
  if (R == 3) dft3<T, SIGN>(v);
  if (R == 4) dft4<T, SIGN>(v);
  if (R == 8) dft8<T, SIGN>(v);
  const int base = (j - k) * R + k;
#pragma unroll
  for (int r = 0; r < R; ++r) dp[(base + r * Ns) * es] = v[r];
}

// Runs all stages; returns the buffer that holds the result (buf0 or buf1).
// batch_fastest selects the thread-to-work mapping: consecutive threads take consecutive
// transforms (for column batches, es > 1, bs == 1) or consecutive butterflies (rows, es == 1).
template <typename T, int SIGN>
__device__ cplx<T>* fft_smem(cplx<T>* buf0, cplx<T>* buf1, const FftFactors& f, int nbatch, int es, int bs,
                             bool batch_fastest, const cplx<T>* __restrict__ tw) {
  const int L = f.L;
  cplx<T>* src = buf0;
  cplx<T>* dst = buf1;
  int Ns = 1;
  for (int s = 0; s < f.nst; ++s) {
    const int R = f.rad[s];
    const int nbf = L / R;
    const int tstride = L / (Ns * R);
    const int total = nbf * nbatch;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
      int t, j;
      if (batch_fastest) {
        t = idx % nbatch;
        j = idx / nbatch;
      } else {
        j = idx % nbf;
        t = idx / nbf;
      }
      const cplx<T>* sp = src + t * bs;
      cplx<T>* dp = dst + t * bs;
      switch (R) {
        case 8: butterfly<T, 8, SIGN>(sp, dp, j, nbf, Ns, tstride, es, tw); break;
        case 4: butterfly<T, 4, SIGN>(sp, dp, j, nbf, Ns, tstride, es, tw); break;
        case 3: butterfly<T, 3, SIGN>(sp, dp, j, nbf, Ns, tstride, es, tw); break;
        default: butterfly<T, 2, SIGN>(sp, dp, j, nbf, Ns, tstride, es, tw); break;
      }
    }
    __syncthreads();
    cplx<T>* tmp = src;
    src = dst;
    dst = tmp;
    Ns *= R;
  }
  return src;
}

}  // namespace pp
