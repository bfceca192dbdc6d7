// Two-pass register z-transform (FP32): the tile function shared by the standalone kernel
// (k_fft_z_fast.cu) and the persistent batched kernel (batch_persistent.cu).
#pragma once

#include "fft_reg.cuh"
#include "internal.h"

namespace pp {

// ---- two-pass register z-transform (FP32) ------------------------------------------------------
// Nz = N1 x N2 (N1 >= N2, both <= 32).  A CTA owns W adjacent kx columns of one y-plane.  Pass 1:
// thread (c, n1) loads the N2 values x[n1 + N1 n2] of column c straight from global memory into
// registers, takes their N2-point DFT in registers, multiplies output k2 by W_Nz^{n1 k2} and writes
// it to shared memory at [k2][n1][c].  Pass 2: thread (c, k2) reads the N1 values of its k2, takes
// their N1-point DFT (output k1 is X[k2 + N2 k1]) and stores to global memory.  One shared-memory
// round trip per element (the Stockham kernel makes one per stage plus two), and each thread's
// global loads are all issued before any arithmetic.  The k2 blocks of shared memory are padded so
// that their byte stride is 64 mod 128: the pass-2 reads of a warp (four k2 blocks of W columns)
// then fall on alternating bank halves.
template <typename T, int NZ> struct ZReg {
  static constexpr int N1 = split_n1(NZ), N2 = NZ / N1;
  static constexpr int WMIN = sizeof(T) == 4 ? 8 : 4;   // 64-byte row segments
  static constexpr int W0 = 256 / N1;
  static constexpr int W1 = W0 >= 32 ? 32 : (W0 >= 16 ? 16 : 8);   // a power of two: aligned row segments
  static constexpr int W = W1 < WMIN ? WMIN : W1;
  static constexpr int THREADS = W * N1;
  static constexpr int CB = (int)sizeof(cplx<T>);
  static constexpr int B0 = N1 * W;
  static constexpr int B = B0 + (((64 - (B0 * CB) % 128) + 128) % 128) / CB;   // B * CB == 64 (mod 128)
  static constexpr int SMEM = N2 * B * CB;
  static_assert((B * CB) % 128 == 64, "pad");
  static_assert(N1 <= 32 && N2 <= 32 && N1 * N2 == NZ, "split");
};

// One tile: columns kx_lo + bx W .. + W - 1 of y-plane j.  Called by every thread of the CTA
// (blockDim.x >= C::THREADS; threads past C::THREADS only take part in the barrier).  A caller
// that runs another tile on the same shared memory puts a barrier between the two.
template <typename T, int NZ, int SIGN>
__device__ __forceinline__ void z_reg_tile(const Geometry& g, const Tables<T>& tt, cplx<T>* __restrict__ spec,
                                           int kx_lo, int kx_hi, int bx, int j, unsigned char* smem_raw) {
  using C = ZReg<T, NZ>;
  constexpr int N1 = C::N1, N2 = C::N2, W = C::W, B = C::B;
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
  const int kx0 = kx_lo + bx * W;
  cplx<T>* plane = spec + (size_t)j * NZ * g.pitch + kx0;
  const int ncol = min(W, kx_hi - kx0);
  const int c = threadIdx.x % W, q = threadIdx.x / W;
  const bool live = threadIdx.x < C::THREADS;
  const bool cok = live && c < ncol;
  if (live) {
    const int n1 = q;   // < N1
    cplx<T> v[N2];
    const cplx<T>* src = plane + (size_t)n1 * g.pitch + c;
    const size_t step = (size_t)N1 * g.pitch;
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) v[n2] = cok ? ld_c(src + n2 * step) : mk<T>(T(0), T(0));
    reg_dft<T, N2, SIGN>(v);
    static_for<0, N2>([&](auto sc) {
      constexpr int s = decltype(sc)::value;
      constexpr int k2 = reg_freq(N2, s);
      cplx<T> x = v[s];
      if constexpr (k2 != 0) {
        const cplx<T> w = ldg_c(tt.tw_z + n1 * k2);
        x = SIGN < 0 ? cmul(x, w) : cmulc(x, w);
      }
      buf[k2 * B + n1 * W + c] = x;
    });
  }
  __syncthreads();
  if (live && q < N2) {
    const int k2 = q;
    cplx<T> u[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) u[n1] = buf[k2 * B + n1 * W + c];
    reg_dft<T, N1, SIGN>(u);
    if (cok) {
      cplx<T>* dst = plane + (size_t)k2 * g.pitch + c;
      const size_t step = (size_t)N2 * g.pitch;
      static_for<0, N1>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        constexpr int k1 = reg_freq(N1, s);
        st_c(dst + k1 * step, u[s]);
      });
    }
  }
}

template <typename T, int NZ, int SIGN>
__global__ void __launch_bounds__(ZReg<T, NZ>::THREADS, 2) k_fft_z_reg(Geometry g, Tables<T> tt,
                                                                      cplx<T>* __restrict__ spec, int kx_lo,
                                                                      int kx_hi) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  z_reg_tile<T, NZ, SIGN>(g, tt, spec, kx_lo, kx_hi, blockIdx.x, blockIdx.y, smem_raw);
}

}  // namespace pp
