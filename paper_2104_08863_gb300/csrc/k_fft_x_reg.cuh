// Two-pass register x-transforms for FP32 spectra of FP32 fields (steps (2) and (8) of Sec. 3.2),
// and the forward transform of the refinement residual.
//
// The half-length complex transform of a line (M = Nx/2 = N1 x N2, N1 >= N2, both <= 32) is done
// by threads that each hold a whole short transform in registers: pass 1 thread (t, n1) of line
// t produces z[n1 + N1 n2] for n2 < N2 directly from the field (the right-hand side producer of
// the mode: a plain load, the divergence of Eq. 7, the adjoint's G^T g), takes their
// N2-point DFT, multiplies output k2 by W_M^{n1 k2} and writes it to shared memory at
// [t][k2][n1]; pass 2 thread (t, k2) takes the N1-point DFT of row k2 (output k1 is Z[k2 + N2 k1]).
// Forward: the Z are written back in natural order and the Nx/2+1 spectral bins unpacked from
// Z_k and Z_{M-k} (fwd_post) and stored.  Inverse: pass 1 packs X_k and X_{M-k} (inv_pre) on the
// way in, pass 2 writes (or adds) the real values straight from registers, with the line's
// dy-weighted sum when asked.  Against the Stockham kernels this makes
// one (inverse) or two (forward) shared-memory round trips instead of one per stage plus two, and
// every index is a compile-time constant.  Row k2 of a line's buffer has an odd stride B = N1 + 1
// (in complex values), so the pass-2 reads of consecutive k2 fall on distinct bank pairs.
#pragma once

#include "fft_reg.cuh"
#include "xline.cuh"

namespace pp {

template <int M> struct XReg {
  static constexpr int N1 = split_n1(M), N2 = M / N1;
  static constexpr int LPB0 = 256 / N1;
  static constexpr int LPB = LPB0 < 1 ? 1 : (LPB0 > 32 ? 32 : LPB0);
  static constexpr int THREADS = LPB * N1;
  static constexpr int B = N1 % 2 == 0 ? N1 + 1 : N1;
  static constexpr int LS = N2 * B > M ? N2 * B : M;   // per-line stride (>= M for the natural order)
  static constexpr int SMEM = LPB * LS * (int)sizeof(cplx<float>);
  static_assert(N1 * N2 == M && N1 <= 32 && N2 <= 32, "split");
  static_assert(B % 2 == 1, "odd row stride");
};

// Forward x-transform of an FP32 field into the FP32 half spectrum; MODE as in fwd_load
// (FWD_PLAIN, FWD_DIV, FWD_GRADT).
// One tile: lines tile * LPB .. + LPB - 1.  Called by every thread of the CTA (blockDim.x >=
// C::THREADS; threads past C::THREADS only take part in the barriers).
template <typename TI, int M, int MODE>
__device__ __forceinline__ void fwd_x_reg_tile(const Geometry& g, const FwdArgs& args, const Tables<float>& tt,
                                               const DevTables& tb, cplx<float>* __restrict__ spec, int nlines,
                                               int tile, unsigned char* smem_raw) {
  using C = XReg<M>;
  constexpr int N1 = C::N1, N2 = C::N2, LPB = C::LPB, B = C::B, LS = C::LS, THREADS = C::THREADS;
  cplx<float>* buf = reinterpret_cast<cplx<float>*>(smem_raw);
  const int line0 = tile * LPB;
  const bool live = threadIdx.x < THREADS;
  if (live) {
    const int t = threadIdx.x / N1, n1 = threadIdx.x - t * N1;
    const int line = line0 + t;
    cplx<float> v[N2];
    if (line < nlines) {
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) v[n2] = fwd_load<float, TI, MODE>(g, args, tt, tb, line, n1 + N1 * n2);
    } else {
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) v[n2] = mk<float>(0.f, 0.f);
    }
    reg_dft<float, N2, -1>(v);
    cplx<float>* row = buf + t * LS + n1;
    static_for<0, N2>([&](auto sc) {
      constexpr int s = decltype(sc)::value;
      constexpr int k2 = reg_freq(N2, s);
      cplx<float> x = v[s];
      if constexpr (k2 != 0) x = cmul(x, ldg_c(tt.tw_m + n1 * k2));
      row[k2 * B] = x;
    });
  }
  __syncthreads();
  constexpr int P2 = LPB * N2;   // pass-2 threads
  cplx<float> u[N1];
  const int t2 = threadIdx.x / N2, k2 = threadIdx.x - t2 * N2;
  if (threadIdx.x < P2) {
    const cplx<float>* row = buf + t2 * LS + k2 * B;
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) u[n1] = row[n1];
    reg_dft<float, N1, -1>(u);
  }
  __syncthreads();
  if (threadIdx.x < P2) {
    cplx<float>* nat = buf + t2 * LS + k2;
    static_for<0, N1>([&](auto sc) {
      constexpr int s = decltype(sc)::value;
      nat[N2 * reg_freq(N1, s)] = u[s];
    });
  }
  __syncthreads();
  constexpr int M1 = M + 1;
  if (live) {
#pragma unroll 4
    for (int idx = threadIdx.x; idx < LPB * M1; idx += THREADS) {
      const int t = idx / M1, kx = idx - t * M1;
      const int line = line0 + t;
      if (line >= nlines) continue;
      const cplx<float>* nat = buf + t * LS;
      const cplx<float> Zk = nat[kx == M ? 0 : kx];
      const cplx<float> Zc = conj(nat[kx == 0 ? 0 : M - kx]);
      st_c(spec + (size_t)line * g.pitch + kx, fwd_post(Zk, Zc, ldg_c(tt.tw_post + kx)));
    }
  }
}

// Three CTAs per SM (85 registers), as for the inverse below.
template <typename TI, int M, int MODE>
__global__ void __launch_bounds__(XReg<M>::THREADS, 3)
    k_fwd_x_reg(Geometry g, FwdArgs args, Tables<float> tt, DevTables tb, cplx<float>* __restrict__ spec,
                int nlines) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  fwd_x_reg_tile<TI, M, MODE>(g, args, tt, tb, spec, nlines, blockIdx.x, smem_raw);
}

// Refinement residual r = (f - <f>) - L_h p, or rin - L_h p for a later correction
// (resid_pair_line2), transformed into the FP32 half spectrum.  Phase 0: one warp per line forms
// the residual pairs in natural order in shared memory (the line's set-up amortised over M/32
// pairs per lane, loads coalesced across the warp); the register transform then reads its inputs from there (one more
// barrier, since pass 1 overwrites the natural order with the transposed rows of the same line).
template <int M, bool RIN>
__device__ __forceinline__ void fwd_x_reg_resid_tile(const Geometry& g, const FwdArgs& args, const Tables<float>& tt,
                                                     const DevTables& tb, cplx<float>* __restrict__ spec,
                                                     int nlines, int tile, unsigned char* smem_raw) {
  using C = XReg<M>;
  constexpr int N1 = C::N1, N2 = C::N2, LPB = C::LPB, B = C::B, LS = C::LS, THREADS = C::THREADS;
  constexpr int NW = THREADS / 32;   // whole warps (a partial last warp skips phase 0)
  static_assert(NW >= 1, "at least one warp");
  cplx<float>* buf = reinterpret_cast<cplx<float>*>(smem_raw);
  const int line0 = tile * LPB;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp < NW) {
    float mh, ml;
    f64_split(tb.acc[0], mh, ml);
    for (int t = warp; t < LPB; t += NW) {
      const int line = line0 + t;
      cplx<float>* nat = buf + t * LS;
      if (line < nlines) {
        const ResidLine R = resid_line(g, args, tt, tb, line, mh, ml);
#pragma unroll 3
        for (int n = lane; n < M; n += 32) {
          const float2 r = resid_pair_line2<RIN>(R, n);
          nat[n] = mk<float>(r.x, r.y);
        }
      } else {
        for (int n = lane; n < M; n += 32) nat[n] = mk<float>(0.f, 0.f);
      }
    }
  }
  __syncthreads();
  const bool live = threadIdx.x < THREADS;
  const int t = threadIdx.x / N1, n1 = threadIdx.x - t * N1;
  cplx<float> v[N2];
  if (live) {
    const cplx<float>* nat = buf + t * LS + n1;
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) v[n2] = nat[N1 * n2];
  }
  __syncthreads();
  if (live) {
    reg_dft<float, N2, -1>(v);
    cplx<float>* row = buf + t * LS + n1;
    static_for<0, N2>([&](auto sc) {
      constexpr int s = decltype(sc)::value;
      constexpr int k2 = reg_freq(N2, s);
      cplx<float> x = v[s];
      if constexpr (k2 != 0) x = cmul(x, ldg_c(tt.tw_m + n1 * k2));
      row[k2 * B] = x;
    });
  }
  __syncthreads();
  constexpr int P2 = LPB * N2;   // pass-2 threads
  cplx<float> u[N1];
  const int t2 = threadIdx.x / N2, k2 = threadIdx.x - t2 * N2;
  if (threadIdx.x < P2) {
    const cplx<float>* row = buf + t2 * LS + k2 * B;
#pragma unroll
    for (int q = 0; q < N1; ++q) u[q] = row[q];
    reg_dft<float, N1, -1>(u);
  }
  __syncthreads();
  if (threadIdx.x < P2) {
    cplx<float>* nat = buf + t2 * LS + k2;
    static_for<0, N1>([&](auto sc) {
      constexpr int s = decltype(sc)::value;
      nat[N2 * reg_freq(N1, s)] = u[s];
    });
  }
  __syncthreads();
  constexpr int M1 = M + 1;
  if (live) {
#pragma unroll 4
    for (int idx = threadIdx.x; idx < LPB * M1; idx += THREADS) {
      const int tl = idx / M1, kx = idx - tl * M1;
      const int line = line0 + tl;
      if (line >= nlines) continue;
      const cplx<float>* nat = buf + tl * LS;
      const cplx<float> Zk = nat[kx == M ? 0 : kx];
      const cplx<float> Zc = conj(nat[kx == 0 ? 0 : M - kx]);
      st_c(spec + (size_t)line * g.pitch + kx, fwd_post(Zk, Zc, ldg_c(tt.tw_post + kx)));
    }
  }
}

// RIN: a later correction (the stored first residual in place of f - <f>, see resid_line).
template <int M, bool RIN>
__global__ void __launch_bounds__(XReg<M>::THREADS, 3)
    k_fwd_x_reg_resid(Geometry g, FwdArgs args, Tables<float> tt, DevTables tb, cplx<float>* __restrict__ spec,
                      int nlines) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  fwd_x_reg_resid_tile<M, RIN>(g, args, tt, tb, spec, nlines, blockIdx.x, smem_raw);
}

// Inverse x-transform of the FP32 half spectrum into an FP32 field with the epilogue MODE
// (INV_STORE, INV_ACCUM); ACC also adds the dy-weighted sum of the result to acc[1], formed in
// double-float arithmetic on the FP32 units (one FP64 atomic per warp).
template <typename TO, int M, int MODE, bool ACC>
__device__ __forceinline__ void inv_x_reg_tile(const Geometry& g, const Tables<float>& tt,
                                               const cplx<float>* __restrict__ spec, TO* __restrict__ out,
                                               double scl, int nlines, const double* __restrict__ dy,
                                               double* __restrict__ acc, const PairArgs& pair, int tile,
                                               unsigned char* smem_raw) {
  using C = XReg<M>;
  constexpr int N1 = C::N1, N2 = C::N2, LPB = C::LPB, B = C::B, LS = C::LS;
  cplx<float>* buf = reinterpret_cast<cplx<float>*>(smem_raw);
  const int line0 = tile * LPB;
  if (threadIdx.x < C::THREADS) {
    const int t = threadIdx.x / N1, n1 = threadIdx.x - t * N1;
    const int line = line0 + t;
    cplx<float> v[N2];
    if (line < nlines) {
      const cplx<float>* X = spec + (size_t)line * g.pitch;
      cplx<float> xk[N2], xm[N2];
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) {
        const int n = n1 + N1 * n2;
        xk[n2] = ld_c_cg(X + n);   // coherent with a persistent launch's earlier stores
        xm[n2] = ld_c_cg(X + (M - n));
      }
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) {
        const int n = n1 + N1 * n2;
        v[n2] = inv_pre(n, xk[n2], xm[n2], ldg_c(tt.tw_post + n));
      }
    } else {
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) v[n2] = mk<float>(0.f, 0.f);
    }
    reg_dft<float, N2, 1>(v);
    cplx<float>* row = buf + t * LS + n1;
    static_for<0, N2>([&](auto sc) {
      constexpr int s = decltype(sc)::value;
      constexpr int k2 = reg_freq(N2, s);
      cplx<float> x = v[s];
      if constexpr (k2 != 0) x = cmulc(x, ldg_c(tt.tw_m + n1 * k2));
      row[k2 * B] = x;
    });
  }
  __syncthreads();
  constexpr int P2 = LPB * N2;
  const int t2 = threadIdx.x / N2, k2 = threadIdx.x - t2 * N2;
  const int line = line0 + t2;
  const bool act = threadIdx.x < P2 && line < nlines;
  df w{0.f, 0.f};   // this thread's dy-weighted sum as a double-float
  if (act) {
    cplx<float> u[N1];
    const cplx<float>* row = buf + t2 * LS + k2 * B;
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) u[n1] = row[n1];
    reg_dft<float, N1, 1>(u);
    const float s = float(scl);
    const size_t o0 = (size_t)line * g.nx + 2 * k2;
    // compensated sums with the pair (x0, x1) in the two lanes of packed FP32x2 operations, the
    // thread's successive outputs alternating between two independent chains
    float2 hs[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    float2 hc[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    static_for<0, N1>([&](auto sc) {
      constexpr int sl = decltype(sc)::value;
      constexpr int k1 = reg_freq(N1, sl);
      const float x0 = u[sl].x * s, x1 = u[sl].y * s;
      inv_store<float, TO, MODE>(out + o0 + 2 * N2 * k1, o0 + 2 * N2 * k1, x0, x1, pair);
      if constexpr (ACC) {
        const df2 t = two_sum2(hs[sl & 1], make_float2(x0, x1));
        hs[sl & 1] = t.hi;
        hc[sl & 1] = f2add(hc[sl & 1], t.lo);
      }
    });
    if constexpr (ACC) {
      // the four partial sums, then times dy_j split into two floats (TwoProd by FMA)
      df a = two_sum_df(hs[0].x, hs[0].y), b = two_sum_df(hs[1].x, hs[1].y);
      a.lo += (hc[0].x + hc[0].y);
      b.lo += (hc[1].x + hc[1].y);
      const df sum = df_add(a, b);
      float dh, dl;
      f64_split(dy[line / g.nz], dh, dl);
      const float ph = sum.hi * dh;
      w = df{ph, fmaf(sum.hi, dh, -ph) + (sum.hi * dl + sum.lo * dh)};
    }
  }
  if constexpr (ACC) {
    // warp sum in double-float, one FP64 atomic per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const df y{__shfl_xor_sync(0xffffffffu, w.hi, o), __shfl_xor_sync(0xffffffffu, w.lo, o)};
      w = df_add(w, y);
    }
    if ((threadIdx.x & 31) == 0) {
      const double wsum = (double)w.hi + (double)w.lo;
      if (wsum != 0.0) atomicAdd(acc + 1, wsum);
    }
  }
}

// Three CTAs per SM (85 registers): the inverse's pass 2 streams its results straight from
// registers, and the extra resident warps hide that more than the spills it causes cost (1.9 vs
// 2.1 ms per pass at 1536x768x1024; the forward and the z-transform measured the other way).
template <typename TO, int M, int MODE, bool ACC>
__global__ void __launch_bounds__(XReg<M>::THREADS, 3)
    k_inv_x_reg(Geometry g, Tables<float> tt, const cplx<float>* __restrict__ spec, TO* __restrict__ out, double scl,
                int nlines, const double* __restrict__ dy, double* __restrict__ acc, PairArgs pair) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  inv_x_reg_tile<TO, M, MODE, ACC>(g, tt, spec, out, scl, nlines, dy, acc, pair, blockIdx.x, smem_raw);
}

}  // namespace pp
