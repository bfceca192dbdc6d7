// Specialised x-transform kernels (steps (2) and (8) of Sec. 3.2) for the half-lengths
// M = Nx/2 in {16, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024}.
//
// A CTA takes LPB consecutive x-lines, which are one contiguous stretch of the field, packs
// each real line as M complex values, transforms all lines in place in padded shared memory
// with the compile-time Stockham engine, and unpacks the Nx/2+1 spectral bins (forward) or
// writes the Nx real values (inverse).  LPB and the thread count give each thread 16 (FP32) or
// 8 (FP64) staged complex values per stage.
#pragma once

#include <map>
#include <mutex>
#include <utility>

#include "bulk_copy.cuh"
#include "fft_static.cuh"
#include "k_fft_x_reg.cuh"
#include "xline.cuh"

namespace pp {

template <typename T, int M> struct XTile {
  static constexpr int E = 8;
  static constexpr int MAXR = 8;
  static constexpr int LPB0 = (E * 256) / M;
  static constexpr int LPB = LPB0 < 1 ? 1 : (LPB0 > 64 ? 64 : LPB0);
  static constexpr int T0 = ((LPB * M / E) + 31) / 32 * 32;
  static constexpr int THREADS = T0 < 64 ? 64 : (T0 > 512 ? 512 : T0);
  static constexpr int SMEM = padded_size<T>(LPB * M) * (int)sizeof(cplx<T>);
  static constexpr int MINB = sizeof(T) == 4 ? 4 : 2;
};

template <typename T, typename TI, int M, int MODE>
__global__ void __launch_bounds__(XTile<T, M>::THREADS, XTile<T, M>::MINB)
    k_fwd_x_fast(Geometry g, FwdArgs args, Tables<T> tt, DevTables tb, cplx<T>* __restrict__ spec, int nlines) {
  using C = XTile<T, M>;
  constexpr int LPB = C::LPB, THREADS = C::THREADS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
  const int line0 = blockIdx.x * LPB;
  if constexpr (MODE == FWD_RESID && sizeof(T) == 4) {
    // refinement residual: per-line setup, then pairs of cells
    float mh, ml;
    f64_split(tb.acc[0], mh, ml);
    for (int t = 0; t < LPB; ++t) {
      const int line = line0 + t;
      if (line < nlines) {
        const ResidLine R = resid_line(g, args, tt, tb, line, mh, ml);
#pragma unroll
        for (int n = threadIdx.x; n < M; n += THREADS) {
          const float2 r = R.rin ? resid_pair_line2<true>(R, n) : resid_pair_line2<false>(R, n);
          buf[padi<T>(t * M + n)] = mk<T>(r.x, r.y);
        }
      } else {
        for (int n = threadIdx.x; n < M; n += THREADS) buf[padi<T>(t * M + n)] = mk<T>(T(0), T(0));
      }
    }
  } else {
    // all of a thread's loads are issued before any shared-memory store
    constexpr int PER = (LPB * M + THREADS - 1) / THREADS;
    cplx<T> v[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int idx = threadIdx.x + q * THREADS;
      const int t = idx / M, n = idx % M;
      const int line = line0 + t;
      v[q] = (idx < LPB * M && line < nlines) ? fwd_load<T, TI, MODE>(g, args, tt, tb, line, n) : mk<T>(T(0), T(0));
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int idx = threadIdx.x + q * THREADS;
      if (idx < LPB * M) buf[padi<T>(idx)] = v[q];
    }
  }
  __syncthreads();
  fft_static<T, M, -1, LPB, THREADS, 1, M, false, C::MAXR>(buf, tt.tw_m);
  constexpr int M1 = M + 1;
#pragma unroll 4
  for (int idx = threadIdx.x; idx < LPB * M1; idx += THREADS) {
    const int t = idx / M1, kx = idx % M1;
    const int line = line0 + t;
    if (line >= nlines) continue;
    const cplx<T> Zk = buf[padi<T>(t * M + (kx == M ? 0 : kx))];
    const cplx<T> Zc = conj(buf[padi<T>(t * M + (kx == 0 ? 0 : M - kx))]);
    st_c(spec + (size_t)line * g.pitch + kx, fwd_post(Zk, Zc, ldg_c(tt.tw_post + kx)));
  }
}

template <typename T, typename TO, int M, int MODE, bool ACC>
__global__ void __launch_bounds__(XTile<T, M>::THREADS, XTile<T, M>::MINB)
    k_inv_x_fast(Geometry g, Tables<T> tt, const cplx<T>* __restrict__ spec, TO* __restrict__ out, double scl,
                 int nlines, const double* __restrict__ dy, double* __restrict__ acc, PairArgs pair) {
  using C = XTile<T, M>;
  constexpr int LPB = C::LPB, THREADS = C::THREADS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
  const int line0 = blockIdx.x * LPB;
  {
    constexpr int PER = (LPB * M + THREADS - 1) / THREADS;
    cplx<T> Xk[PER], Xm[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int idx = threadIdx.x + q * THREADS;
      const int t = idx / M, kx = idx % M;
      const int line = line0 + t;
      Xk[q] = Xm[q] = mk<T>(T(0), T(0));
      if (idx < LPB * M && line < nlines) {
        const cplx<T>* row = spec + (size_t)line * g.pitch;
        Xk[q] = ld_c(row + kx);
        Xm[q] = ld_c(row + (M - kx));
      }
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int idx = threadIdx.x + q * THREADS;
      const int kx = idx % M;
      if (idx < LPB * M) buf[padi<T>(idx)] = inv_pre(kx, Xk[q], Xm[q], ldg_c(tt.tw_post + kx));
    }
  }
  __syncthreads();
  fft_static<T, M, 1, LPB, THREADS, 1, M, false, C::MAXR>(buf, tt.tw_m);
  const T s = T(scl);
  if constexpr (!ACC && MODE == INV_FINAL) {
    // refined pressure: the pair (hi, lo) of every element is loaded before any assembly
    constexpr int PER = (LPB * M + THREADS - 1) / THREADS;
    float2 h[PER], l[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int idx = threadIdx.x + q * THREADS;
      const int t = idx / M, n = idx % M;
      const int line = line0 + t;
      h[q] = l[q] = make_float2(0.f, 0.f);
      if (idx < LPB * M && line < nlines) {
        const size_t off = (size_t)line * g.nx + 2 * n;
        h[q] = *reinterpret_cast<const float2*>(pair.hi + off);
        if (pair.lo) l[q] = *reinterpret_cast<const float2*>(pair.lo + off);
      }
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int idx = threadIdx.x + q * THREADS;
      const int t = idx / M, n = idx % M;
      const int line = line0 + t;
      if (idx >= LPB * M || line >= nlines) continue;
      const cplx<T> z = buf[padi<T>(idx)];
      const size_t off = (size_t)line * g.nx + 2 * n;
      final_store(out + off, h[q], l[q], float(z.x * s), float(z.y * s));
    }
  } else if constexpr (!ACC) {
#pragma unroll 4
    for (int idx = threadIdx.x; idx < LPB * M; idx += THREADS) {
      const int t = idx / M, n = idx % M;
      const int line = line0 + t;
      if (line >= nlines) continue;
      const cplx<T> z = buf[padi<T>(idx)];
      const size_t off = (size_t)line * g.nx + 2 * n;
      inv_store<T, TO, MODE>(out + off, off, z.x * s, z.y * s, pair);
    }
  } else {
    // one warp per line: the line's dy-weighted sum is reduced with compensated sums
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NWARPS = THREADS / 32;
    double wsum = 0.0;
    for (int t = warp; t < LPB; t += NWARPS) {
      const int line = line0 + t;
      if (line >= nlines) break;
      T hs = T(0), hc = T(0);
#pragma unroll 8
      for (int n = lane; n < M; n += 32) {
        const cplx<T> z = buf[padi<T>(t * M + n)];
        const T x0 = z.x * s, x1 = z.y * s;
        const size_t off = (size_t)line * g.nx + 2 * n;
        inv_store<T, TO, MODE>(out + off, off, x0, x1, pair);
        acc_add(hs, hc, x0);
        acc_add(hs, hc, x1);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T os = __shfl_xor_sync(0xffffffffu, hs, o), oc = __shfl_xor_sync(0xffffffffu, hc, o);
        T e;
        if constexpr (sizeof(T) == 4) {
          two_sum(hs, os, hs, e);
        } else {
          hs += os;
          e = T(0);
        }
        hc += oc + e;
      }
      if (lane == 0) wsum += dy[line / g.nz] * ((double)hs + (double)hc);
    }
    if (lane == 0 && wsum != 0.0) atomicAdd(acc + 1, wsum);
  }
}

// ---- persistent forward x-transform with the next tile's input in flight -------------------
// A CTA walks tiles b, b + gridDim.x, ...; each tile's input lines are one contiguous stretch,
// which one thread copies into a shared-memory staging area with a single bulk asynchronous copy
// (the TMA engine, completion counted in bytes on an mbarrier).  The first FFT stage reads the
// staging area directly (packing or converting on the way), after which the copy of the next tile
// is issued, so it travels while this tile is transformed and stored.  The arithmetic is that of
// the single-tile kernels above.

template <typename TI, int M> struct XPipe {
  using X = XTile<float, M>;
  static constexpr int LPB = X::LPB, THREADS = X::THREADS;
  static constexpr int STAGE = LPB * 2 * M * (int)sizeof(TI);   // raw input lines
  static constexpr int SMEM = STAGE + padded_size<float>(LPB * M) * (int)sizeof(cplx<float>);
  static constexpr int MINB = 768 / THREADS > 0 ? 768 / THREADS : 1;   // <= 85 registers per thread
};

// Forward x-transform of a plain real field into the FP32 half spectrum.
template <typename TI, int M>
__global__ void __launch_bounds__(XPipe<TI, M>::THREADS, XPipe<TI, M>::MINB)
    k_fwd_x_pipe(Geometry g, FwdArgs args, Tables<float> tt, cplx<float>* __restrict__ spec, int lbeg, int nlines,
                 int* status) {
  using C = XPipe<TI, M>;
  constexpr int LPB = C::LPB, THREADS = C::THREADS;
  extern __shared__ __align__(128) unsigned char xpipe_smem[];
  __shared__ __align__(8) uint64_t bar;
  const TI* stage = reinterpret_cast<const TI*>(xpipe_smem);
  cplx<float>* buf = reinterpret_cast<cplx<float>*>(xpipe_smem + C::STAGE);
  const TI* in = reinterpret_cast<const TI*>(args.in);
  const TI sc = TI(args.in_scale);
  const int ntiles = (nlines - lbeg + LPB - 1) / LPB;
  auto issue = [&](int b) {
    if (threadIdx.x == 0) {
      const int l0 = lbeg + b * LPB;
      bulk_load(xpipe_smem, in + (size_t)l0 * g.nx, (unsigned)((size_t)min(LPB, nlines - l0) * g.nx * sizeof(TI)), &bar);
    }
  };
  if (threadIdx.x == 0) mbar_init(&bar);
  __syncthreads();
  if (blockIdx.x < ntiles && !g.selftest_wait) issue(blockIdx.x);
  unsigned parity = 0;
  for (int b = blockIdx.x; b < ntiles; b += gridDim.x, parity ^= 1u) {
    const int line0 = lbeg + b * LPB, nl = min(LPB, nlines - line0);
    // the tile has landed (or, uniformly for the CTA, the bounded wait gave up)
    if (!__syncthreads_and(mbar_wait(&bar, parity))) {
      if (threadIdx.x == 0) atomicExch(status, (int)DEV_TIMEOUT);
      return;
    }
    auto load = [&](int t, int n) -> cplx<float> {
      if (t >= nl) return mk<float>(0.f, 0.f);
      if constexpr (sizeof(TI) == 8) {
        const double2 v = *reinterpret_cast<const double2*>(stage + (size_t)t * g.nx + 2 * n);
        return mk<float>(f64_to_f32_trunc(v.x), f64_to_f32_trunc(v.y));
      } else {
        const float2 v = *reinterpret_cast<const float2*>(stage + (size_t)t * g.nx + 2 * n);
        return mk<float>(float(v.x * sc), float(v.y * sc));
      }
    };
    auto refill = [&]() {
      if (b + (int)gridDim.x < ntiles) issue(b + gridDim.x);
    };
    fft_static_from<float, M, -1, LPB, THREADS, 1, M, false, XTile<float, M>::MAXR>(buf, tt.tw_m, load, refill);
    constexpr int M1 = M + 1;
#pragma unroll 4
    for (int idx = threadIdx.x; idx < LPB * M1; idx += THREADS) {
      const int t = idx / M1, kx = idx % M1;
      if (t >= nl) continue;
      const cplx<float> Zk = buf[padi<float>(t * M + (kx == M ? 0 : kx))];
      const cplx<float> Zc = conj(buf[padi<float>(t * M + (kx == 0 ? 0 : M - kx))]);
      st_c(spec + (size_t)(line0 + t) * g.pitch + kx, fwd_post(Zk, Zc, ldg_c(tt.tw_post + kx)));
    }
  }
}

// Resident CTAs of a kernel on the whole GPU (queried once per kernel and shared-memory size).
template <typename K>
inline cudaError_t resident_grid(K kernel, int threads, int smem, int& grid) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> cache;
  cudaError_t e = ensure_smem_limit((const void*)kernel, (size_t)smem);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  auto key = std::make_pair((const void*)kernel, smem);
  auto it = cache.find(key);
  if (it != cache.end()) { grid = it->second; return cudaSuccess; }
  int dev = 0, sms = 0, per = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, (size_t)smem)) != cudaSuccess)
    return e;
  if (per < 1) return cudaErrorInvalidConfiguration;
  grid = sms * per;
  cache[key] = grid;
  return cudaSuccess;
}

template <typename K>
inline cudaError_t set_smem(K kernel, int smem) {
  return ensure_smem_limit((const void*)kernel, (size_t)smem);
}

// FP32 spectra of FP32 fields: the two-pass register kernels (k_fft_x_reg.cuh); the refinement
// residual (Nx/2 >= 256) too, with its residual formed warp by warp into shared memory first.
// For the plain FP64 right-hand side and the FP64 assembly of the refined pressure the Stockham
// kernels measured faster: those passes are latency-bound on their FP64 streams and want the
// finer-grained CTAs (two lines, 63-80 registers) that the register kernels do not give.
template <typename TI, int M>
cudaError_t launch_fwd_x_reg(const Geometry& g, const DevTables& tb, FwdMode mode, const FwdArgs& args,
                             cplx<float>* spec, cudaStream_t st) {
  using C = XReg<M>;
  const int nlines = g.ny * g.nz;
  const dim3 grid((nlines + C::LPB - 1) / C::LPB);
  cudaError_t e = cudaSuccess;
#define PP_FWDR(MODEV)                                                                  \
  {                                                                                     \
    auto k = k_fwd_x_reg<TI, M, MODEV>;                                                 \
    if ((e = set_smem(k, C::SMEM)) != cudaSuccess) return e;                            \
    k<<<grid, C::THREADS, C::SMEM, st>>>(g, args, tb.f, tb, spec, nlines);              \
  }
  switch (mode) {
    case FWD_PLAIN: PP_FWDR(FWD_PLAIN) break;
    case FWD_DIV: PP_FWDR(FWD_DIV) break;
    case FWD_GRADT: PP_FWDR(FWD_GRADT) break;
    default: return cudaErrorNotSupported;
  }
#undef PP_FWDR
  return cudaGetLastError();
}

template <typename TO, int M>
cudaError_t launch_inv_x_reg(const Geometry& g, const DevTables& tb, InvMode mode, const cplx<float>* spec, TO* out,
                             double scale, bool accumulate, cudaStream_t st, PairArgs pair) {
  using C = XReg<M>;
  const int nlines = g.ny * g.nz;
  const dim3 grid((nlines + C::LPB - 1) / C::LPB);
  cudaError_t e = cudaSuccess;
#define PP_INVR(MODEV, ACCV)                                                                       \
  {                                                                                                \
    auto k = k_inv_x_reg<TO, M, MODEV, ACCV>;                                                      \
    if ((e = set_smem(k, C::SMEM)) != cudaSuccess) return e;                                       \
    k<<<grid, C::THREADS, C::SMEM, st>>>(g, tb.f, spec, out, scale, nlines, tb.dy, tb.acc, pair); \
  }
  if (mode == INV_ACCUM) {
    if (accumulate) PP_INVR(INV_ACCUM, true) else PP_INVR(INV_ACCUM, false)
  } else if (mode == INV_STORE) {
    if (accumulate) PP_INVR(INV_STORE, true) else PP_INVR(INV_STORE, false)
  } else {
    return cudaErrorNotSupported;
  }
#undef PP_INVR
  return cudaGetLastError();
}

template <typename T, typename TI, int M>
cudaError_t launch_fwd_x_stockham(const Geometry& g, const DevTables& tb, const Tables<T>& tt, FwdMode mode,
                                  const FwdArgs& args, cplx<T>* spec, cudaStream_t st);

template <typename T, typename TI, int M>
cudaError_t launch_fwd_x_m(const Geometry& g, const DevTables& tb, const Tables<T>& tt, FwdMode mode,
                           const FwdArgs& args, cplx<T>* spec, cudaStream_t st) {
  if constexpr (sizeof(T) == 4 && sizeof(TI) == 4) {
    return launch_fwd_x_reg<TI, M>(g, tb, mode, args, spec, st);
  } else {
    return launch_fwd_x_stockham<T, TI, M>(g, tb, tt, mode, args, spec, st);
  }
}

// FP64 spectra and FP64 fields: the Stockham kernels above.
template <typename T, typename TI, int M>
cudaError_t launch_fwd_x_stockham(const Geometry& g, const DevTables& tb, const Tables<T>& tt, FwdMode mode,
                                  const FwdArgs& args, cplx<T>* spec, cudaStream_t st) {
  using C = XTile<T, M>;
  const int nlines = g.ny * g.nz;
  const dim3 grid((nlines + C::LPB - 1) / C::LPB);
  cudaError_t e = cudaSuccess;
#define PP_FWDF(MODEV)                                                                  \
  {                                                                                     \
    auto k = k_fwd_x_fast<T, TI, M, MODEV>;                                             \
    if ((e = set_smem(k, C::SMEM)) != cudaSuccess) return e;                            \
    k<<<grid, C::THREADS, C::SMEM, st>>>(g, args, tt, tb, spec, nlines);                \
  }
  if constexpr (sizeof(T) == 4 && sizeof(TI) == 8 && M >= 256 && M != 384) {
    // FP64 right-hand side into the FP32 spectrum: the input is the widest stream of the solve,
    // and keeping the next tile's lines in flight pays for the smaller CTA count (long lines:
    // tiles of 2-8 lines; Nx/2 = 384 spills and keeps the single-tile kernel; FP32 inputs, half
    // as wide, measured faster with the single-tile kernel)
    if (mode == FWD_PLAIN) {
      using P = XPipe<TI, M>;
      auto k = k_fwd_x_pipe<TI, M>;
      int rg = 0;
      if ((e = resident_grid(k, P::THREADS, P::SMEM, rg)) != cudaSuccess) return e;
      const int ntiles = (nlines + P::LPB - 1) / P::LPB;
      k<<<rg < ntiles ? rg : ntiles, P::THREADS, P::SMEM, st>>>(g, args, tt, spec, 0, nlines, tb.status);
      return cudaGetLastError();
    }
  }
  if constexpr (sizeof(T) == 4 && sizeof(TI) == 8 && M >= 256) {
    // refinement residual: warp-per-line residual into shared memory, then the register transform
    if (mode == FWD_RESID) {
      using R = XReg<M>;
      auto k = args.rin ? k_fwd_x_reg_resid<M, true> : k_fwd_x_reg_resid<M, false>;
      if ((e = set_smem(k, R::SMEM)) != cudaSuccess) return e;
      k<<<(nlines + R::LPB - 1) / R::LPB, R::THREADS, R::SMEM, st>>>(g, args, tt, tb, spec, nlines);
      return cudaGetLastError();
    }
  }
  if constexpr (sizeof(T) == sizeof(TI)) {
    switch (mode) {
      case FWD_PLAIN: PP_FWDF(FWD_PLAIN) break;
      case FWD_DIV: PP_FWDF(FWD_DIV) break;
      case FWD_GRADT: PP_FWDF(FWD_GRADT) break;
      default: return cudaErrorNotSupported;
    }
  } else {
    switch (mode) {
      case FWD_PLAIN: PP_FWDF(FWD_PLAIN) break;
      case FWD_RESID: PP_FWDF(FWD_RESID) break;
      default: return cudaErrorNotSupported;
    }
  }
#undef PP_FWDF
  return cudaGetLastError();
}

template <typename T, typename TO, int M>
cudaError_t launch_inv_x_stockham(const Geometry& g, const DevTables& tb, const Tables<T>& tt, InvMode mode,
                                  const cplx<T>* spec, TO* out, double scale, bool accumulate, cudaStream_t st,
                                  PairArgs pair) {
  using C = XTile<T, M>;
  const int nlines = g.ny * g.nz;
  const dim3 grid((nlines + C::LPB - 1) / C::LPB);
  cudaError_t e = cudaSuccess;
#define PP_INVF(MODEV, ACCV)                                                                     \
  {                                                                                              \
    auto k = k_inv_x_fast<T, TO, M, MODEV, ACCV>;                                                \
    if ((e = set_smem(k, C::SMEM)) != cudaSuccess) return e;                                     \
    k<<<grid, C::THREADS, C::SMEM, st>>>(g, tt, spec, out, scale, nlines, tb.dy, tb.acc, pair); \
  }
  if constexpr (sizeof(T) == sizeof(TO)) {
    if (mode == INV_FINAL) return cudaErrorNotSupported;
    if (mode == INV_ACCUM) {
      if (accumulate) PP_INVF(INV_ACCUM, true) else PP_INVF(INV_ACCUM, false)
    } else {
      if (accumulate) PP_INVF(INV_STORE, true) else PP_INVF(INV_STORE, false)
    }
  } else {
    if (mode != INV_FINAL) return cudaErrorNotSupported;
    if (accumulate) PP_INVF(INV_FINAL, true) else PP_INVF(INV_FINAL, false)
  }
#undef PP_INVF
  return cudaGetLastError();
}

template <typename T, typename TO, int M>
cudaError_t launch_inv_x_m(const Geometry& g, const DevTables& tb, const Tables<T>& tt, InvMode mode,
                           const cplx<T>* spec, TO* out, double scale, bool accumulate, cudaStream_t st,
                           PairArgs pair) {
  if constexpr (sizeof(T) == 4 && sizeof(TO) == 4) {
    return launch_inv_x_reg<TO, M>(g, tb, mode, spec, out, scale, accumulate, st, pair);
  } else {
    return launch_inv_x_stockham<T, TO, M>(g, tb, tt, mode, spec, out, scale, accumulate, st, pair);
  }
}

#define PP_X_SIZES(F) F(16) F(32) F(48) F(64) F(96) F(128) F(192) F(256) F(384) F(512) F(768) F(1024)

template <typename T, typename TI>
cudaError_t launch_fwd_x_fast_impl(const Geometry& g, const DevTables& tb, const Tables<T>& tt, FwdMode mode,
                                   const FwdArgs& args, cplx<T>* spec, cudaStream_t st) {
  // the per-line residual addresses its neighbour lines by 32-bit offsets
  if (mode == FWD_RESID && (long long)g.nx * g.nz >= (1LL << 31)) return cudaErrorNotSupported;
  switch (g.M) {
#define PP_CASE(MV) \
  case MV: return launch_fwd_x_m<T, TI, MV>(g, tb, tt, mode, args, spec, st);
    PP_X_SIZES(PP_CASE)
#undef PP_CASE
    default: return cudaErrorNotSupported;
  }
}

template <typename T, typename TO>
cudaError_t launch_inv_x_fast_impl(const Geometry& g, const DevTables& tb, const Tables<T>& tt, InvMode mode,
                                   const cplx<T>* spec, TO* out, double scale, bool accumulate, cudaStream_t st,
                                   PairArgs pair) {
  switch (g.M) {
#define PP_CASE(MV) \
  case MV: return launch_inv_x_m<T, TO, MV>(g, tb, tt, mode, spec, out, scale, accumulate, st, pair);
    PP_X_SIZES(PP_CASE)
#undef PP_CASE
    default: return cudaErrorNotSupported;
  }
}

}  // namespace pp
