// Transform kernels of the pressure solve (Eq. 9; steps (2), (4), (6), (8) of Sec. 3.2).
//
//  k_fwd_x : per x-line (j, k), Nx real values -> Nx/2+1 complex (e^{-2 pi i kx x / Nx}).
//            The real line is packed as Nx/2 complex values, transformed by the Stockham
//            routine and unpacked with the standard even/odd split.  The load is fused with
//            the producer of the right-hand side: a plain field, the divergence of Eq. 7
//            (projection), the residual f - L_h p (refinement) or G^T g / dy (adjoint).
//  k_fft_z : per (j, kx), the Nz-point complex transform along z (forward or inverse) on a
//            tile of W adjacent kx columns; this replaces the x->y pencil transposes.
//  k_inv_x : per line, Nx/2+1 complex -> Nx real, scaled by 1/(Nx Nz); the imaginary parts of
//            the kx = 0 and kx = Nx/2 bins are ignored.  Epilogue: store or accumulate.
#include "xline.cuh"

namespace pp {

template <typename T, typename TI, int MODE>
__global__ void __launch_bounds__(256) k_fwd_x(Geometry g, FwdArgs args, Tables<T> tt, DevTables tb, FftFactors fm,
                                               cplx<T>* __restrict__ spec, int lpb, int nlines) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int M = fm.L;
  cplx<T>* buf0 = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* buf1 = buf0 + (size_t)lpb * M;
  const int line0 = blockIdx.x * lpb;
  for (int idx = threadIdx.x; idx < lpb * M; idx += blockDim.x) {
    const int t = idx / M, n = idx - t * M;
    const int line = line0 + t;
    cplx<T> z = mk<T>(T(0), T(0));
    if (line < nlines) z = fwd_load<T, TI, MODE>(g, args, tt, tb, line, n);
    buf0[idx] = z;
  }
  __syncthreads();
  cplx<T>* res = fft_smem<T, -1>(buf0, buf1, fm, lpb, 1, M, false, tt.tw_m);
  const int M1 = M + 1;
  for (int idx = threadIdx.x; idx < lpb * M1; idx += blockDim.x) {
    const int t = idx / M1, kx = idx - t * M1;
    const int line = line0 + t;
    if (line >= nlines) continue;
    const cplx<T> Zk = res[t * M + (kx == M ? 0 : kx)];
    const cplx<T> Zc = conj(res[t * M + (kx == 0 ? 0 : M - kx)]);
    st_c(spec + (size_t)line * g.pitch + kx, fwd_post(Zk, Zc, ldg_c(tt.tw_post + kx)));
  }
}

template <typename T, typename TO, int MODE, bool ACC>
__global__ void __launch_bounds__(256) k_inv_x(Geometry g, Tables<T> tt, FftFactors fm,
                                               const cplx<T>* __restrict__ spec, TO* __restrict__ out, double scl,
                                               int lpb, int nlines, const double* __restrict__ dy,
                                               double* __restrict__ acc, PairArgs pair) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int M = fm.L;
  cplx<T>* buf0 = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* buf1 = buf0 + (size_t)lpb * M;
  const int line0 = blockIdx.x * lpb;
  for (int idx = threadIdx.x; idx < lpb * M; idx += blockDim.x) {
    const int t = idx / M, kx = idx - t * M;
    const int line = line0 + t;
    cplx<T> Z = mk<T>(T(0), T(0));
    if (line < nlines) {
      const cplx<T>* row = spec + (size_t)line * g.pitch;
      Z = inv_pre(kx, ld_c(row + kx), ld_c(row + (M - kx)), ldg_c(tt.tw_post + kx));
    }
    buf0[idx] = Z;
  }
  __syncthreads();
  cplx<T>* res = fft_smem<T, 1>(buf0, buf1, fm, lpb, 1, M, false, tt.tw_m);
  const T s = T(scl);
  // Epilogue: one warp per line, so each line's weighted sum can be reduced in the warp.
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  double wsum = 0.0;
  for (int t = warp; t < lpb; t += nwarps) {
    const int line = line0 + t;
    if (line >= nlines) break;
    T hs = T(0), hc = T(0);
    for (int n = lane; n < M; n += 32) {
      const cplx<T> z = res[t * M + n];
      const T x0 = z.x * s, x1 = z.y * s;
      const size_t off = (size_t)line * g.nx + 2 * n;
      inv_store<T, TO, MODE>(out + off, off, x0, x1, pair);
      if (ACC) {
        acc_add(hs, hc, x0);
        acc_add(hs, hc, x1);
      }
    }
    if (ACC) {
      // compensated warp reduction of (hs, hc)
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
  }
  if (ACC && lane == 0 && wsum != 0.0) atomicAdd(acc + 1, wsum);
}

template <typename T, int SIGN>
__global__ void __launch_bounds__(256) k_fft_z(Geometry g, Tables<T> tt, FftFactors fz, cplx<T>* __restrict__ spec,
                                               int W) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Nz = fz.L;
  cplx<T>* buf0 = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* buf1 = buf0 + (size_t)Nz * W;
  const int j = blockIdx.y;
  const int kx0 = blockIdx.x * W;
  cplx<T>* plane = spec + (size_t)j * Nz * g.pitch;
  for (int idx = threadIdx.x; idx < Nz * W; idx += blockDim.x) {
    const int n = idx / W, c = idx - n * W;
    const int col = kx0 + c;
    buf0[idx] = col < g.ncols ? ld_c(plane + (size_t)n * g.pitch + col) : mk<T>(T(0), T(0));
  }
  __syncthreads();
  cplx<T>* res = fft_smem<T, SIGN>(buf0, buf1, fz, W, W, 1, true, tt.tw_z);
  for (int idx = threadIdx.x; idx < Nz * W; idx += blockDim.x) {
    const int n = idx / W, c = idx - n * W;
    const int col = kx0 + c;
    if (col < g.ncols) st_c(plane + (size_t)n * g.pitch + col, res[idx]);
  }
}

// ------------------------------------------------------------------------------ launchers
static int lines_per_cta(int M) {
  int lpb = 2048 / M;
  return lpb < 1 ? 1 : lpb;
}

template <typename T> static const Tables<T>& tabs(const DevTables& tb);
template <> const Tables<double>& tabs<double>(const DevTables& tb) { return tb.d; }
template <> const Tables<float>& tabs<float>(const DevTables& tb) { return tb.f; }

template <typename K>
static cudaError_t prep(K kernel, size_t smem) {
  return ensure_smem_limit((const void*)kernel, smem);
}

template <typename T, typename TI>
cudaError_t launch_fwd_x(const Geometry& g, const DevTables& tb, const FftFactors& fm, FwdMode mode,
                         const FwdArgs& args, cplx<T>* spec, cudaStream_t st) {
  if (!g.generic_fft) {
    cudaError_t ef;
    if constexpr (sizeof(T) == 8) ef = launch_fwd_x_fast_dd(g, tb, mode, args, (cplx<double>*)spec, st);
    else if constexpr (sizeof(TI) == 4) ef = launch_fwd_x_fast_ff(g, tb, mode, args, (cplx<float>*)spec, st);
    else ef = launch_fwd_x_fast_fd(g, tb, mode, args, (cplx<float>*)spec, st);
    if (ef != cudaErrorNotSupported) return ef;
  }
  const int nlines = g.ny * g.nz;
  const int lpb = lines_per_cta(fm.L);
  const size_t smem = 2 * (size_t)lpb * fm.L * sizeof(cplx<T>);
  const dim3 grid((nlines + lpb - 1) / lpb);
  cudaError_t e = cudaSuccess;
#define PP_FWD(MODEV)                                                                           \
  {                                                                                             \
    auto kern = k_fwd_x<T, TI, MODEV>;                                                          \
    if ((e = prep(kern, smem)) != cudaSuccess) return e;                                        \
    kern<<<grid, 256, smem, st>>>(g, args, tabs<T>(tb), tb, fm, spec, lpb, nlines);             \
  }
  switch (mode) {
    case FWD_PLAIN: PP_FWD(FWD_PLAIN) break;
    case FWD_DIV: PP_FWD(FWD_DIV) break;
    case FWD_GRADT: PP_FWD(FWD_GRADT) break;
    case FWD_RESID: PP_FWD(FWD_RESID) break;
  }
#undef PP_FWD
  return cudaGetLastError();
}

template <typename T, typename TO>
cudaError_t launch_inv_x(const Geometry& g, const DevTables& tb, const FftFactors& fm, InvMode mode,
                         const cplx<T>* spec, TO* out, double scale, bool accumulate, cudaStream_t st,
                         PairArgs pair) {
  if (!g.generic_fft) {
    cudaError_t ef;
    if constexpr (sizeof(T) == 8)
      ef = launch_inv_x_fast_dd(g, tb, mode, (const cplx<double>*)spec, (double*)out, scale, accumulate, st, pair);
    else if constexpr (sizeof(TO) == 4)
      ef = launch_inv_x_fast_ff(g, tb, mode, (const cplx<float>*)spec, (float*)out, scale, accumulate, st, pair);
    else
      ef = launch_inv_x_fast_fd(g, tb, mode, (const cplx<float>*)spec, (double*)out, scale, accumulate, st, pair);
    if (ef != cudaErrorNotSupported) return ef;
  }
  const int nlines = g.ny * g.nz;
  const int lpb = lines_per_cta(fm.L);
  const size_t smem = 2 * (size_t)lpb * fm.L * sizeof(cplx<T>);
  const dim3 grid((nlines + lpb - 1) / lpb);
  cudaError_t e;
#define PP_INV(MODEV, ACCV)                                                                               \
  {                                                                                                       \
    auto kern = k_inv_x<T, TO, MODEV, ACCV>;                                                              \
    if ((e = prep(kern, smem)) != cudaSuccess) return e;                                                  \
    kern<<<grid, 256, smem, st>>>(g, tabs<T>(tb), fm, spec, out, scale, lpb, nlines, tb.dy, tb.acc, pair); \
  }
  if (mode == INV_FINAL) {
    if constexpr (sizeof(T) == 4 && sizeof(TO) == 8) {
      if (accumulate) PP_INV(INV_FINAL, true) else PP_INV(INV_FINAL, false)
    } else {
      return cudaErrorInvalidValue;
    }
  } else if (mode == INV_ACCUM) {
    if (accumulate) PP_INV(INV_ACCUM, true) else PP_INV(INV_ACCUM, false)
  } else {
    if (accumulate) PP_INV(INV_STORE, true) else PP_INV(INV_STORE, false)
  }
#undef PP_INV
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fft_z(const Geometry& g, const DevTables& tb, const FftFactors& fz, int sign, cplx<T>* spec,
                         cudaStream_t st) {
  if (!g.generic_fft) {
    const cudaError_t ef = launch_fft_z_fast<T>(g, tabs<T>(tb), sign, spec, st);
    if (ef != cudaErrorNotSupported) return ef;
  }
  int W = (int)(64 / sizeof(cplx<T>));           // 64-byte row segments
  while (W * fz.L < 2048 && W < 32) W *= 2;       // small Nz: widen the tile
  if (W > g.ncols) W = g.ncols;
  const size_t smem = 2 * (size_t)W * fz.L * sizeof(cplx<T>);
  const dim3 grid((g.ncols + W - 1) / W, g.ny);
  cudaError_t e;
  if (sign < 0) {
    auto kern = k_fft_z<T, -1>;
    if ((e = prep(kern, smem)) != cudaSuccess) return e;
    kern<<<grid, 256, smem, st>>>(g, tabs<T>(tb), fz, spec, W);
  } else {
    auto kern = k_fft_z<T, 1>;
    if ((e = prep(kern, smem)) != cudaSuccess) return e;
    kern<<<grid, 256, smem, st>>>(g, tabs<T>(tb), fz, spec, W);
  }
  return cudaGetLastError();
}

template cudaError_t launch_fwd_x<double, double>(const Geometry&, const DevTables&, const FftFactors&, FwdMode,
                                                  const FwdArgs&, cplx<double>*, cudaStream_t);
template cudaError_t launch_fwd_x<float, float>(const Geometry&, const DevTables&, const FftFactors&, FwdMode,
                                                const FwdArgs&, cplx<float>*, cudaStream_t);
template cudaError_t launch_fwd_x<float, double>(const Geometry&, const DevTables&, const FftFactors&, FwdMode,
                                                 const FwdArgs&, cplx<float>*, cudaStream_t);
template cudaError_t launch_inv_x<double, double>(const Geometry&, const DevTables&, const FftFactors&, InvMode,
                                                  const cplx<double>*, double*, double, bool, cudaStream_t,
                                                  PairArgs);
template cudaError_t launch_inv_x<float, float>(const Geometry&, const DevTables&, const FftFactors&, InvMode,
                                                const cplx<float>*, float*, double, bool, cudaStream_t,
                                                  PairArgs);
template cudaError_t launch_inv_x<float, double>(const Geometry&, const DevTables&, const FftFactors&, InvMode,
                                                 const cplx<float>*, double*, double, bool, cudaStream_t,
                                                  PairArgs);
template cudaError_t launch_fft_z<double>(const Geometry&, const DevTables&, const FftFactors&, int, cplx<double>*,
                                          cudaStream_t);
template cudaError_t launch_fft_z<float>(const Geometry&, const DevTables&, const FftFactors&, int, cplx<float>*,
                                         cudaStream_t);

}  // namespace pp
