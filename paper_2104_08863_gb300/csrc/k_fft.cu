// Transform kernels of the pressure solve (Eq. 9; steps (2), (4), (6), (8) of Sec. 3.1).
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
#include "internal.h"

namespace pp {

template <typename T> struct RealIO;
template <> struct RealIO<double> {
  static __device__ __forceinline__ void load2(const double* p, double& a, double& b) {
    double2 v = *reinterpret_cast<const double2*>(p); a = v.x; b = v.y;
  }
  static __device__ __forceinline__ void store2(double* p, double a, double b) {
    *reinterpret_cast<double2*>(p) = make_double2(a, b);
  }
};
template <> struct RealIO<float> {
  static __device__ __forceinline__ void load2(const float* p, float& a, float& b) {
    float2 v = *reinterpret_cast<const float2*>(p); a = v.x; b = v.y;
  }
  static __device__ __forceinline__ void store2(float* p, float a, float b) {
    *reinterpret_cast<float2*>(p) = make_float2(a, b);
  }
};

// Divergence (Eq. 7) at cells (j, k, i) and (j, k, i+1); TI arithmetic.
template <typename TI>
__device__ __forceinline__ void divergence_pair(const Geometry& g, const TI* __restrict__ u,
                                                const TI* __restrict__ v, const TI* __restrict__ w, int j, int k,
                                                int i0, TI inv_dx, TI inv_dy, TI inv_dz, TI& f0, TI& f1) {
  const size_t nx = g.nx;
  const size_t row = ((size_t)j * g.nz + k) * nx;
  const TI* ur = u + row;
  const TI ui0 = ur[i0], ui1 = ur[i0 + 1], ui2 = ur[(i0 + 2) % g.nx];
  const TI* vlo = v + row;
  const TI* vhi = v + row + (size_t)g.nz * nx;
  const TI* w0 = w + row;
  const TI* w1 = w + ((size_t)j * g.nz + (k + 1 == g.nz ? 0 : k + 1)) * nx;
  f0 = (ui1 - ui0) * inv_dx + (vhi[i0] - vlo[i0]) * inv_dy + (w1[i0] - w0[i0]) * inv_dz;
  f1 = (ui2 - ui1) * inv_dx + (vhi[i0 + 1] - vlo[i0 + 1]) * inv_dy + (w1[i0 + 1] - w0[i0 + 1]) * inv_dz;
}

// (G^T g)_{jki} / dy_j at cells (j,k,i0) and (j,k,i0+1) (adjoint right-hand side).
template <typename TI>
__device__ __forceinline__ void gradT_pair(const Geometry& g, const TI* __restrict__ gu, const TI* __restrict__ gv,
                                           const TI* __restrict__ gw, int j, int k, int i0, TI inv_dx, TI inv_dz,
                                           TI inv_hj, TI inv_hj1, TI inv_dy, TI& f0, TI& f1) {
  const size_t nx = g.nx;
  const size_t row = ((size_t)j * g.nz + k) * nx;
  const TI* ur = gu + row;
  const TI u0 = ur[i0], u1 = ur[i0 + 1], u2 = ur[(i0 + 2) % g.nx];
  const TI* w0 = gw + row;
  const TI* w1 = gw + ((size_t)j * g.nz + (k + 1 == g.nz ? 0 : k + 1)) * nx;
  const TI* vlo = gv + row;                         // face j (bottom of cell j)
  const TI* vhi = gv + row + (size_t)g.nz * nx;     // face j+1
  TI ty0 = TI(0), ty1 = TI(0);
  if (j >= 1) { ty0 += vlo[i0] * inv_hj; ty1 += vlo[i0 + 1] * inv_hj; }
  if (j + 1 <= g.ny - 1) { ty0 -= vhi[i0] * inv_hj1; ty1 -= vhi[i0 + 1] * inv_hj1; }
  f0 = ((u0 - u1) * inv_dx + (w0[i0] - w1[i0]) * inv_dz + ty0) * inv_dy;
  f1 = ((u1 - u2) * inv_dx + (w0[i0 + 1] - w1[i0 + 1]) * inv_dz + ty1) * inv_dy;
}

// (f - <f>) - L_h p at cells (j,k,i0), (j,k,i0+1), FP64 (refinement residual).  Removing the
// mean of f here keeps the FP32 transform of the residual free of a large constant whose
// rounding noise would otherwise leak into the weakly damped low modes at every step.
__device__ __forceinline__ void residual_pair(const Geometry& g, const double* __restrict__ f,
                                              const double* __restrict__ p, int j, int k, int i0, double idx2,
                                              double idz2, double aj, double cj, double fmean, double& r0,
                                              double& r1) {
  const size_t nx = g.nx;
  const size_t row = ((size_t)j * g.nz + k) * nx;
  const double* pr = p + row;
  const double* pkm = p + ((size_t)j * g.nz + (k == 0 ? g.nz - 1 : k - 1)) * nx;
  const double* pkp = p + ((size_t)j * g.nz + (k + 1 == g.nz ? 0 : k + 1)) * nx;
  const int im = i0 == 0 ? g.nx - 1 : i0 - 1;
  const int ip = i0 + 2 == g.nx ? 0 : i0 + 2;
  const double pm = pr[im], p0 = pr[i0], p1 = pr[i0 + 1], pp = pr[ip];
  double l0 = (pm - 2.0 * p0 + p1) * idx2 + (pkm[i0] - 2.0 * p0 + pkp[i0]) * idz2;
  double l1 = (p0 - 2.0 * p1 + pp) * idx2 + (pkm[i0 + 1] - 2.0 * p1 + pkp[i0 + 1]) * idz2;
  if (j >= 1) {
    const double* pl = pr - (size_t)g.nz * nx;
    l0 += aj * (pl[i0] - p0);
    l1 += aj * (pl[i0 + 1] - p1);
  }
  if (j + 1 <= g.ny - 1) {
    const double* pu = pr + (size_t)g.nz * nx;
    l0 += cj * (pu[i0] - p0);
    l1 += cj * (pu[i0 + 1] - p1);
  }
  r0 = (f[row + i0] - fmean) - l0;
  r1 = (f[row + i0 + 1] - fmean) - l1;
}

template <typename T, typename TI, int MODE>
__global__ void __launch_bounds__(256) k_fwd_x(Geometry g, FwdArgs args, Tables<T> tt, DevTables tb, FftFactors fm,
                                               cplx<T>* __restrict__ spec, int lpb, int nlines) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int M = fm.L;
  cplx<T>* buf0 = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* buf1 = buf0 + (size_t)lpb * M;
  const int line0 = blockIdx.x * lpb;
  const TI inv_dx = TI(1.0 / g.dx), inv_dz = TI(1.0 / g.dz);
  for (int idx = threadIdx.x; idx < lpb * M; idx += blockDim.x) {
    const int t = idx / M, n = idx - t * M;
    const int line = line0 + t;
    cplx<T> z = mk<T>(T(0), T(0));
    if (line < nlines) {
      const int j = line / g.nz, k = line - j * g.nz;
      const int i0 = 2 * n;
      if (MODE == FWD_PLAIN) {
        TI a, b;
        RealIO<TI>::load2(reinterpret_cast<const TI*>(args.in) + (size_t)line * g.nx + i0, a, b);
        const TI s = TI(args.in_scale);
        z = mk<T>(T(a * s), T(b * s));
      } else if (MODE == FWD_DIV) {
        TI f0, f1;
        const TI inv_dy = TI(tt.inv_dy[j]);
        divergence_pair<TI>(g, reinterpret_cast<const TI*>(args.u), reinterpret_cast<const TI*>(args.v),
                            reinterpret_cast<const TI*>(args.w), j, k, i0, inv_dx, inv_dy, inv_dz, f0, f1);
        const TI s = TI(args.in_scale);
        z = mk<T>(T(f0 * s), T(f1 * s));
      } else if (MODE == FWD_GRADT) {
        TI f0, f1;
        const TI inv_hj = TI(tt.inv_h[j]);        // 0 on the walls
        const TI inv_hj1 = TI(tt.inv_h[j + 1]);
        const TI inv_dy = TI(tt.inv_dy[j]);
        gradT_pair<TI>(g, reinterpret_cast<const TI*>(args.u), reinterpret_cast<const TI*>(args.v),
                       reinterpret_cast<const TI*>(args.w), j, k, i0, inv_dx, inv_dz, inv_hj, inv_hj1, inv_dy, f0,
                       f1);
        z = mk<T>(T(f0), T(f1));
      } else {  // FWD_RESID (FP64 operands)
        double r0, r1;
        const double idx2 = 1.0 / (g.dx * g.dx), idz2 = 1.0 / (g.dz * g.dz);
        residual_pair(g, reinterpret_cast<const double*>(args.in), reinterpret_cast<const double*>(args.p), j, k,
                      i0, idx2, idz2, tb.d.a[j], tb.d.c[j], tb.acc[0], r0, r1);
        z = mk<T>(T(r0), T(r1));
      }
    }
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
    const cplx<T> W = ldg_c(tt.tw_post + kx);
    const cplx<T> s = Zk + Zc, d = Zk - Zc;
    const cplx<T> X = scale(s - mul_i(cmul(W, d), 1), T(0.5));
    st_c(spec + (size_t)line * g.pitch + kx, X);
  }
}

// Error-free sum of two floats (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}
// Compensated accumulation (s, c) += x.
__device__ __forceinline__ void acc_add(float& s, float& c, float x) {
  float e;
  two_sum(s, x, s, e);
  c += e;
}
__device__ __forceinline__ void acc_add(double& s, double& c, double x) {
  s += x;
  (void)c;
}

template <typename T, typename TO, int MODE, bool ACC>
__global__ void __launch_bounds__(256) k_inv_x(Geometry g, Tables<T> tt, FftFactors fm,
                                               const cplx<T>* __restrict__ spec, TO* __restrict__ out, double scl,
                                               int lpb, int nlines, const double* __restrict__ dy,
                                               double* __restrict__ acc) {
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
      const cplx<T> Xk = ld_c(row + kx);
      const cplx<T> Xm = ld_c(row + (M - kx));
      if (kx == 0) {
        Z = mk<T>(Xk.x + Xm.x, Xk.x - Xm.x);
      } else {
        const cplx<T> Xc = conj(Xm);
        const cplx<T> s = Xk + Xc, d = Xk - Xc;
        const cplx<T> W = ldg_c(tt.tw_post + kx);
        Z = s + mul_i(cmulc(d, W), 1);   // i conj(W) (Xk - Xc)
      }
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
      TO* o = out + (size_t)line * g.nx + 2 * n;
      if (MODE == INV_ACCUM) {
        TO a, b;
        RealIO<TO>::load2(o, a, b);
        RealIO<TO>::store2(o, a + TO(x0), b + TO(x1));
      } else {
        RealIO<TO>::store2(o, TO(x0), TO(x1));
      }
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
  if (smem > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

template <typename T, typename TI>
cudaError_t launch_fwd_x(const Geometry& g, const DevTables& tb, const FftFactors& fm, FwdMode mode,
                         const FwdArgs& args, cplx<T>* spec, cudaStream_t st) {
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
                         const cplx<T>* spec, TO* out, double scale, bool accumulate, cudaStream_t st) {
  const int nlines = g.ny * g.nz;
  const int lpb = lines_per_cta(fm.L);
  const size_t smem = 2 * (size_t)lpb * fm.L * sizeof(cplx<T>);
  const dim3 grid((nlines + lpb - 1) / lpb);
  cudaError_t e;
#define PP_INV(MODEV, ACCV)                                                                               \
  {                                                                                                       \
    auto kern = k_inv_x<T, TO, MODEV, ACCV>;                                                              \
    if ((e = prep(kern, smem)) != cudaSuccess) return e;                                                  \
    kern<<<grid, 256, smem, st>>>(g, tabs<T>(tb), fm, spec, out, scale, lpb, nlines, tb.dy, tb.acc);     \
  }
  if (mode == INV_ACCUM) {
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
  {
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
                                                  const cplx<double>*, double*, double, bool, cudaStream_t);
template cudaError_t launch_inv_x<float, float>(const Geometry&, const DevTables&, const FftFactors&, InvMode,
                                                const cplx<float>*, float*, double, bool, cudaStream_t);
template cudaError_t launch_inv_x<float, double>(const Geometry&, const DevTables&, const FftFactors&, InvMode,
                                                 const cplx<float>*, double*, double, bool, cudaStream_t);
template cudaError_t launch_fft_z<double>(const Geometry&, const DevTables&, const FftFactors&, int, cplx<double>*,
                                          cudaStream_t);
template cudaError_t launch_fft_z<float>(const Geometry&, const DevTables&, const FftFactors&, int, cplx<float>*,
                                         cudaStream_t);

}  // namespace pp
