// Per-line pieces of the x-transform kernels, shared by the generic and the specialised ones:
// the fused right-hand-side producers (plain field, divergence of Eq. 7, refinement residual,
// adjoint G^T g / dy), the even/odd packing of a real line into half-length complex data and
// its inverse, and compensated sums.
#pragma once

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

// Right-hand side at cells (j, k, 2n) and (j, k, 2n+1) of line = j * nz + k, packed as one
// complex value for the half-length transform.
template <typename T, typename TI, int MODE>
__device__ __forceinline__ cplx<T> fwd_load(const Geometry& g, const FwdArgs& args, const Tables<T>& tt,
                                            const DevTables& tb, int line, int n) {
  const int j = line / g.nz, k = line - j * g.nz;
  const int i0 = 2 * n;
  if constexpr (MODE == FWD_PLAIN) {
    TI a, b;
    RealIO<TI>::load2(reinterpret_cast<const TI*>(args.in) + (size_t)line * g.nx + i0, a, b);
    const TI s = TI(args.in_scale);
    return mk<T>(T(a * s), T(b * s));
  } else if constexpr (MODE == FWD_DIV) {
    TI f0, f1;
    const TI s = TI(args.in_scale);
    divergence_pair<TI>(g, reinterpret_cast<const TI*>(args.u), reinterpret_cast<const TI*>(args.v),
                        reinterpret_cast<const TI*>(args.w), j, k, i0, TI(1.0 / g.dx), TI(tt.inv_dy[j]),
                        TI(1.0 / g.dz), f0, f1);
    return mk<T>(T(f0 * s), T(f1 * s));
  } else if constexpr (MODE == FWD_GRADT) {
    TI f0, f1;
    gradT_pair<TI>(g, reinterpret_cast<const TI*>(args.u), reinterpret_cast<const TI*>(args.v),
                   reinterpret_cast<const TI*>(args.w), j, k, i0, TI(1.0 / g.dx), TI(1.0 / g.dz),
                   TI(tt.inv_h[j]), TI(tt.inv_h[j + 1]), TI(tt.inv_dy[j]), f0, f1);
    return mk<T>(T(f0), T(f1));
  } else {  // FWD_RESID (FP64 operands)
    double r0, r1;
    residual_pair(g, reinterpret_cast<const double*>(args.in), reinterpret_cast<const double*>(args.p), j, k, i0,
                  1.0 / (g.dx * g.dx), 1.0 / (g.dz * g.dz), tb.d.a[j], tb.d.c[j], tb.acc[0], r0, r1);
    return mk<T>(T(r0), T(r1));
  }
}

// Unpack bin kx (0..M) of a real line from the half-length transform Z (even/odd split):
// X_k = (Z_k + conj Z_{M-k}) / 2 - i W^k (Z_k - conj Z_{M-k}) / 2,  W = e^{-2 pi i / Nx}.
template <typename T>
__device__ __forceinline__ cplx<T> fwd_post(cplx<T> Zk, cplx<T> ZmConj, cplx<T> W) {
  const cplx<T> s = Zk + ZmConj, d = Zk - ZmConj;
  return scale(s - mul_i(cmul(W, d), 1), T(0.5));
}

// Pack bins k and M-k of a Hermitian half spectrum for the half-length inverse transform
// (k = 0 uses the real parts of bins 0 and M only).
template <typename T>
__device__ __forceinline__ cplx<T> inv_pre(int kx, cplx<T> Xk, cplx<T> Xm, cplx<T> W) {
  if (kx == 0) return mk<T>(Xk.x + Xm.x, Xk.x - Xm.x);
  const cplx<T> Xc = conj(Xm);
  const cplx<T> s = Xk + Xc, d = Xk - Xc;
  return s + mul_i(cmulc(d, W), 1);   // i conj(W) (Xk - Xc)
}

}  // namespace pp
