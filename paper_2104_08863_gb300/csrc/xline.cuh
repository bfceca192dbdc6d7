// Per-line pieces of the x-transform kernels, shared by the generic and the specialised ones:
// the fused right-hand-side producers (plain field, divergence of Eq. 7, refinement residual,
// adjoint G^T g / dy), the even/odd packing of a real line into half-length complex data and
// its inverse, and compensated sums.
#pragma once

#include "df2.cuh"
#include "fpconv.cuh"
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

// Refinement residual r = (f - <f>) - L_h p at cells (j,k,i0) and (j,k,i0+1), where f is the
// FP64 right-hand side and p the first solve's FP32 pressure hi; with a stored residual rin of
// the same solve (the first correction's, an FP32 pair per cell) a later correction forms
// r = rin - L_h lo instead, lo the FP32 sum of the corrections so far (by linearity the same
// f - <f> - L_h (hi + lo)).  Removing <f> keeps the FP32 transform of r free of a large constant
// whose rounding noise would otherwise leak into the weakly damped low modes at every step.
// L_h p is formed in double-float arithmetic on FP32 units: neighbour differences of the FP32
// field are exact (TwoDiff; near the walls the stencil terms cancel strongly, so plain FP32
// differences would floor the refinement), products with the double-float stencil coefficients
// recover their rounding error with FMAs, and the sums carry a compensation term, so r is
// accurate to ~2^-47 of the stencil terms.
template <typename TT>
__device__ __forceinline__ void residual_pair_df(const Geometry& g, const FwdArgs& args, const TT& tt,
                                                 const DevTables& tb, int j, int k, int i0, float& r0, float& r1) {
  const size_t nx = g.nx, plane = (size_t)g.nz * nx;
  const size_t row = ((size_t)j * g.nz + k) * nx;
  const size_t rkm = ((size_t)j * g.nz + (k == 0 ? g.nz - 1 : k - 1)) * nx;
  const size_t rkp = ((size_t)j * g.nz + (k + 1 == g.nz ? 0 : k + 1)) * nx;
  const int im = i0 == 0 ? g.nx - 1 : i0 - 1;
  const int ip = i0 + 2 == g.nx ? 0 : i0 + 2;
  const bool has_lo = j >= 1, has_hi = j + 1 <= g.ny - 1;
  const df cx{args.idx2h, args.idx2l}, cz{args.idz2h, args.idz2l};
  const df ca{tt.a[j], tt.a_lo[j]}, cc{tt.c[j], tt.c_lo[j]};
  float mh, ml;
  f64_split(tb.acc[0], mh, ml);
  const float* P = reinterpret_cast<const float*>(args.p);
  const double* f = reinterpret_cast<const double*>(args.in);
  const float2* rin = reinterpret_cast<const float2*>(args.rin);
  float2* rout = reinterpret_cast<float2*>(args.rout);
  // neighbour difference d(n) = p_n - p_c, exact as a double-float
  auto diff = [&](size_t n, size_t o) -> df { return two_diff_df(P[n], P[o]); };
  float out[2];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const size_t o = row + i0 + c;
    const size_t xm = row + (c == 0 ? im : i0), xp = row + (c == 0 ? i0 + 1 : ip);
    df L = df_mul(df_add(diff(xp, o), diff(xm, o)), cx);
    L = df_add(L, df_mul(df_add(diff(rkp + i0 + c, o), diff(rkm + i0 + c, o)), cz));
    if (has_lo) L = df_add(L, df_mul(diff(o - plane, o), ca));
    if (has_hi) L = df_add(L, df_mul(diff(o + plane, o), cc));
    df r;
    if (rin) {
      const float2 q = rin[o];
      r = df{q.x, q.y};
    } else {
      float fh, fl;
      f64_split(f[o], fh, fl);
      r = df_add(df{fh, fl}, df{-mh, -ml});
    }
    r = df_add(r, df_neg(L));
    if (rout) rout[o] = make_float2(r.hi, r.lo);
    out[c] = r.hi + r.lo;
  }
  r0 = out[0];
  r1 = out[1];
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
    if constexpr (sizeof(T) < sizeof(TI)) {
      // FP64 input to the FP32 solve: integer truncation keeps the FP64 pipe idle
      return mk<T>(f64_to_f32_trunc(a), f64_to_f32_trunc(b));
    } else {
      const TI s = TI(args.in_scale);
      return mk<T>(T(a * s), T(b * s));
    }
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
  } else {  // FWD_RESID: FP64 rhs (or a stored residual), FP32 pressure field, double-float arithmetic
    if constexpr (sizeof(T) == 4) {
      float r0, r1;
      residual_pair_df(g, args, tt, tb, j, k, i0, r0, r1);
      return mk<T>(r0, r1);
    } else {
      return mk<T>(T(0), T(0));   // not used: the FP64 path never refines
    }
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

// Epilogue of the inverse x-transform: store, accumulate, or (INV_FINAL) assemble the FP64
// pressure hi + (lo + v) of the refined solve (exact widenings, one FP64 addition).
template <typename T, typename TO, int MODE>
__device__ __forceinline__ void inv_store(TO* o, size_t off, T x0, T x1, const PairArgs& pair) {
  if constexpr (MODE == INV_ACCUM) {
    TO a, b;
    RealIO<TO>::load2(o, a, b);
    RealIO<TO>::store2(o, a + TO(x0), b + TO(x1));
  } else if constexpr (MODE == INV_FINAL) {
    if constexpr (sizeof(T) == 4 && sizeof(TO) == 8) {
      const float2 h = *reinterpret_cast<const float2*>(pair.hi + off);
      float2 l = make_float2(0.0f, 0.0f);
      if (pair.lo) l = *reinterpret_cast<const float2*>(pair.lo + off);
      RealIO<TO>::store2(o, f32_add_to_f64(h.x, l.x + x0), f32_add_to_f64(h.y, l.y + x1));
    }
  } else {
    RealIO<TO>::store2(o, TO(x0), TO(x1));
  }
}

// INV_FINAL epilogue on preloaded pairs: p = hi + (lo + v), v the last correction.
// hi + (lo + v) in FP64: both FP32 terms widened exactly by integer operations and added by one
// FP64 addition (correctly rounded), which costs fewer issue slots than assembling the sum by
// integer operations and runs on the FP64 pipe, idle in this pass.
__device__ __forceinline__ void final_store(double* o, float2 h, float2 l, float v0, float v1) {
  RealIO<double>::store2(o, f32_to_f64_exact(h.x) + f32_to_f64_exact(l.x + v0),
                         f32_to_f64_exact(h.y) + f32_to_f64_exact(l.y + v1));
}

// ---- per-line form of the refinement residual (specialised kernels) --------------------------
// Everything that depends only on the line (neighbour line offsets, double-float stencil
// coefficients, the split mean of f) is set up once per line.  The stencil sum is accumulated
// in the compensated "Dot2" form (Ogita, Rump and Oishi, 2005): each product coef * d is split
// exactly into p + pi by an FMA, the p are summed with TwoSum and all error terms go into one
// correction, giving the result as if computed with twice the FP32 precision.
struct ResidLine {
  const float* P;      // the FP32 pressure field (hi, or lo for a later correction) of this line
  const double* f;     // rhs of this line
  const float2* rin;   // stored residual of this line (replaces f - <f>; null when absent)
  float2* rout;        // the residual stored as an FP32 pair (null: not stored)
  int ozm, ozp;        // element offsets of the z-1 and z+1 lines (periodic)
  int oym, oyp;        // offsets of the y-1 and y+1 lines (0 at a wall: no such face)
  bool hym, hyp;       // the y-1 / y+1 face exists
  df cx, cz, ca, cc;
  float mh, ml;
  int nx;
};

// The offsets are 32-bit: the launchers send planes of 2^31 points or more to the generic kernels.
template <typename TT>
__device__ __forceinline__ ResidLine resid_line(const Geometry& g, const FwdArgs& args, const TT& tt,
                                                const DevTables& tb, int line, float mh, float ml) {
  const int j = line / g.nz, k = line - j * g.nz;
  const int plane = g.nz * g.nx;
  const size_t row = (size_t)line * g.nx;
  ResidLine R;
  R.P = reinterpret_cast<const float*>(args.p) + row;
  R.f = reinterpret_cast<const double*>(args.in) + row;
  R.rin = args.rin ? reinterpret_cast<const float2*>(args.rin) + row : nullptr;
  R.rout = args.rout ? reinterpret_cast<float2*>(args.rout) + row : nullptr;
  R.ozm = (k == 0 ? g.nz - 1 : -1) * g.nx;
  R.ozp = (k + 1 == g.nz ? 1 - g.nz : 1) * g.nx;
  R.hym = j >= 1;
  R.hyp = j + 1 <= g.ny - 1;
  R.oym = R.hym ? -plane : 0;
  R.oyp = R.hyp ? plane : 0;
  R.cx = df{args.idx2h, args.idx2l};
  R.cz = df{args.idz2h, args.idz2l};
  R.ca = df{tt.a[j], tt.a_lo[j]};
  R.cc = df{tt.c[j], tt.c_lo[j]};
  R.mh = mh;
  R.ml = ml;
  R.nx = g.nx;
  return R;
}

__device__ __forceinline__ float2 ld_f2(const float* p) { return *reinterpret_cast<const float2*>(p); }

// ---- the residual of a pair of cells in packed FP32x2 operations (df2.cuh), cell 0 in .x and
// cell 1 in .y
__device__ __forceinline__ df2 diff_sum2(df2 a, df2 b) {
  const df2 s = two_sum2(a.hi, b.hi);
  return df2{s.hi, f2add(s.lo, f2add(a.lo, b.lo))};
}
// (S, C) -= coef * (d.hi + d.lo), compensated (Dot2), coef a double-float broadcast to both lanes.
__device__ __forceinline__ void dot2_sub2(float2& S, float2& C, float2 ch, float2 cl, df2 d) {
  const float2 p = f2mul(ch, d.hi);
  float2 q = f2fma(ch, d.hi, make_float2(-p.x, -p.y));
  q = f2fma(cl, d.hi, q);
  q = f2fma(ch, d.lo, q);
  const df2 s = two_diff2(S, p);
  S = s.hi;
  C = f2add(C, f2sub(s.lo, q));
}

// The loads of one pair (the pressure's hi values around the two cells and the rhs), issued
// apart from the arithmetic so that a caller can keep the next pair's loads in flight.
struct ResidIn {
  float2 pc, zm, zp, ym, yp;
  float pm, pp;
  double2 fv;   // rhs (the first correction)
  float4 rv;    // stored residual pairs of the two cells (later corrections)
};
template <bool RIN>
__device__ __forceinline__ ResidIn resid_load(const ResidLine& R, int n) {
  const int i0 = 2 * n;
  const int im = i0 == 0 ? R.nx - 1 : i0 - 1;
  const int ip = i0 + 2 == R.nx ? 0 : i0 + 2;
  ResidIn in;
  in.pc = ld_f2(R.P + i0);
  in.pm = R.P[im];
  in.pp = R.P[ip];
  in.zm = ld_f2(R.P + (i0 + R.ozm));
  in.zp = ld_f2(R.P + (i0 + R.ozp));
  in.ym = R.hym ? ld_f2(R.P + (i0 + R.oym)) : make_float2(0.f, 0.f);
  in.yp = R.hyp ? ld_f2(R.P + (i0 + R.oyp)) : make_float2(0.f, 0.f);
  if constexpr (RIN) {
    in.rv = *reinterpret_cast<const float4*>(R.rin + i0);
  } else {
    in.fv = *reinterpret_cast<const double2*>(R.f + i0);
  }
  return in;
}

template <bool RIN>
__device__ __forceinline__ float2 resid_pair_from(const ResidLine& R, int n, const ResidIn& in) {
  const int i0 = 2 * n;
  const float2 pc = in.pc, zm = in.zm, zp = in.zp, ym = in.ym, yp = in.yp;
  const float pm = in.pm, pp = in.pp;
  // x-neighbours: cell 0 pairs (p_{i-1}, p_{i+1} = cell 1), cell 1 pairs (p_{i+2}, p_i = cell 0);
  // the difference between the two cells is shared with opposite signs
  df2 dout = two_diff2(make_float2(pm, pp), pc);
  const df2 d01 = two_diff2(make_float2(pc.y, pc.x), pc);   // (p1 - p0, p0 - p1), exact
  df2 dz0 = two_diff2(zp, pc), dz1 = two_diff2(zm, pc);
  df2 dy0 = two_diff2(ym, pc), dy1 = two_diff2(yp, pc);
  dout = diff_sum2(dout, d01);
  float2 S, C;
  if constexpr (RIN) {   // the stored residual (already without <f>)
    S = make_float2(in.rv.x, in.rv.z);
    C = make_float2(in.rv.y, in.rv.w);
  } else {
    float2 fh, fl;
    f64_split(in.fv.x, fh.x, fl.x);
    f64_split(in.fv.y, fh.y, fl.y);
    const df2 s0 = two_sum2(fh, make_float2(-R.mh, -R.mh));
    S = s0.hi;
    C = f2add(s0.lo, f2sub(fl, make_float2(R.ml, R.ml)));
  }
  dot2_sub2(S, C, make_float2(R.cx.hi, R.cx.hi), make_float2(R.cx.lo, R.cx.lo), dout);
  dot2_sub2(S, C, make_float2(R.cz.hi, R.cz.hi), make_float2(R.cz.lo, R.cz.lo), diff_sum2(dz0, dz1));
  if (R.hym) dot2_sub2(S, C, make_float2(R.ca.hi, R.ca.hi), make_float2(R.ca.lo, R.ca.lo), dy0);
  if (R.hyp) dot2_sub2(S, C, make_float2(R.cc.hi, R.cc.hi), make_float2(R.cc.lo, R.cc.lo), dy1);
  const float2 r = f2add(S, C);
  if (R.rout) {   // the residual as normalised pairs (quick TwoSum of S and C), one per cell
    const float2 e = f2sub(C, f2sub(r, S));
    *reinterpret_cast<float4*>(R.rout + i0) = make_float4(r.x, e.x, r.y, e.y);
  }
  return r;
}

template <bool RIN>
__device__ __forceinline__ float2 resid_pair_line2(const ResidLine& R, int n) {
  return resid_pair_from<RIN>(R, n, resid_load<RIN>(R, n));
}

}  // namespace pp
