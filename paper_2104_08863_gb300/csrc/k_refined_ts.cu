// The FP64-accurate timestep on FP32 units (the refined form of the projection timestep).
//
// The state (u, v, w) is carried through the step as FP32 pairs (hi, lo) with hi + lo equal to
// the FP64 value to about 2^-47 (same bytes as FP64), and every per-point operation runs in
// double-float arithmetic on the FP32 pipes (GB300 issues ~2 FP64 instructions per clock per SM
// against 128 FP32):
//   k_to_pairs        FP64 field -> pairs, in place (integer split, no FP64 instruction), and
//   k_from_pairs      back (faithful integer assembly);
//   k_momentum_df     one Heun stage (Eqs. 5-6) of the momentum right-hand side, the same
//                     central differences and edge-flux sharing as k_momentum, in double-float;
//   k_divergence_df   f = D(u*)/dt (Eq. 7) from the pairs, assembled as FP64 for the refined
//                     Poisson solve;
//   k_gradient_pairs  u = u* - dt G p (Eq. 4) from the pairs and the solve's FP32 pressure pair,
//                     FP64 out.
#include "df2.cuh"
#include "fpconv.cuh"
#include "internal.h"

namespace pp {

namespace {

__device__ __forceinline__ df dadd(df a, df b) { return df_add(a, b); }
__device__ __forceinline__ df dsub(df a, df b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df dmul(df a, df b) { return df_mul(a, b); }
__device__ __forceinline__ df dfma(df a, df b, df c) { return df_add(df_mul(a, b), c); }
__device__ __forceinline__ df dtwice(df a) { return df{2.f * a.hi, 2.f * a.lo}; }
// Sum of two pairs left unnormalised (TwoSum of the high parts, the low parts added): a valid
// double-float operand for a product, three operations cheaper than dadd.
__device__ __forceinline__ df uadd(df a, df b) {
  const df s = two_sum_df(a.hi, b.hi);
  return df{s.hi, s.lo + (a.lo + b.lo)};
}
__device__ __forceinline__ df usub(df a, df b) {
  const df s = two_diff_df(a.hi, b.hi);
  return df{s.hi, s.lo + (a.lo - b.lo)};
}
// Compensated accumulator (S, C) += c * x: the product's rounding error by FMAs, the sum's by
// TwoSum, all error terms collected in C (the Dot2 scheme); normalised once at the end.
struct Acc { float S, C; };
__device__ __forceinline__ void acc_prod(Acc& a, df c, df x) {
  const float p = c.hi * x.hi;
  float e = fmaf(c.hi, x.hi, -p);
  e = fmaf(c.hi, x.lo, e);
  e = fmaf(c.lo, x.hi, e);
  const df t = two_sum_df(a.S, p);
  a.S = t.hi;
  a.C += t.lo + e;
}
__device__ __forceinline__ Acc acc_of(df x) { return Acc{x.hi, x.lo}; }
__device__ __forceinline__ float2 acc_out(const Acc& a) {
  const df r = quick_two_sum_df(a.S, a.C);
  return make_float2(r.hi, r.lo);
}
__device__ __forceinline__ df ldp(const float2* p) {
  const float2 v = __ldg(p);
  return df{v.x, v.y};
}
__device__ __forceinline__ df split(double x) {
  df r;
  f64_split(x, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ float2 f2(df a) { return make_float2(a.hi, a.lo); }

// The same operations on two values at once (df2.cuh): lane x one value, lane y the other, each
// lane giving the scalar form's result.
__device__ __forceinline__ df2 pk(df a, df b) { return df2{make_float2(a.hi, b.hi), make_float2(a.lo, b.lo)}; }
__device__ __forceinline__ df2 bc(df a) { return pk(a, a); }
__device__ __forceinline__ df2 uadd2(df2 a, df2 b) {
  const df2 s = two_sum2(a.hi, b.hi);
  return df2{s.hi, f2add(s.lo, f2add(a.lo, b.lo))};
}
__device__ __forceinline__ df2 usub2(df2 a, df2 b) {
  const df2 s = two_diff2(a.hi, b.hi);
  return df2{s.hi, f2add(s.lo, f2sub(a.lo, b.lo))};
}
__device__ __forceinline__ df2 dmul2(df2 a, df2 b) {
  const float2 p = f2mul(a.hi, b.hi);
  float2 e = f2fma(a.hi, b.hi, make_float2(-p.x, -p.y));
  e = f2fma(a.hi, b.lo, e);
  e = f2fma(a.lo, b.hi, e);
  return df2{p, e};
}
__device__ __forceinline__ df2 dtwice2(df2 a) {
  return df2{f2mul(a.hi, make_float2(2.f, 2.f)), f2mul(a.lo, make_float2(2.f, 2.f))};
}
struct Acc2 { float2 S, C; };
__device__ __forceinline__ void acc_prod2(Acc2& a, df2 c, df2 x) {
  const float2 p = f2mul(c.hi, x.hi);
  float2 e = f2fma(c.hi, x.hi, make_float2(-p.x, -p.y));
  e = f2fma(c.hi, x.lo, e);
  e = f2fma(c.lo, x.hi, e);
  const df2 t = two_sum2(a.S, p);
  a.S = t.hi;
  a.C = f2add(a.C, f2add(t.lo, e));
}
// (S + C) normalised (quick TwoSum) lane by lane; lane x as the first pair, lane y the second.
__device__ __forceinline__ void acc_out2(const Acc2& a, float2& x, float2& y) {
  const float2 s = f2add(a.S, a.C);
  const float2 lo = f2sub(a.C, f2sub(s, a.S));
  x = make_float2(s.x, lo.x);
  y = make_float2(s.y, lo.y);
}

constexpr int MTX = 32, MTZ = 8;

struct RowCoefDF {
  df c0, ca, cc, cay;
  df v0, va, vc, vay;
};

__global__ void __launch_bounds__(256) k_to_pairs(double* __restrict__ x, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const df s = split(x[i]);
    reinterpret_cast<float2*>(x)[i] = f2(s);
  }
}

__global__ void __launch_bounds__(256) k_from_pairs(double* __restrict__ x, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float2 v = reinterpret_cast<const float2*>(x)[i];
    x[i] = f32_add_to_f64(v.x, v.y);
  }
}

// out = alpha * base + beta * s + bdt * R(s) on pairs (see k_momentum for the stencil).
__global__ void __launch_bounds__(MTX * MTZ) k_momentum_df(Geometry g, MomArgsDF a, const double* __restrict__ inv_dy,
                                                          const double* __restrict__ inv_h,
                                                          const double* __restrict__ lo,
                                                          const double* __restrict__ up, int jc) {
  extern __shared__ unsigned char smem_raw[];
  RowCoefDF* rc = reinterpret_cast<RowCoefDF*>(smem_raw);
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int j0 = blockIdx.z * jc;
  const int j1 = min(ny, j0 + jc);
  const double bdtnu = a.bdt * a.nu;
  const double cdx = bdtnu / (g.dx * g.dx), cdz = bdtnu / (g.dz * g.dz);
  for (int r = threadIdx.y * MTX + threadIdx.x; r < j1 - j0; r += MTX * MTZ) {
    const int j = j0 + r;
    RowCoefDF c;
    const double A = j > 0 ? lo[j] : 2.0 * inv_dy[0] * inv_dy[0];
    const double C = j < ny - 1 ? up[j] : 2.0 * inv_dy[ny - 1] * inv_dy[ny - 1];
    c.c0 = split(a.beta - 2.0 * cdx - 2.0 * cdz - bdtnu * (A + C));
    c.ca = split(j > 0 ? bdtnu * lo[j] : 0.0);
    c.cc = split(j < ny - 1 ? bdtnu * up[j] : 0.0);
    c.cay = split(-0.25 * a.bdt * inv_dy[j]);
    if (j >= 1) {
      const double va = bdtnu * inv_h[j] * inv_dy[j - 1], vc = bdtnu * inv_h[j] * inv_dy[j];
      c.v0 = split(a.beta - 2.0 * cdx - 2.0 * cdz - va - vc);
      c.va = split(va);
      c.vc = split(vc);
      c.vay = split(-0.25 * a.bdt * inv_h[j]);
    } else {
      c.v0 = c.va = c.vc = c.vay = df{0.f, 0.f};
    }
    rc[r] = c;
  }
  __syncthreads();
  const int i = blockIdx.x * MTX + threadIdx.x;
  const int k = blockIdx.y * MTZ + threadIdx.y;
  if (i >= nx || k >= nz) return;
  const df cDx = split(cdx), cDz = split(cdz);
  const df cAx = split(-0.25 * a.bdt / g.dx), cAz = split(-0.25 * a.bdt / g.dz);
  const df2 cD_xz = pk(cDx, cDz), cD_zx = pk(cDz, cDx), cA_xz = pk(cAx, cAz), cA_zx = pk(cAz, cAx);
  const df fterm = split(a.bdt * a.fx);
  const df alpha = split(a.alpha);
  const bool has_base = a.bu != nullptr;
  const size_t plane = (size_t)nz * nx;
  const int im = i == 0 ? nx - 1 : i - 1, ip = i == nx - 1 ? 0 : i + 1;
  const int km = k == 0 ? nz - 1 : k - 1, kp = k == nz - 1 ? 0 : k + 1;
  const size_t oc = (size_t)k * nx + i, oxm = (size_t)k * nx + im, oxp = (size_t)k * nx + ip;
  const size_t ozm = (size_t)km * nx + i, ozp = (size_t)kp * nx + i;
  const size_t ozm_xp = (size_t)km * nx + ip, ozp_xm = (size_t)kp * nx + im;
  const float2* su = a.su;
  const float2* sv = a.sv;
  const float2* sw = a.sw;
  const df zero{0.f, 0.f};

  df u_m = zero, w_m = zero;
  df u_c = ldp(su + (size_t)j0 * plane + oc), w_c = ldp(sw + (size_t)j0 * plane + oc);
  df v_m = j0 > 0 ? ldp(sv + (size_t)(j0 - 1) * plane + oc) : zero;
  df v_c = ldp(sv + (size_t)j0 * plane + oc);
  df u_m_xp = zero, w_m_zp = zero;
  df e_uv = zero, e_vw = zero;
  if (j0 > 0) {
    const size_t pm = (size_t)(j0 - 1) * plane, pc = (size_t)j0 * plane;
    u_m = ldp(su + pm + oc);
    w_m = ldp(sw + pm + oc);
    u_m_xp = ldp(su + pm + oxp);
    w_m_zp = ldp(sw + pm + ozp);
    e_uv = dmul(uadd(ldp(sv + pc + oxm), v_c), uadd(u_m, u_c));
    e_vw = dmul(uadd(ldp(sv + pc + ozm), v_c), uadd(w_m, w_c));
  }
  df vs_m = uadd(v_m, v_c);
  if (j0 == 0) a.ov[oc] = has_base ? a.bv[oc] : f2(v_c);
  for (int j = j0; j < j1; ++j) {
    const RowCoefDF c = rc[j - j0];
    const size_t pc = (size_t)j * plane, pn = pc + plane;
    const bool top = j + 1 < ny;
    const df u_n = top ? ldp(su + pn + oc) : zero;
    const df w_n = top ? ldp(sw + pn + oc) : zero;
    const df v_n = ldp(sv + pn + oc);
    const df u_xm = ldp(su + pc + oxm), u_xp = ldp(su + pc + oxp), u_zm = ldp(su + pc + ozm), u_zp = ldp(su + pc + ozp);
    const df u_zm_xp = ldp(su + pc + ozm_xp);
    const df w_xm = ldp(sw + pc + oxm), w_xp = ldp(sw + pc + oxp), w_zm = ldp(sw + pc + ozm), w_zp = ldp(sw + pc + ozp);
    const df w_zp_xm = ldp(sw + pc + ozp_xm);
    const df v_xm = ldp(sv + pc + oxm), v_xp = ldp(sv + pc + oxp), v_zm = ldp(sv + pc + ozm), v_zp = ldp(sv + pc + ozp);
    df e_uv_n = zero, e_vw_n = zero;   // fluxes through face j+1 (zero on the top wall), as a pair
    if (top) {
      const df2 e = dmul2(uadd2(pk(ldp(sv + pn + oxm), ldp(sv + pn + ozm)), bc(v_n)), uadd2(pk(u_c, w_c), pk(u_n, w_n)));
      e_uv_n = df{e.hi.x, e.lo.x};
      e_vw_n = df{e.hi.y, e.lo.y};
    }
    const df e_uw = dmul(uadd(w_xm, w_c), uadd(u_zm, u_c));
    float2 bu2 = make_float2(0.f, 0.f), bw2 = bu2, bv2 = bu2;
    if (has_base) {   // the stage-2 base values, loaded together with the stencil
      bu2 = a.bu[pc + oc];
      bw2 = a.bw[pc + oc];
      if (j >= 1) bv2 = a.bv[pc + oc];
    }
    {   // u (lane x) and w (lane y): their equations mirror each other under x <-> z, term by term
      Acc2 acc{make_float2(fterm.hi, 0.f), make_float2(fterm.lo, 0.f)};
      if (has_base) acc_prod2(acc, bc(alpha), pk(df{bu2.x, bu2.y}, df{bw2.x, bw2.y}));
      const df2 cuw = pk(u_c, w_c);
      acc_prod2(acc, bc(c.c0), cuw);
      const df2 xp = pk(u_xp, w_zp), xm = pk(u_xm, w_zm);   // along x for u, along z for w
      const df2 s1 = uadd2(xp, xm);
      acc_prod2(acc, cD_xz, s1);
      acc_prod2(acc, cA_xz, dmul2(usub2(xp, xm), uadd2(s1, dtwice2(cuw))));
      acc_prod2(acc, cD_zx, uadd2(pk(u_zp, w_xp), pk(u_zm, w_xm)));
      acc_prod2(acc, cA_zx, usub2(dmul2(uadd2(pk(w_zp_xm, w_c), pk(w_zp, w_xp)), uadd2(pk(u_c, u_zm_xp), pk(u_zp, u_xp))),
                                  bc(e_uw)));
      acc_prod2(acc, bc(c.cay), usub2(pk(e_uv_n, e_vw_n), pk(e_uv, e_vw)));
      acc_prod2(acc, bc(c.ca), pk(u_m, w_m));
      acc_prod2(acc, bc(c.cc), pk(u_n, w_n));
      float2 ou, ow;
      acc_out2(acc, ou, ow);
      a.ou[pc + oc] = ou;
      a.ow[pc + oc] = ow;
    }
    if (j >= 1) {   // v at face j
      Acc acc{0.f, 0.f};
      if (has_base) acc_prod(acc, alpha, df{bv2.x, bv2.y});
      acc_prod(acc, c.v0, v_c);
      const df vs = uadd(v_c, v_n);
      acc_prod(acc, c.vay, dmul(usub(vs, vs_m), uadd(vs, vs_m)));
      acc_prod(acc, cDx, uadd(v_xp, v_xm));
      acc_prod(acc, cAx, usub(dmul(uadd(v_c, v_xp), uadd(u_m_xp, u_xp)), e_uv));
      acc_prod(acc, cDz, uadd(v_zp, v_zm));
      acc_prod(acc, cAz, usub(dmul(uadd(v_c, v_zp), uadd(w_m_zp, w_zp)), e_vw));
      acc_prod(acc, c.va, v_m);
      acc_prod(acc, c.vc, v_n);
      a.ov[pc + oc] = acc_out(acc);
    }
    vs_m = uadd(v_c, v_n);
    u_m = u_c; u_c = u_n;
    w_m = w_c; w_c = w_n;
    v_m = v_c; v_c = v_n;
    u_m_xp = u_xp;
    w_m_zp = w_zp;
    e_uv = e_uv_n;
    e_vw = e_vw_n;
  }
  if (j1 == ny) {
    const size_t pw = (size_t)ny * plane + oc;
    a.ov[pw] = has_base ? a.bv[pw] : __ldg(sv + pw);
  }
}

// f = D(u*) / dt at every cell from the pairs, written as FP64 (faithful assembly).
__global__ void __launch_bounds__(256) k_divergence_df(Geometry g, const float2* __restrict__ u,
                                                      const float2* __restrict__ v, const float2* __restrict__ w,
                                                      const double* __restrict__ inv_dy, double inv_dt,
                                                      double* __restrict__ f) {
  const size_t plane = (size_t)g.nz * g.nx;
  const int nlines = g.ny * g.nz;
  const df cx = split(inv_dt / g.dx), cz = split(inv_dt / g.dz), cdt = split(inv_dt);
  for (int line = blockIdx.x; line < nlines; line += gridDim.x) {
    const int j = line / g.nz, k = line - j * g.nz;
    const df cy = dmul(cdt, split(inv_dy[j]));
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
      const size_t idx = (size_t)line * g.nx + i;
      const size_t oxp = idx - i + (i + 1 == g.nx ? 0 : i + 1);
      const size_t ozp = (size_t)j * plane + (size_t)(k + 1 == g.nz ? 0 : k + 1) * g.nx + i;
      df s = dmul(cx, dsub(ldp(u + oxp), ldp(u + idx)));
      s = dfma(cz, dsub(ldp(w + ozp), ldp(w + idx)), s);
      s = dfma(cy, dsub(ldp(v + idx + plane), ldp(v + idx)), s);
      f[idx] = f32_add_to_f64(s.hi, s.lo);
    }
  }
}

// u = u* - dt G p (Eq. 4): u* as pairs, p = hi + lo the refined solve's FP32 pair, the result in
// FP64 (v's walls copied); the pressure differences and the products run in double-float and the
// sums are assembled into FP64 with integer operations (no FP64 instruction per point).  p_out,
// when given, receives p in FP64.
__global__ void __launch_bounds__(256) k_gradient_pairs(Geometry g, const float* __restrict__ hi,
                                                        const float* __restrict__ lo, double* __restrict__ u,
                                                        double* __restrict__ v, double* __restrict__ w,
                                                        double* __restrict__ p_out, const double* __restrict__ inv_h,
                                                        double dt) {
  const size_t plane = (size_t)g.nz * g.nx;
  const int nlines = (g.ny + 1) * g.nz;
  const df cx = split(dt / g.dx), cz = split(dt / g.dz), cdt = split(dt);
  const float2* up = reinterpret_cast<const float2*>(u);
  const float2* vp = reinterpret_cast<const float2*>(v);
  const float2* wp = reinterpret_cast<const float2*>(w);
  auto P = [&](size_t o) { return df{__ldg(hi + o), __ldg(lo + o)}; };
  for (int line = blockIdx.x; line < nlines; line += gridDim.x) {
    const int j = line / g.nz, k = line - j * g.nz;
    const df cy = (j >= 1 && j < g.ny) ? dmul(cdt, split(inv_h[j])) : df{0.f, 0.f};
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
      const size_t idx = (size_t)line * g.nx + i;
      const float2 vv = vp[idx];
      df vn{vv.x, vv.y};
      if (j < g.ny) {
        const float2 uu = up[idx], ww = wp[idx];
        const df pc = P(idx);
        const df pxm = P(idx - i + (i == 0 ? g.nx - 1 : i - 1));
        const df pzm = P((size_t)j * plane + (size_t)(k == 0 ? g.nz - 1 : k - 1) * g.nx + i);
        const df un = dsub(df{uu.x, uu.y}, dmul(cx, dsub(pc, pxm)));
        const df wn = dsub(df{ww.x, ww.y}, dmul(cz, dsub(pc, pzm)));
        u[idx] = f32_add_to_f64(un.hi, un.lo);
        w[idx] = f32_add_to_f64(wn.hi, wn.lo);
        if (p_out) p_out[idx] = f32_add_to_f64(pc.hi, pc.lo);
        if (j >= 1) {
          vn = dsub(vn, dmul(cy, dsub(pc, P(idx - plane))));
          v[idx] = f32_add_to_f64(vn.hi, vn.lo);
        } else {
          v[idx] = f32_add_to_f64(vn.hi, vn.lo);
        }
      } else {
        v[idx] = f32_add_to_f64(vn.hi, vn.lo);
      }
    }
  }
}

int line_grid(int nlines) { return nlines < 152 * 16 ? nlines : 152 * 16; }
int line_block(int nx) { return nx >= 256 ? 256 : (nx + 31) / 32 * 32; }

int grid_for(size_t total) {
  size_t blocks = (total + 255) / 256;
  const size_t cap = 152 * 16;
  return (int)(blocks < cap ? (blocks ? blocks : 1) : cap);
}

}  // namespace

cudaError_t launch_to_pairs(double* x, size_t n, cudaStream_t st) {
  k_to_pairs<<<grid_for(n), 256, 0, st>>>(x, n);
  return cudaGetLastError();
}

cudaError_t launch_from_pairs(double* x, size_t n, cudaStream_t st) {
  k_from_pairs<<<grid_for(n), 256, 0, st>>>(x, n);
  return cudaGetLastError();
}

cudaError_t launch_momentum_df(const Geometry& g, const DevTables& tb, const MomArgsDF& a, cudaStream_t st) {
  const int tx = (g.nx + MTX - 1) / MTX, tz = (g.nz + MTZ - 1) / MTZ;
  const long long tiles = (long long)tx * tz;
  int chunks = (int)((3LL * 2 * 152 + tiles - 1) / tiles);
  if (chunks > g.ny / 16) chunks = g.ny / 16;
  if (chunks < 1) chunks = 1;
  const int jc = (g.ny + chunks - 1) / chunks;
  chunks = (g.ny + jc - 1) / jc;
  const size_t smem = sizeof(RowCoefDF) * (size_t)jc;
  const cudaError_t e = ensure_smem_limit((const void*)k_momentum_df, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(tx, tz, chunks), block(MTX, MTZ);
  k_momentum_df<<<grid, block, smem, st>>>(g, a, tb.d.inv_dy, tb.d.inv_h, tb.d.a, tb.d.c, jc);
  return cudaGetLastError();
}

cudaError_t launch_divergence_df(const Geometry& g, const DevTables& tb, const float2* u, const float2* v,
                                 const float2* w, double dt, double* f, cudaStream_t st) {
  k_divergence_df<<<line_grid(g.ny * g.nz), line_block(g.nx), 0, st>>>(g, u, v, w, tb.d.inv_dy, 1.0 / dt, f);
  return cudaGetLastError();
}

cudaError_t launch_gradient_pairs(const Geometry& g, const DevTables& tb, const float* hi, const float* lo, double* u,
                                  double* v, double* w, double* p_out, double dt, cudaStream_t st) {
  k_gradient_pairs<<<line_grid((g.ny + 1) * g.nz), line_block(g.nx), 0, st>>>(g, hi, lo, u, v, w, p_out,
                                                                                tb.d.inv_h, dt);
  return cudaGetLastError();
}

}  // namespace pp
