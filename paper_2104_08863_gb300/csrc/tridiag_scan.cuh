// Wall-normal pieces shared by the standalone kernels (k_tridiag.cu) and the persistent batched
// kernel (batch_persistent.cu): the low-mode test, the reciprocal, 8- and 4-byte asynchronous
// copies, the warp-scan FP32 PDD tile (Sec. 2.2, Eqs. 10-21, exact reduced system) and the exact
// solve of the singular (0, 0) mode.
#pragma once

#include "internal.h"

namespace pp {

__device__ __forceinline__ bool is_low(int kx, int kz, int nz, int L) {
  return L >= 0 && kx <= L && (kz <= L || kz >= nz - L);
}

__device__ __forceinline__ float rcp_nr(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  const float e = fmaf(-x, r, 1.f);
  return fmaf(r, e, r);
}

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// ---- FP32 PDD with the reduced system solved by warp scans (P a power of two <= 32) ---------
// Same blocks and factors as k_tridiag_reg, but threads are numbered system-major (tid = s*P + b),
// so the P blocks of a system are P consecutive lanes of one warp and the reduced interface
// system needs no shared memory and no barrier.  With the per-mode LU (vL, inv, X01, X10, tw) of
// interface i, its two sweeps are first-order linear recurrences
//   y0_i = (inv_i vL_i) y0_{i-1} + (inv_i xL_i + X01_i xF_{i+1}),
//   z1_i = (tw_i inv_i) z1_{i+1} + y1_i,   y1_i = X10_i (xL_i + vL_i y0_{i-1}) + inv_i xF_{i+1},
// solved by log2(P)-step inclusive scans of affine maps over the segment's lanes; then
// z0_i = y0_i + tw_i X01_i z1_{i+1}, the neighbour values are alpha_b = z0_{b-1}, beta_b = z1_b.
// The tile is staged through shared memory in both directions (coalesced copies of S-system row
// segments), laid out [block][row][system] with an odd block stride so that a warp's lanes, which
// walk different blocks of the same rows, fall on distinct bank pairs.

// (A, B) <- (A, B) o (A', B') from the lane d below within segments of P lanes (inclusive scan)
__device__ __forceinline__ void scan_up(int P, int lseg, float& A, float2& B) {
  for (int d = 1; d < P; d <<= 1) {
    const float Ap = __shfl_up_sync(0xffffffffu, A, d);
    const float Bx = __shfl_up_sync(0xffffffffu, B.x, d), By = __shfl_up_sync(0xffffffffu, B.y, d);
    if (lseg >= d) {
      B = make_float2(fmaf(A, Bx, B.x), fmaf(A, By, B.y));
      A *= Ap;
    }
  }
}
__device__ __forceinline__ void scan_down(int P, int lseg, float& A, float2& B) {
  for (int d = 1; d < P; d <<= 1) {
    const float Ap = __shfl_down_sync(0xffffffffu, A, d);
    const float Bx = __shfl_down_sync(0xffffffffu, B.x, d), By = __shfl_down_sync(0xffffffffu, B.y, d);
    if (lseg + d < P) {
      B = make_float2(fmaf(A, Bx, B.x), fmaf(A, By, B.y));
      A *= Ap;
    }
  }
}
__device__ __forceinline__ float2 shfl_up2(float2 v, int d) {
  return make_float2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
}
__device__ __forceinline__ float2 shfl_down2(float2 v, int d) {
  return make_float2(__shfl_down_sync(0xffffffffu, v.x, d), __shfl_down_sync(0xffffffffu, v.y, d));
}

// The sweeps of one system's block and the reduced interface system, on a staged tile: thread
// (s, b) with `blk` its block's first row (row i at blk[i * S], updated in place), `ab`, `cb` the
// block's a and c (a_{bM+i} at ab[i]); `active` false for the (0, 0) mode, the FP64 low modes
// and columns outside the launch, which take part in the shuffles only; (vL, inv, X01, X10, tw)
// the record of interface b of the system's reduced LU (b < P-1).
template <int M>
__device__ __forceinline__ void scan_sweeps(int P, int S, float2* blk, const float* ab, const float* cb, int b,
                                            bool active, float sigma, float vL, float inv, float X01, float X10,
                                            float tw) {
  const int lseg = b;
  // The backward sweep x_i = rb_i (gg_i + alpha gv_i + c_i x_{i+1}) takes its three products with
  // the pivot reciprocal rb_i from the forward sweep: rb_i gg_i in the tile (in place of gg_i),
  // rb_i c_i and rb_i gv_i in registers, so that it loads no coefficient from shared memory (whose
  // bandwidth bounds both sweeps).
  float rcv[M], rgv[M];
  float2 xF = make_float2(0.f, 0.f), xL = make_float2(0.f, 0.f);
  if (active) {
    float e = ab[0] + sigma, gv = ab[0], rb = rcp_nr(cb[0] + e);
    float run = 1.f;
    float2 gg = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < M; ++i) {
      const float cj = cb[i];
      const float2 F = blk[i * S];
      float mult = 0.f;
      if (i > 0) {
        mult = ab[i] * rb;
        e = fmaf(mult, e, sigma);
        gv = mult * gv;
        rb = rcp_nr(cj + e);
      }
      gg = make_float2(fmaf(mult, gg.x, -F.x), fmaf(mult, gg.y, -F.y));
      blk[i * S] = make_float2(gg.x * rb, gg.y * rb);
      const float crb = cj * rb;
      rcv[i] = crb;
      rgv[i] = gv * rb;
      const float kap = run * rb;
      xF.x = fmaf(kap, gg.x, xF.x);
      xF.y = fmaf(kap, gg.y, xF.y);
      run *= crb;
    }
    xL = make_float2(gg.x * rb, gg.y * rb);
  }
  float2 alpha = make_float2(0.f, 0.f), beta = make_float2(0.f, 0.f);
  if (P > 1) {
    // interface i = b (lanes b <= P-2); every lane takes part in the shuffles
    const float2 xFn = shfl_down2(xF, 1);                 // xF_{i+1}
    float A = inv * vL;
    float2 B = make_float2(fmaf(inv, xL.x, X01 * xFn.x), fmaf(inv, xL.y, X01 * xFn.y));
    scan_up(P, lseg, A, B);                               // B = y0_i
    const float2 y0 = B;
    float2 y0m = shfl_up2(y0, 1);                         // y0_{i-1}
    if (lseg == 0) y0m = make_float2(0.f, 0.f);
    const float2 q0 = make_float2(fmaf(vL, y0m.x, xL.x), fmaf(vL, y0m.y, xL.y));
    float G = tw * inv;
    float2 Y = make_float2(fmaf(X10, q0.x, inv * xFn.x), fmaf(X10, q0.y, inv * xFn.y));
    if (lseg == P - 1) { G = 0.f; Y = make_float2(0.f, 0.f); }
    scan_down(P, lseg, G, Y);                             // Y = z1_i
    const float2 z1 = Y;
    const float2 z1n = shfl_down2(z1, 1);                 // z1_{i+1}
    const float a0 = tw * X01;
    const float2 z0 = make_float2(fmaf(a0, z1n.x, y0.x), fmaf(a0, z1n.y, y0.y));
    const float2 z0m = shfl_up2(z0, 1);                   // z0_{b-1}
    if (lseg > 0) alpha = z0m;
    if (lseg < P - 1) beta = z1;
  }
  if (active) {
    float2 xn = beta;
#pragma unroll
    for (int i = M - 1; i >= 0; --i) {
      const float2 G2 = blk[i * S];   // rb_i gg_i
      xn = make_float2(fmaf(rcv[i], xn.x, fmaf(rgv[i], alpha.x, G2.x)),
                       fmaf(rcv[i], xn.y, fmaf(rgv[i], alpha.y, G2.y)));
      blk[i * S] = xn;
    }
  }
}

// One tile of S systems (tile = kz * ntile + kx tile, ntile tiles over [kx_lo, kx_hi)); P * S
// threads (256 with S = 256/P); `smem` holds the staged rows and the coefficient copies.
template <int M>
__device__ __forceinline__ void tridiag_scan_tile(const Geometry& g, int P, int S, int low, const float* __restrict__ a,
                                                  const float* __restrict__ c, const double* __restrict__ lamx,
                                                  const double* __restrict__ lamz, const float* __restrict__ rtab,
                                                  cplx<float>* __restrict__ spec, int kx_lo, int kx_hi, int tile_id,
                                                  unsigned char* smem) {
  float2* tile = reinterpret_cast<float2*>(smem);   // [b][i][s] with block stride BS, then a and c
  const int NT = P * S;
  const int BS = M * S + 1;
  constexpr int MS = M | 1;                        // odd per-block stride of the coefficient copies
  float* as = reinterpret_cast<float*>(tile + (size_t)P * BS);
  float* csm = as + P * MS;
  for (int j = threadIdx.x; j < g.ny; j += NT) {
    const int bj = j / M, ij = j - bj * M;
    as[bj * MS + ij] = a[j];
    csm[bj * MS + ij] = c[j];
  }
  // a CTA owns the S systems kx0 .. kx0+S-1 of one kz, within the launch's columns
  // [kx_lo, kx_hi) (kx_lo a multiple of S); columns past the padded row (pitch) are not touched,
  // columns in [ncols, pitch) are padding and go back unchanged (the last slab copies them)
  const int ntile = (kx_hi - kx_lo + S - 1) / S;
  const int kz = tile_id / ntile;
  const int kx0 = kx_lo + (tile_id - kz * ntile) * S;
  const int copy_hi = kx_hi >= g.ncols ? g.pitch : kx_hi;
  const size_t rstride = (size_t)g.nz * g.pitch;
  // ---- coalesced copy-in: thread t copies block t / S of system t % S (S-system row segments)
  const int cpb = threadIdx.x / S, cps = threadIdx.x - cpb * S;
  const bool cvalid = kx0 + cps < copy_hi;
  const float2* gsrc = reinterpret_cast<const float2*>(spec) + (size_t)kz * g.pitch + kx0 + cps +
                       (size_t)cpb * M * rstride;
  float2* tsrc = tile + cpb * BS + cps;
  if (cvalid) {
#pragma unroll
    for (int i = 0; i < M; ++i) cp_async8(tsrc + i * S, gsrc + (size_t)i * rstride);
  }
  // ---- compute role: thread (s, b); its interface record is fetched while the tile lands
  const int s = threadIdx.x / P, b = threadIdx.x - s * P;
  const int kx = kx0 + s;
  const int sys = kz * g.ncols + kx;
  const bool active = kx < kx_hi && kx < g.ncols && !(kx == 0 && kz == 0) && !is_low(kx, kz, g.nz, low);
  float vL = 0.f, inv = 0.f, X01 = 0.f, X10 = 0.f, tw = 0.f;
  if (P > 1 && active && b < P - 1) {
    const float* t = rtab + ((size_t)sys * (P - 1) + b) * 5;
    vL = __ldg(t); inv = __ldg(t + 1); X01 = __ldg(t + 2); X10 = __ldg(t + 3); tw = __ldg(t + 4);
  }
  cp_async_wait_all();
  __syncthreads();
  scan_sweeps<M>(P, S, tile + b * BS + s, as + b * MS, csm + b * MS, b, active,
                 active ? float(-(lamx[kx] + lamz[kz])) : 0.f, vL, inv, X01, X10, tw);
  __syncthreads();
  // ---- coalesced copy-out
  if (cvalid) {
    float2* gdst = reinterpret_cast<float2*>(spec) + (size_t)kz * g.pitch + kx0 + cps + (size_t)cpb * M * rstride;
#pragma unroll
    for (int i = 0; i < M; ++i) gdst[(size_t)i * rstride] = tsrc[i * S];
  }
}

template <int M>
__global__ void __launch_bounds__(256, 2) k_tridiag_scan(Geometry g, int P, int S, int low, const float* __restrict__ a,
                                                         const float* __restrict__ c, const double* __restrict__ lamx,
                                                         const double* __restrict__ lamz, const float* __restrict__ rtab,
                                                         cplx<float>* __restrict__ spec, int kx_lo, int kx_hi) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  tridiag_scan_tile<M>(g, P, S, low, a, c, lamx, lamz, rtab, spec, kx_lo, kx_hi, blockIdx.x, smem_raw);
}

// The (0, 0) mode: T p = F - mean with sum_j dy_j p_j = 0 (compatibility and gauge), by the
// exact flux prefix sums  q_j = sum_{l<=j} dy_l F^c_l,  p_0 = 0,  p_{j+1} = p_j + h_{j+1} q_j,
// followed by removal of the dy-weighted mean.  One warp, FP64, chunked warp scans.
__device__ __forceinline__ double warp_excl_scan(double v, double& total) {
  const int lane = threadIdx.x & 31;
  double x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  total = __shfl_sync(0xffffffffu, x, 31);
  return x - v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Executed by one warp (lane = threadIdx.x & 31); `work` holds 2 ny doubles.
template <typename TD>
__device__ __forceinline__ void mode00_warp(const Geometry& g, const double* __restrict__ dy,
                                            const double* __restrict__ h, cplx<TD>* __restrict__ spec,
                                            double* __restrict__ acc, int gauge, double* work) {
  double* fr = work;
  double* fi = fr + g.ny;
  const int lane = threadIdx.x & 31;
  const int ny = g.ny;
  const int ch = (ny + 31) / 32;
  const int lo = lane * ch, hi = min(ny, lo + ch);
  const size_t rstride = (size_t)g.nz * g.pitch;
  double sr = 0, si = 0, sw = 0;
  for (int j = lo; j < hi; ++j) {
    const cplx<TD> F = ld_c_cg(spec + (size_t)j * rstride);
    fr[j] = double(F.x);
    fi[j] = double(F.y);
    sr += dy[j] * fr[j];
    si += dy[j] * fi[j];
    sw += dy[j];
  }
  sr = warp_sum(sr); si = warp_sum(si); sw = warp_sum(sw);
  const double mr = sr / sw, mi = si / sw;
  // <f> = (sum_j dy_j F_j) / (sum_j dy_j Nx Nz): kept for the residual of the refined solve
  if (gauge == GAUGE_STORE_MEAN && lane == 0) acc[0] = mr / ((double)g.nx * (double)g.nz);
  // flux prefix sums, in place: q_j (inclusive)
  double lr = 0, li = 0;
  for (int j = lo; j < hi; ++j) {
    lr += dy[j] * (fr[j] - mr);
    li += dy[j] * (fi[j] - mi);
    fr[j] = lr;
    fi[j] = li;
  }
  double tr, ti;
  const double orr = warp_excl_scan(lr, tr), oi = warp_excl_scan(li, ti);
  for (int j = lo; j < hi; ++j) { fr[j] += orr; fi[j] += oi; }
  __syncwarp();
  // p_j = sum_{l<j} h_{l+1} q_l  (exclusive prefix of t_l = h_{l+1} q_l, l <= ny-2)
  double pr = 0, pi = 0;
  double lastr = 0, lasti = 0;
  for (int j = lo; j < hi; ++j) {
    const double tq_r = j + 1 <= ny - 1 ? h[j + 1] * fr[j] : 0.0;
    const double tq_i = j + 1 <= ny - 1 ? h[j + 1] * fi[j] : 0.0;
    fr[j] = pr;   // exclusive
    fi[j] = pi;
    pr += tq_r;
    pi += tq_i;
    lastr = pr; lasti = pi;
  }
  (void)lastr; (void)lasti;
  const double o2r = warp_excl_scan(pr, tr), o2i = warp_excl_scan(pi, ti);
  double mr2 = 0, mi2 = 0;
  for (int j = lo; j < hi; ++j) {
    fr[j] += o2r;
    fi[j] += o2i;
    mr2 += dy[j] * fr[j];
    mi2 += dy[j] * fi[j];
  }
  mr2 = warp_sum(mr2) / sw;
  mi2 = warp_sum(mi2) / sw;
  // Offset gauge: the running total p has weighted sum acc[1]; shift this (0,0) profile by
  // -acc[1] / sum(dy) so that sum_j dy_j (P_j + shift) = -acc[1].
  if (gauge == GAUGE_OFFSET) mr2 += acc[1] / sw;
  for (int j = lo; j < hi; ++j)
    st_c(spec + (size_t)j * rstride, mk<TD>(TD(fr[j] - mr2), TD(fi[j] - mi2)));
}

template <typename TD>
__global__ void __launch_bounds__(32) k_mode00(Geometry g, const double* __restrict__ dy,
                                               const double* __restrict__ h, cplx<TD>* __restrict__ spec,
                                               double* __restrict__ acc, int gauge) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  mode00_warp<TD>(g, dy, h, spec, acc, gauge, reinterpret_cast<double*>(smem_raw));
}

}  // namespace pp
