// Wall-normal tridiagonal solves of Eq. 9: one system per (kx, kz) mode.
//
// Row j of mode (kx, kz), written as an M-matrix (all off-diagonals non-positive):
//     -a_j x_{j-1} + (a_j + c_j + sigma) x_j - c_j x_{j+1} = -F_j,
//     sigma = -(lambda_x(kx) + lambda_z(kz)) >= 0,
// with a_0 = c_{ny-1} = 0 (zero wall flux).
//
// PDD (Sec. 2.2, Eqs. 10-21): each system is cut into P blocks of m = ny/P rows; one thread
// owns one block, S systems share a CTA and a warp holds 32 consecutive systems of one block
// index, so every row access is a coalesced 32-system segment.  Per block:
//   1. forward elimination of the block matrix A_i (Eq. 20) for the data and for the spike
//      a_1^i e_1, storing the eliminated data g_j in place and the pivots in shared memory;
//   2. a backward recurrence that yields the block's first-row values of x~, v, w (Eq. 20);
//   3. the reduced interface system Z (Eqs. 18, 21) solved EXACTLY, framed entries included,
//      as a 2x2-block tridiagonal system over the P-1 interfaces by one thread per system;
//   4. a final backward sweep that folds the two neighbour values into the right-hand side,
//      which equals the correction x = x~ - Y y of Eq. 19.
// P = 1 is the Thomas algorithm (steps 1 and 4).
//
// The pivots use the cancellation-free "margin" recurrence: with beta_j the Thomas pivot and
// e_j = beta_j - c_j,  e_j = sigma + a_j e_{j-1} / beta_{j-1}  (all terms >= 0), so the
// weakly dominant low modes keep full relative accuracy.
//
// The singular (0, 0) mode is skipped here and solved by k_mode00.  In the FP32 forms the
// lowest modes are skipped by the FP32 pass and re-solved in FP64 by a list pass whose
// intermediates live in an FP64 scratch buffer.
#include "internal.h"

namespace pp {

struct TriParams {
  int P, m, S;        // blocks per system, rows per block, systems per CTA
  int low;            // low-mode half-width L (-1: none)
  int list;           // 1: iterate the low-mode list instead of all modes
  int nsys;           // number of systems addressed by the grid
};

__device__ __forceinline__ bool is_low(int kx, int kz, int nz, int L) {
  return L >= 0 && kx <= L && (kz <= L || kz >= nz - L);
}

template <typename TD, typename TC, bool SCR>
__global__ void __launch_bounds__(512) k_tridiag(Geometry g, TriParams tp, const TC* __restrict__ a,
                                                 const TC* __restrict__ c, const double* __restrict__ lamx,
                                                 const double* __restrict__ lamz, cplx<TD>* __restrict__ spec,
                                                 cplx<TC>* __restrict__ scratch) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int P = tp.P, m = tp.m, S = tp.S;
  const int nth = P * S;
  const int tid = threadIdx.x;
  const int b = tid / S, s = tid - b * S;
  TC* rbs = reinterpret_cast<TC*>(smem_raw);          // [m][nth] pivots 1/beta_j
  TC* gvs = rbs + (size_t)m * nth;                      // [m][nth] forward-eliminated spike
  TC* itf = gvs + (size_t)m * nth;                      // interface arrays, [18][P*S]
  const int PS = P * S;
  TC* xFr = itf;          TC* xFi = itf + PS;      TC* xLr = itf + 2 * PS;  TC* xLi = itf + 3 * PS;
  TC* vFs = itf + 4 * PS; TC* vLs = itf + 5 * PS;  TC* wFs = itf + 6 * PS;  TC* wLs = itf + 7 * PS;
  TC* alr = itf + 8 * PS; TC* ali = itf + 9 * PS;  TC* ber = itf + 10 * PS; TC* bei = itf + 11 * PS;
  TC* y0r = itf + 12 * PS; TC* y0i = itf + 13 * PS; TC* y1r = itf + 14 * PS; TC* y1i = itf + 15 * PS;
  TC* X01s = itf + 16 * PS; TC* X11s = itf + 17 * PS;

  const int sys = blockIdx.x * S + s;
  int kx = 0, kz = 0;
  bool active = sys < tp.nsys;
  if (active) {
    if (tp.list) {
      const int nlx = tp.low + 1;
      kx = sys % nlx;
      const int q = sys / nlx;
      kz = q <= tp.low ? q : g.nz - (q - tp.low);
    } else {
      kz = sys / g.ncols;
      kx = sys - kz * g.ncols;
      if (is_low(kx, kz, g.nz, tp.low)) active = false;
    }
    if (kx == 0 && kz == 0) active = false;
  }
  const TC sigma = active ? TC(-(lamx[kx] + lamz[kz])) : TC(1);
  const size_t rstride = (size_t)g.nz * g.pitch;
  cplx<TD>* col = spec + (size_t)kz * g.pitch + kx;
  cplx<TC>* scol = SCR ? scratch + sys : nullptr;
  const size_t sstride = SCR ? (size_t)tp.nsys : 0;
  const int r0 = b * m;

  // ---- 1. forward elimination ------------------------------------------------------------
  cplx<TC> gg = mk<TC>(TC(0), TC(0));
  TC e = TC(0), rbp = TC(0), gvv = TC(0);
  cplx<TC> xL = mk<TC>(TC(0), TC(0));
  TC vL = TC(0), wL = TC(0);
  if (active) {
    e = a[r0] + sigma;
    gvv = a[r0];
    for (int i = 0; i < m; ++i) {
      const int j = r0 + i;
      const cplx<TD> F = ld_c(col + (size_t)j * rstride);
      const cplx<TC> rhs = mk<TC>(-TC(F.x), -TC(F.y));
      if (i == 0) {
        gg = rhs;
      } else {
        const TC mult = a[j] * rbp;
        e = sigma + mult * e;
        gg = mk<TC>(rhs.x + mult * gg.x, rhs.y + mult * gg.y);
        gvv = mult * gvv;
      }
      const TC rb = TC(1) / (c[j] + e);
      rbs[(size_t)i * nth + tid] = rb;
      gvs[(size_t)i * nth + tid] = gvv;
      if constexpr (SCR) st_c(scol + (size_t)j * sstride, gg);
      else st_c(col + (size_t)j * rstride, gg);
      rbp = rb;
    }
    xL = scale(gg, rbp);
    vL = gvv * rbp;
    wL = c[r0 + m - 1] * rbp;
  }

  auto gload = [&](int j) -> cplx<TC> {
    if constexpr (SCR) return ld_c(scol + (size_t)j * sstride);
    else return ld_c(col + (size_t)j * rstride);
  };

  cplx<TC> alpha = mk<TC>(TC(0), TC(0)), beta = mk<TC>(TC(0), TC(0));
  if (P > 1) {
    // ---- 2. first-row values of x~, v, w --------------------------------------------------
    cplx<TC> xn = xL;
    TC vn = vL, wn = wL;
    if (active) {
      for (int i = m - 2; i >= 0; --i) {
        const int j = r0 + i;
        const TC rb = rbs[(size_t)i * nth + tid];
        const TC cj = c[j];
        const cplx<TC> gj = gload(j);
        xn = mk<TC>((gj.x + cj * xn.x) * rb, (gj.y + cj * xn.y) * rb);
        vn = (gvs[(size_t)i * nth + tid] + cj * vn) * rb;
        wn = cj * rb * wn;
      }
    }
    const int me = b * S + s;
    xFr[me] = xn.x; xFi[me] = xn.y; xLr[me] = xL.x; xLi[me] = xL.y;
    vFs[me] = vn; vLs[me] = vL; wFs[me] = wn; wLs[me] = wL;
    __syncthreads();
    // ---- 3. exact reduced system over the P-1 interfaces (unknowns L_i, F_{i+1}) --------------
    // L_i     = x~L_i + vL_i L_{i-1} + wL_i F_{i+1}
    // F_{i+1} = x~F_{i+1} + vF_{i+1} L_i + wF_{i+1} F_{i+2}
    if (b == 0 && active) {
      TC pX01 = TC(0);
      cplx<TC> py0 = mk<TC>(TC(0), TC(0));
      for (int i = 0; i < P - 1; ++i) {
        const int ii = i * S + s, in = (i + 1) * S + s;
        const TC vLi = vLs[ii], wLi = wLs[ii], vFn = vFs[in], wFi = wFs[ii];
        // eliminating z_{i-1} fills entry (0,1): L_i reaches F_{i+1} through L_{i-1} and F_i
        const TC d01 = -wLi - vLi * wFi * pX01, d10 = -vFn;
        const TC inv = TC(1) / (TC(1) - d01 * d10);
        const TC X00 = inv, X01 = -d01 * inv, X10 = -d10 * inv, X11 = inv;
        const cplx<TC> q0 = mk<TC>(xLr[ii] + vLi * py0.x, xLi[ii] + vLi * py0.y);
        const cplx<TC> q1 = mk<TC>(xFr[in], xFi[in]);
        const cplx<TC> y0 = mk<TC>(X00 * q0.x + X01 * q1.x, X00 * q0.y + X01 * q1.y);
        const cplx<TC> y1 = mk<TC>(X10 * q0.x + X11 * q1.x, X10 * q0.y + X11 * q1.y);
        y0r[ii] = y0.x; y0i[ii] = y0.y; y1r[ii] = y1.x; y1i[ii] = y1.y;
        X01s[ii] = X01; X11s[ii] = X11;
        pX01 = X01;
        py0 = y0;
      }
      cplx<TC> z1n = mk<TC>(TC(0), TC(0));   // F_{i+2}
      for (int i = P - 2; i >= 0; --i) {
        const int ii = i * S + s;
        const TC t = (i == P - 2) ? TC(0) : wFs[(i + 1) * S + s];
        const cplx<TC> z0 = mk<TC>(y0r[ii] + t * z1n.x * X01s[ii], y0i[ii] + t * z1n.y * X01s[ii]);
        const cplx<TC> z1 = mk<TC>(y1r[ii] + t * z1n.x * X11s[ii], y1i[ii] + t * z1n.y * X11s[ii]);
        alr[(i + 1) * S + s] = z0.x; ali[(i + 1) * S + s] = z0.y;   // alpha of block i+1 = L_i
        ber[ii] = z1.x; bei[ii] = z1.y;                              // beta of block i = F_{i+1}
        z1n = z1;
      }
    }
    __syncthreads();
    if (b > 0) alpha = mk<TC>(alr[me], ali[me]);
    if (b < P - 1) beta = mk<TC>(ber[me], bei[me]);
  }

  // ---- 4. final backward sweep with the neighbour values folded in --------------------------
  if (active) {
    cplx<TC> xn = beta;   // x_{r1+1}; multiplied by c_{r1} (0 for the last block)
    for (int i = m - 1; i >= 0; --i) {
      const int j = r0 + i;
      const TC rb = rbs[(size_t)i * nth + tid];
      const TC gv = gvs[(size_t)i * nth + tid];
      const TC cj = c[j];
      const cplx<TC> gj = gload(j);
      xn = mk<TC>((gj.x + alpha.x * gv + cj * xn.x) * rb, (gj.y + alpha.y * gv + cj * xn.y) * rb);
      st_c(col + (size_t)j * rstride, mk<TD>(TD(xn.x), TD(xn.y)));
    }
  }
}

// ---- PDD with per-mode factors (the production path) ----------------------------------------
// The RHS-independent part of each block's elimination (pivots, spikes, first-row weights)
// depends only on the mode, so k_tridiag_setup computes it once per plan in FP64 and stores it
// in the solve's precision.  Per solve a thread then runs, for its m rows,
//   forward : g_j = -F_j + mult_j g_{j-1},  x~_{r0} += kappa_j g_j
//   exact reduced interface system (Eq. 21, framed entries included)
//   backward: x_j = (g_j + alpha gv_j + c_j x_{j+1}) rb_j
// FULL (FP64, FP64-issue bound) reads mult and kappa from tables; the lean FP32 variant
// (HBM bound) stores only rb and gv and recomputes mult_j = a_j rb_{j-1} and
// kappa_j = rb_j prod c_l rb_l with a few FP32 multiplies.  Rows are processed in chunks of
// CH so that a thread keeps CH independent loads in flight.

__device__ __forceinline__ void sys_to_mode(int sys, int ncols, int& kx, int& kz) {
  kz = sys / ncols;
  kx = sys - kz * ncols;
}

template <typename T, bool FULL>
__global__ void __launch_bounds__(256) k_tridiag_setup(Geometry g, int P, int m, const double* __restrict__ a,
                                                       const double* __restrict__ c,
                                                       const double* __restrict__ lamx,
                                                       const double* __restrict__ lamz, TriFactors<T> tf) {
  const int nsys = tf.nsys;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (long long)nsys * P) return;
  const int b = (int)(tid / nsys), sys = (int)(tid - (long long)b * nsys);
  int kx, kz;
  sys_to_mode(sys, g.ncols, kx, kz);
  // (0,0) is solved elsewhere; give it a harmless positive shift so its factors stay finite
  const double sigma = (kx == 0 && kz == 0) ? 1.0 : -(lamx[kx] + lamz[kz]);
  const int r0 = b * m, r1 = r0 + m - 1;
  double e = a[r0] + sigma, gvv = a[r0], rbp = 0.0, run = 1.0, vF = 0.0, kap = 0.0;
  for (int i = 0; i < m; ++i) {
    const int j = r0 + i;
    double mult = 0.0;
    if (i > 0) {
      mult = a[j] * rbp;
      e = sigma + mult * e;
      gvv = mult * gvv;
    }
    const double rb = 1.0 / (c[j] + e);
    kap = run * rb;
    const size_t o = (size_t)j * nsys + sys;
    if constexpr (FULL) {
      tf.mult[o] = T(mult);
      tf.kappa[o] = T(kap);
    }
    tf.rb[o] = T(rb);
    tf.gv[o] = T(gvv);
    vF += kap * gvv;
    run *= c[j] * rb;
    rbp = rb;
  }
  const size_t ob = (size_t)b * nsys + sys;
  tf.vF[ob] = T(vF);
  tf.vL[ob] = T(gvv * rbp);
  tf.wF[ob] = T(kap * c[r1]);
  tf.wL[ob] = T(c[r1] * rbp);
}

template <typename T, bool FULL>
__global__ void __launch_bounds__(256) k_tridiag_factored(Geometry g, int P, int m, int S, int low,
                                                          const T* __restrict__ a, const T* __restrict__ c,
                                                          TriFactors<T> tf, cplx<T>* __restrict__ spec) {
  constexpr int CH = 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int PS = P * S;
  T* xFr = sm;          T* xFi = sm + PS;      T* xLr = sm + 2 * PS;  T* xLi = sm + 3 * PS;
  T* alr = sm + 4 * PS; T* ali = sm + 5 * PS;  T* ber = sm + 6 * PS;  T* bei = sm + 7 * PS;
  T* y0r = sm + 8 * PS; T* y0i = sm + 9 * PS;  T* y1r = sm + 10 * PS; T* y1i = sm + 11 * PS;
  T* X01s = sm + 12 * PS; T* X11s = sm + 13 * PS;
  const int nsys = tf.nsys;
  const int tid = threadIdx.x;
  const int b = tid / S, s = tid - b * S;
  const int sys = blockIdx.x * S + s;
  int kx = 0, kz = 0;
  bool active = sys < nsys;
  if (active) {
    sys_to_mode(sys, g.ncols, kx, kz);
    if ((kx == 0 && kz == 0) || is_low(kx, kz, g.nz, low)) active = false;
  }
  const size_t rstride = (size_t)g.nz * g.pitch;
  cplx<T>* col = spec + (size_t)kz * g.pitch + kx;
  const int r0 = b * m;
  const int me = b * S + s;
  // ---- forward elimination and the block's end values of x~ ----
  cplx<T> xF = mk<T>(T(0), T(0)), xL = mk<T>(T(0), T(0));
  if (active) {
    cplx<T> gg = mk<T>(T(0), T(0));
    T rbp = T(0), run = T(1);
    for (int i0 = 0; i0 < m; i0 += CH) {
      cplx<T> F[CH];
      T t1[CH], t2[CH];
#pragma unroll
      for (int q = 0; q < CH; ++q) {
        if (i0 + q < m) {
          const int j = r0 + i0 + q;
          const size_t o = (size_t)j * nsys + sys;
          F[q] = ld_c(col + (size_t)j * rstride);
          if constexpr (FULL) {
            t1[q] = tf.mult[o];
            t2[q] = tf.kappa[o];
          } else {
            t1[q] = tf.rb[o];
          }
        }
      }
#pragma unroll
      for (int q = 0; q < CH; ++q) {
        if (i0 + q < m) {
          const int j = r0 + i0 + q;
          T mult, kap;
          if constexpr (FULL) {
            mult = t1[q];
            kap = t2[q];
          } else {
            const T rb = t1[q];
            mult = (i0 + q == 0) ? T(0) : a[j] * rbp;
            kap = run * rb;
            run *= c[j] * rb;
            rbp = rb;
          }
          gg = mk<T>(fma(mult, gg.x, -F[q].x), fma(mult, gg.y, -F[q].y));
          xF = mk<T>(fma(kap, gg.x, xF.x), fma(kap, gg.y, xF.y));
          F[q] = gg;
        }
      }
#pragma unroll
      for (int q = 0; q < CH; ++q)
        if (i0 + q < m) st_c(col + (size_t)(r0 + i0 + q) * rstride, F[q]);
    }
    T rbl;
    if constexpr (FULL) rbl = tf.rb[(size_t)(r0 + m - 1) * nsys + sys];
    else rbl = rbp;
    xL = mk<T>(gg.x * rbl, gg.y * rbl);
  }
  cplx<T> alpha = mk<T>(T(0), T(0)), beta = mk<T>(T(0), T(0));
  if (P > 1) {
    xFr[me] = xF.x; xFi[me] = xF.y; xLr[me] = xL.x; xLi[me] = xL.y;
    __syncthreads();
    if (b == 0 && active) {
      // exact reduced system over the interfaces, unknowns z_i = (L_i, F_{i+1})
      T pX01 = T(0);
      cplx<T> py0 = mk<T>(T(0), T(0));
      for (int i = 0; i < P - 1; ++i) {
        const int ii = i * S + s, in = (i + 1) * S + s;
        const size_t bi = (size_t)i * nsys + sys, bn = (size_t)(i + 1) * nsys + sys;
        const T vLi = tf.vL[bi], wLi = tf.wL[bi], vFn = tf.vF[bn], wFi = tf.wF[bi];
        // eliminating z_{i-1} fills entry (0,1): L_i reaches F_{i+1} through L_{i-1} and F_i
        const T d01 = -wLi - vLi * wFi * pX01, d10 = -vFn;
        const T inv = T(1) / (T(1) - d01 * d10);
        const T X00 = inv, X01 = -d01 * inv, X10 = -d10 * inv, X11 = inv;
        const cplx<T> q0 = mk<T>(xLr[ii] + vLi * py0.x, xLi[ii] + vLi * py0.y);
        const cplx<T> q1 = mk<T>(xFr[in], xFi[in]);
        const cplx<T> y0 = mk<T>(X00 * q0.x + X01 * q1.x, X00 * q0.y + X01 * q1.y);
        const cplx<T> y1 = mk<T>(X10 * q0.x + X11 * q1.x, X10 * q0.y + X11 * q1.y);
        y0r[ii] = y0.x; y0i[ii] = y0.y; y1r[ii] = y1.x; y1i[ii] = y1.y;
        X01s[ii] = X01; X11s[ii] = X11;
        pX01 = X01;
        py0 = y0;
      }
      cplx<T> z1n = mk<T>(T(0), T(0));
      for (int i = P - 2; i >= 0; --i) {
        const int ii = i * S + s;
        const T tw = (i == P - 2) ? T(0) : tf.wF[(size_t)(i + 1) * nsys + sys];
        const cplx<T> z0 = mk<T>(y0r[ii] + tw * z1n.x * X01s[ii], y0i[ii] + tw * z1n.y * X01s[ii]);
        const cplx<T> z1 = mk<T>(y1r[ii] + tw * z1n.x * X11s[ii], y1i[ii] + tw * z1n.y * X11s[ii]);
        alr[(i + 1) * S + s] = z0.x; ali[(i + 1) * S + s] = z0.y;   // alpha of block i+1 = L_i
        ber[ii] = z1.x; bei[ii] = z1.y;                              // beta of block i = F_{i+1}
        z1n = z1;
      }
    }
    __syncthreads();
    if (b > 0) alpha = mk<T>(alr[me], ali[me]);
    if (b < P - 1) beta = mk<T>(ber[me], bei[me]);
  }
  // ---- backward sweep with the neighbour values folded in ----
  if (active) {
    cplx<T> xn = beta;
    for (int i1 = m; i1 > 0; i1 -= CH) {
      cplx<T> G[CH];
      T rbv[CH], gvv[CH];
#pragma unroll
      for (int q = 0; q < CH; ++q) {
        const int i = i1 - 1 - q;
        if (i >= 0) {
          const int j = r0 + i;
          const size_t o = (size_t)j * nsys + sys;
          G[q] = ld_c(col + (size_t)j * rstride);
          rbv[q] = tf.rb[o];
          gvv[q] = tf.gv[o];
        }
      }
#pragma unroll
      for (int q = 0; q < CH; ++q) {
        const int i = i1 - 1 - q;
        if (i >= 0) {
          const T cj = c[r0 + i];
          const T tx = fma(cj, xn.x, fma(alpha.x, gvv[q], G[q].x));
          const T ty = fma(cj, xn.y, fma(alpha.y, gvv[q], G[q].y));
          xn = mk<T>(tx * rbv[q], ty * rbv[q]);
          G[q] = xn;
        }
      }
#pragma unroll
      for (int q = 0; q < CH; ++q) {
        const int i = i1 - 1 - q;
        if (i >= 0) st_c(col + (size_t)(r0 + i) * rstride, G[q]);
      }
    }
  }
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

template <typename TD>
__global__ void __launch_bounds__(32) k_mode00(Geometry g, const double* __restrict__ dy,
                                               const double* __restrict__ h, cplx<TD>* __restrict__ spec,
                                               double* __restrict__ acc, int gauge) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* fr = reinterpret_cast<double*>(smem_raw);
  double* fi = fr + g.ny;
  const int lane = threadIdx.x;
  const int ny = g.ny;
  const int ch = (ny + 31) / 32;
  const int lo = lane * ch, hi = min(ny, lo + ch);
  const size_t rstride = (size_t)g.nz * g.pitch;
  double sr = 0, si = 0, sw = 0;
  for (int j = lo; j < hi; ++j) {
    const cplx<TD> F = ld_c(spec + (size_t)j * rstride);
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

// ------------------------------------------------------------------------------ launchers
template <typename K>
static cudaError_t prep(K kernel, size_t smem) {
  return ensure_smem_limit((const void*)kernel, smem);
}

template <typename TC> static const TC* coef_a(const DevTables& tb);
template <> const double* coef_a<double>(const DevTables& tb) { return tb.d.a; }
template <> const float* coef_a<float>(const DevTables& tb) { return tb.f.a; }
template <typename TC> static const TC* coef_c(const DevTables& tb);
template <> const double* coef_c<double>(const DevTables& tb) { return tb.d.c; }
template <> const float* coef_c<float>(const DevTables& tb) { return tb.f.c; }

static size_t tridiag_smem(int P, int m, int S, size_t tc) {
  return ((size_t)2 * m * P * S + (size_t)18 * P * S) * tc;
}

static int pick_systems_per_cta(int P, int m, size_t tc) {
  int S = 32;
  while (S > 8 && (tridiag_smem(P, m, S, tc) > 100 * 1024 || P * S > 512)) S /= 2;
  while (S > 1 && (tridiag_smem(P, m, S, tc) > 200 * 1024 || P * S > 512)) S /= 2;
  return S;
}

template <typename TD, typename TC, bool SCR>
cudaError_t launch_tridiag_impl(const Geometry& g, const DevTables& tb, int parts, int low_modes, bool low_list,
                                cplx<TD>* spec, cplx<TC>* scratch, cudaStream_t st) {
  TriParams tp;
  tp.P = parts;
  tp.m = g.ny / parts;
  tp.low = low_modes;
  tp.list = low_list ? 1 : 0;
  tp.nsys = low_list ? (low_modes + 1) * (2 * low_modes + 1) : g.nz * g.ncols;
  tp.S = pick_systems_per_cta(tp.P, tp.m, sizeof(TC));
  const size_t smem = tridiag_smem(tp.P, tp.m, tp.S, sizeof(TC));
  const dim3 grid((tp.nsys + tp.S - 1) / tp.S);
  auto kern = k_tridiag<TD, TC, SCR>;
  cudaError_t e;
  if ((e = prep(kern, smem)) != cudaSuccess) return e;
  kern<<<grid, tp.P * tp.S, smem, st>>>(g, tp, coef_a<TC>(tb), coef_c<TC>(tb), tb.lamx, tb.lamz, spec, scratch);
  return cudaGetLastError();
}

template <>
cudaError_t launch_tridiag<double, double>(const Geometry& g, const DevTables& tb, int parts, int low_modes,
                                           bool low_list, cplx<double>* spec, cudaStream_t st) {
  return launch_tridiag_impl<double, double, false>(g, tb, parts, low_modes, low_list, spec, nullptr, st);
}
template <>
cudaError_t launch_tridiag<float, float>(const Geometry& g, const DevTables& tb, int parts, int low_modes,
                                         bool low_list, cplx<float>* spec, cudaStream_t st) {
  return launch_tridiag_impl<float, float, false>(g, tb, parts, low_modes, low_list, spec, nullptr, st);
}

cudaError_t launch_tridiag_low64(const Geometry& g, const DevTables& tb, int parts, int low_modes,
                                 cplx<float>* spec, cplx<double>* scratch, cudaStream_t st) {
  return launch_tridiag_impl<float, double, true>(g, tb, parts, low_modes, true, spec, scratch, st);
}

cudaError_t launch_tridiag_setup(const Geometry& g, const DevTables& tb, int parts, cudaStream_t st) {
  if (tb.tri_d.nsys) {
    const long long n = (long long)tb.tri_d.nsys * parts;
    k_tridiag_setup<double, true><<<(int)((n + 255) / 256), 256, 0, st>>>(g, parts, g.ny / parts, tb.d.a, tb.d.c,
                                                                          tb.lamx, tb.lamz, tb.tri_d);
  }
  if (tb.tri_f.nsys) {
    const long long n = (long long)tb.tri_f.nsys * parts;
    k_tridiag_setup<float, false><<<(int)((n + 255) / 256), 256, 0, st>>>(g, parts, g.ny / parts, tb.d.a, tb.d.c,
                                                                          tb.lamx, tb.lamz, tb.tri_f);
  }
  return cudaGetLastError();
}

template <typename T, bool FULL>
static cudaError_t launch_factored(const Geometry& g, const T* a, const T* c, const TriFactors<T>& tf, int parts,
                                   int low, cplx<T>* spec, cudaStream_t st) {
  int S = 256 / parts;
  if (S < 1) S = 1;
  if (S > 32) S = 32;
  const size_t smem = (size_t)14 * parts * S * sizeof(T);
  const int blocks = (tf.nsys + S - 1) / S;
  auto kern = k_tridiag_factored<T, FULL>;
  cudaError_t e;
  if ((e = prep(kern, smem)) != cudaSuccess) return e;
  kern<<<blocks, parts * S, smem, st>>>(g, parts, g.ny / parts, S, low, a, c, tf, spec);
  return cudaGetLastError();
}

cudaError_t launch_tridiag_factored(const Geometry& g, const DevTables& tb, int parts, cplx<double>* spec,
                                    cudaStream_t st) {
  return launch_factored<double, true>(g, tb.d.a, tb.d.c, tb.tri_d, parts, -1, spec, st);
}

cudaError_t launch_tridiag_factored_f32(const Geometry& g, const DevTables& tb, int parts, int low_modes,
                                        cplx<float>* spec, cudaStream_t st) {
  return launch_factored<float, false>(g, tb.f.a, tb.f.c, tb.tri_f, parts, low_modes, spec, st);
}

template <typename TD>
cudaError_t launch_mode00(const Geometry& g, const DevTables& tb, GaugeMode gauge, cplx<TD>* spec, cudaStream_t st) {
  const size_t smem = 2 * (size_t)g.ny * sizeof(double);
  auto kern = k_mode00<TD>;
  cudaError_t e;
  if ((e = prep(kern, smem)) != cudaSuccess) return e;
  kern<<<1, 32, smem, st>>>(g, tb.dy, tb.h, spec, tb.acc, (int)gauge);
  return cudaGetLastError();
}
template cudaError_t launch_mode00<double>(const Geometry&, const DevTables&, GaugeMode, cplx<double>*,
                                           cudaStream_t);
template cudaError_t launch_mode00<float>(const Geometry&, const DevTables&, GaugeMode, cplx<float>*, cudaStream_t);

}  // namespace pp
