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
#include "tridiag_scan.cuh"

namespace pp {

struct TriParams {
  int P, m, S;        // blocks per system, rows per block, systems per CTA
  int low;            // low-mode half-width L (-1: none)
  int list;           // 1: iterate the low-mode list instead of all modes
  int nsys;           // number of systems addressed by the grid
};

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
__global__ void __launch_bounds__(256) k_tridiag_factored(Geometry g, int P, int m, int S, int low, int trunc,
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
        // truncated (Sec. 2.2): the framed entries v_m^i and w_1^{i+1} of Z are dropped
        const T vLi = trunc ? T(0) : tf.vL[bi], wLi = tf.wL[bi], vFn = tf.vF[bn], wFi = tf.wF[bi];
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
        const T tw = (i == P - 2 || trunc) ? T(0) : tf.wF[(size_t)(i + 1) * nsys + sys];
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

// ---- FP32 PDD with thread-private blocks (the FP32 production path) -------------------------
// One thread owns one block of M rows of one system.  It copies its M rows into a private slice
// of shared memory with 8-byte cp.async (all M copies in flight, no register staging; layout
// [row][thread], so every shared access of a warp is conflict-free), eliminates forward while
// building the block's pivots and spike on the fly in FP32 (margin recurrence, reciprocal by
// MUFU plus one Newton step) and keeping them in registers, exchanges the block-end values
// through shared memory for the exact reduced interface system, and sweeps back, storing each
// result straight to global memory.  The spectrum crosses HBM once in each direction and no
// factor table is read.  Threads are numbered block-major (tid = b * S + s), so a warp's row
// accesses are S-system contiguous segments.

// Per-mode LU of the reduced interface system, built once per plan in FP64 (RHS-independent).
// For interface i (between blocks i and i+1) of system sys, entry k of
// table[(sys*(P-1) + i)*5 + k] (one contiguous record per system):
//   0: vL_i      the spike v of block i at its last row
//   1: inv_i     1 / (1 - d01 d10),  d01 = -wL_i - vL_i wF_i X01_{i-1},  d10 = -vF_{i+1}
//   2: X01_i     -d01 inv_i
//   3: X10_i     -d10 inv_i
//   4: wF_{i+1}  the spike w of block i+1 at its first row (0 for the last interface)
// One thread per system walks the blocks in order, keeping two blocks' spike values.
__device__ void block_spikes64(const double* a, const double* c, double sigma, int r0, int m, double& vF,
                               double& vL, double& wF, double& wL) {
  double e = a[r0] + sigma, gvv = a[r0], rbp = 0.0, run = 1.0, kap = 0.0;
  vF = 0.0;
  for (int i = 0; i < m; ++i) {
    const int j = r0 + i;
    if (i > 0) {
      const double mult = a[j] * rbp;
      e = sigma + mult * e;
      gvv = mult * gvv;
    }
    const double rb = 1.0 / (c[j] + e);
    kap = run * rb;
    vF += kap * gvv;
    run *= c[j] * rb;
    rbp = rb;
  }
  vL = gvv * rbp;
  wF = kap * c[r0 + m - 1];
  wL = c[r0 + m - 1] * rbp;
}

__global__ void __launch_bounds__(128) k_reduced_setup(Geometry g, int P, int m, int trunc, const double* __restrict__ a,
                                                      const double* __restrict__ c, const double* __restrict__ lamx,
                                                      const double* __restrict__ lamz, float* __restrict__ tab) {
  const int nsys = g.nz * g.ncols;
  const int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= nsys) return;
  int kx, kz;
  sys_to_mode(sys, g.ncols, kx, kz);
  const double sigma = (kx == 0 && kz == 0) ? 1.0 : -(lamx[kx] + lamz[kz]);
  double vF0, vL0, wF0, wL0;
  block_spikes64(a, c, sigma, 0, m, vF0, vL0, wF0, wL0);
  double pX01 = 0.0;
  for (int i = 0; i < P - 1; ++i) {
    double vF1, vL1, wF1, wL1;
    block_spikes64(a, c, sigma, (i + 1) * m, m, vF1, vL1, wF1, wL1);
    // truncated (Sec. 2.2): without the framed entries v_m^i, w_1^{i+1} every interface is an
    // independent 2x2 system (no recurrence: vL and tw stored as 0)
    const double d01 = trunc ? -wL0 : -wL0 - vL0 * wF0 * pX01, d10 = -vF1;
    const double inv = 1.0 / (1.0 - d01 * d10);
    const double X01 = -d01 * inv, X10 = -d10 * inv;
    float* t = tab + ((size_t)sys * (P - 1) + i) * 5;
    t[0] = trunc ? 0.f : float(vL0);
    t[1] = float(inv);
    t[2] = float(X01);
    t[3] = float(X10);
    t[4] = (i + 1 < P - 1 && !trunc) ? float(wF1) : 0.f;
    pX01 = X01;
    vF0 = vF1; vL0 = vL1; wF0 = wF1; wL0 = wL1;
  }
}

template <int M>
__global__ void __launch_bounds__(256, 2) k_tridiag_reg(Geometry g, int P, int S, int low, const float* __restrict__ a,
                                                        const float* __restrict__ c, const double* __restrict__ lamx,
                                                        const double* __restrict__ lamz, const float* __restrict__ rtab,
                                                        cplx<float>* __restrict__ spec) {
  // shared: the interface arrays (6 x NT floats), the CTA's slice of the reduced-system table
  // (5 (P-1) S floats, [i][k][s]), then the blocks' rows [row][thread]
  extern __shared__ __align__(16) float red_s[];
  enum { R_XFR, R_XFI, R_XLR, R_XLI, R_ZR, R_ZI };
  const int NT = P * S;
#define RED(k, idx) red_s[(k) * NT + (idx)]
  float* tsh = red_s + 6 * NT;
  float2* Xs = reinterpret_cast<float2*>(tsh + ((5 * (P - 1) * S + 1) & ~1));
  const int nsys = g.nz * g.ncols;
  const int tid = threadIdx.x;
  const int b = tid / S, s = tid - b * S;
  const int sys0 = blockIdx.x * S;
  const int sys = sys0 + s;
  int kx = 0, kz = 0;
  bool active = sys < nsys;
  if (active) {
    sys_to_mode(sys, g.ncols, kx, kz);
    if ((kx == 0 && kz == 0) || is_low(kx, kz, g.nz, low)) active = false;
  }
  const size_t rstride = (size_t)g.nz * g.pitch;
  float2* col = reinterpret_cast<float2*>(spec + (size_t)kz * g.pitch + kx);
  const int r0 = b * M;
  if (active) {
    const float2* src = col + (size_t)r0 * rstride;
#pragma unroll 1
    for (int i = 0; i < M; ++i, src += rstride) cp_async8(&Xs[i * NT + tid], src);
  }
  for (int q = tid; q < 5 * (P - 1) * S; q += NT) {   // the reduced-system table slice, [i][k][s]
    const int qs = q / (5 * (P - 1)), ik = q - qs * 5 * (P - 1);
    if (sys0 + qs < nsys) cp_async4(&tsh[ik * S + qs], &rtab[(size_t)(sys0 + qs) * 5 * (P - 1) + ik]);
  }
  float rbv[M], gvv[M];
  if (active) {
    const float sigma = float(-(lamx[kx] + lamz[kz]));
    cp_async_wait_all();
    float e = a[r0] + sigma, gv = a[r0], rb = rcp_nr(c[r0] + e);
    float run = 1.f;
    float2 gg = make_float2(0.f, 0.f);
    float2 xF = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < M; ++i) {
      const int j = r0 + i;
      const float cj = c[j];
      const float2 F = Xs[i * NT + tid];
      float mult = 0.f;
      if (i > 0) {
        mult = a[j] * rb;
        e = fmaf(mult, e, sigma);
        gv = mult * gv;
        rb = rcp_nr(cj + e);
      }
      gg = make_float2(fmaf(mult, gg.x, -F.x), fmaf(mult, gg.y, -F.y));
      Xs[i * NT + tid] = gg;
      rbv[i] = rb;
      gvv[i] = gv;
      const float kap = run * rb;
      xF.x = fmaf(kap, gg.x, xF.x);
      xF.y = fmaf(kap, gg.y, xF.y);
      run *= cj * rb;
    }
    RED(R_XFR, tid) = xF.x; RED(R_XFI, tid) = xF.y;
    RED(R_XLR, tid) = gg.x * rb; RED(R_XLI, tid) = gg.y * rb;
  } else {
    cp_async_wait_all();
  }
  float2 alpha = make_float2(0.f, 0.f), beta = make_float2(0.f, 0.f);
  if (P > 1) {
    __syncthreads();
    if (b == 0 && active) {
      // forward: y_i = [inv X01; X10 inv] (xL_i + vL_i y0_{i-1}, xF_{i+1}); y0 kept in R_Z, y1 in
      // the block's xF slot (no longer needed)
      float2 py0 = make_float2(0.f, 0.f);
      for (int i = 0; i < P - 1; ++i) {
        const int ii = i * S + s, in = ii + S;
        const float* t = tsh + i * 5 * S + s;
        const float vL = t[0], inv = t[S], X01 = t[2 * S], X10 = t[3 * S];
        const float q0x = fmaf(vL, py0.x, RED(R_XLR, ii)), q0y = fmaf(vL, py0.y, RED(R_XLI, ii));
        const float q1x = RED(R_XFR, in), q1y = RED(R_XFI, in);
        py0 = make_float2(fmaf(inv, q0x, X01 * q1x), fmaf(inv, q0y, X01 * q1y));
        RED(R_ZR, ii) = py0.x; RED(R_ZI, ii) = py0.y;
        RED(R_XFR, in) = fmaf(X10, q0x, inv * q1x); RED(R_XFI, in) = fmaf(X10, q0y, inv * q1y);
      }
      // backward: z1_i = y1_i + wF_{i+1} inv_i z1_{i+1}, z0_i = y0_i + wF_{i+1} X01_i z1_{i+1};
      // alpha of block i+1 = z0_i (stored in its R_XL slot), beta of block i = z1_i (R_Z slot)
      float2 z1n = make_float2(0.f, 0.f);
      for (int i = P - 2; i >= 0; --i) {
        const int ii = i * S + s, in = ii + S;
        const float* t = tsh + i * 5 * S + s;
        const float inv = t[S], X01 = t[2 * S], tw = t[4 * S];
        const float a0 = tw * X01, a1 = tw * inv;
        const float z0x = fmaf(a0, z1n.x, RED(R_ZR, ii)), z0y = fmaf(a0, z1n.y, RED(R_ZI, ii));
        z1n = make_float2(fmaf(a1, z1n.x, RED(R_XFR, in)), fmaf(a1, z1n.y, RED(R_XFI, in)));
        RED(R_XLR, in) = z0x; RED(R_XLI, in) = z0y;
        RED(R_ZR, ii) = z1n.x; RED(R_ZI, ii) = z1n.y;
      }
    }
    __syncthreads();
    if (b > 0) alpha = make_float2(RED(R_XLR, tid), RED(R_XLI, tid));
    if (b < P - 1) beta = make_float2(RED(R_ZR, tid), RED(R_ZI, tid));
  }
#undef RED
  if (active) {
    float2 xn = beta;
    float2* dst = col + (size_t)(r0 + M - 1) * rstride;
#pragma unroll
    for (int i = M - 1; i >= 0; --i) {
      const float cj = c[r0 + i];
      const float2 G = Xs[i * NT + tid];
      const float tx = fmaf(cj, xn.x, fmaf(alpha.x, gvv[i], G.x));
      const float ty = fmaf(cj, xn.y, fmaf(alpha.y, gvv[i], G.y));
      xn = make_float2(tx * rbv[i], ty * rbv[i]);
      *dst = xn;
      dst -= rstride;
    }
  }
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
                                   int low, bool trunc, cplx<T>* spec, cudaStream_t st) {
  int S = 256 / parts;
  if (S < 1) S = 1;
  if (S > 32) S = 32;
  const size_t smem = (size_t)14 * parts * S * sizeof(T);
  const int blocks = (tf.nsys + S - 1) / S;
  auto kern = k_tridiag_factored<T, FULL>;
  cudaError_t e;
  if ((e = prep(kern, smem)) != cudaSuccess) return e;
  kern<<<blocks, parts * S, smem, st>>>(g, parts, g.ny / parts, S, low, trunc ? 1 : 0, a, c, tf, spec);
  return cudaGetLastError();
}

size_t reduced_table_bytes(const Geometry& g, int parts) {
  return parts > 1 ? (size_t)5 * (parts - 1) * g.nz * g.ncols * sizeof(float) : 0;
}

cudaError_t launch_reduced_setup(const Geometry& g, const DevTables& tb, int parts, bool trunc, float* tab,
                                 cudaStream_t st) {
  if (parts <= 1) return cudaSuccess;
  const int nsys = g.nz * g.ncols;
  k_reduced_setup<<<(nsys + 127) / 128, 128, 0, st>>>(g, parts, g.ny / parts, trunc ? 1 : 0, tb.d.a, tb.d.c, tb.lamx,
                                                       tb.lamz, tab);
  return cudaGetLastError();
}

cudaError_t launch_tridiag_reg_f32(const Geometry& g, const DevTables& tb, int parts, int low_modes,
                                   cplx<float>* spec, cudaStream_t st, int kx_lo, int kx_hi) {
  if (!reg_tridiag_ok(g.ny, parts)) return cudaErrorNotSupported;
  const int m = g.ny / parts;
  const int S = reg_systems_per_cta(parts);
  if (kx_hi < 0) kx_hi = g.ncols;
  const bool whole = kx_lo == 0 && kx_hi == g.ncols;
  if (kx_lo < 0 || kx_hi > g.ncols || kx_hi <= kx_lo) return cudaErrorInvalidValue;
  if (!whole && (!scan_tridiag_ok(g.ny, parts) || kx_lo % S)) return cudaErrorNotSupported;
  if (scan_tridiag_ok(g.ny, parts)) {   // warp-scan variant
    const int nt = parts * S;
    const size_t smem = (size_t)parts * (m * S + 1) * 8 + (size_t)2 * parts * (m | 1) * 4;
    const int blocks = g.nz * ((kx_hi - kx_lo + S - 1) / S);
#define PP_SCAN_CASE(MM)                                                                                       \
  case MM: {                                                                                                   \
    cudaError_t e = prep(k_tridiag_scan<MM>, smem);                                                            \
    if (e != cudaSuccess) return e;                                                                            \
    k_tridiag_scan<MM><<<blocks, nt, smem, st>>>(g, parts, S, low_modes, tb.f.a, tb.f.c, tb.lamx, tb.lamz,     \
                                                 tb.red_f, spec, kx_lo, kx_hi);                                \
    return cudaGetLastError();                                                                                 \
  }
    switch (m) {
      PP_SCAN_CASE(1) PP_SCAN_CASE(2) PP_SCAN_CASE(3) PP_SCAN_CASE(4) PP_SCAN_CASE(6) PP_SCAN_CASE(8)
      PP_SCAN_CASE(12) PP_SCAN_CASE(16) PP_SCAN_CASE(24)
      default: break;
    }
#undef PP_SCAN_CASE
  }
  const int nt = parts * S;
  const size_t tabf = ((size_t)5 * (parts - 1) * S + 1) & ~(size_t)1;
  const size_t smem = (size_t)6 * nt * sizeof(float) + tabf * sizeof(float) + (size_t)m * 8 * nt;
  const int nsys = g.nz * g.ncols;
  const int blocks = (nsys + S - 1) / S;
#define PP_REG_CASE(MM)                                                                                         \
  case MM: {                                                                                                    \
    cudaError_t e = prep(k_tridiag_reg<MM>, smem);                                                              \
    if (e != cudaSuccess) return e;                                                                             \
    k_tridiag_reg<MM><<<blocks, nt, smem, st>>>(g, parts, S, low_modes, tb.f.a, tb.f.c, tb.lamx, tb.lamz,       \
                                                tb.red_f, spec);                                                \
    break;                                                                                                      \
  }
  switch (m) {
    PP_REG_CASE(1) PP_REG_CASE(2) PP_REG_CASE(3) PP_REG_CASE(4) PP_REG_CASE(6) PP_REG_CASE(8)
    PP_REG_CASE(12) PP_REG_CASE(16) PP_REG_CASE(24)
    default: return cudaErrorNotSupported;
  }
#undef PP_REG_CASE
  return cudaGetLastError();
}

cudaError_t launch_tridiag_factored(const Geometry& g, const DevTables& tb, int parts, bool trunc, cplx<double>* spec,
                                    cudaStream_t st) {
  return launch_factored<double, true>(g, tb.d.a, tb.d.c, tb.tri_d, parts, -1, trunc, spec, st);
}

cudaError_t launch_tridiag_factored_f32(const Geometry& g, const DevTables& tb, int parts, int low_modes, bool trunc,
                                        cplx<float>* spec, cudaStream_t st) {
  return launch_factored<float, false>(g, tb.f.a, tb.f.c, tb.tri_f, parts, low_modes, trunc, spec, st);
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
