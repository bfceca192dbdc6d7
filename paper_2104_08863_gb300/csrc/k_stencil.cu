// Pointwise stencil passes around the solve.
//
//  k_gradient  : the velocity correction of Eq. 4, u <- u - dt G p, on the staggered faces;
//                wall faces of v are boundary values and are left unchanged (Sec. 2).
//  k_adj_epi   : the adjoint epilogue g <- g - D^T q with q = W p' (W = diag(dy_j)), where p'
//                solves L_h p' = W^-1 G^T g; this is P^T g = g - D^T S^T G^T g because
//                L_h^T = W L_h W^-1 and the forward gauge (zero dy-weighted mean of p') is the
//                zero-sum gauge of q.
//  k_check_finite : sets the device status word when a value is NaN or Inf.
//  k_divergence : f = D(u)/dt of Eq. 7 on the cell centres (the right-hand side of the
//                pressure equation), for callers that want it as a field.
#include "fpconv.cuh"
#include "internal.h"

namespace pp {

// Lines [lbeg, lend) of the (ny + 1) nz face lines (line = j nz + k).
template <typename T>
__global__ void __launch_bounds__(256) k_gradient(Geometry g, const T* __restrict__ p, T* __restrict__ u,
                                                  T* __restrict__ v, T* __restrict__ w,
                                                  const T* __restrict__ inv_h, T dt, int lbeg, int lend) {
  const size_t plane = (size_t)g.nz * g.nx;
  const T cx = T(dt / g.dx), cz = T(dt / g.dz);
  for (int line = lbeg + blockIdx.x; line < lend; line += gridDim.x)
  for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
    const int j = line / g.nz, k = line - j * g.nz;
    const size_t idx = (size_t)line * g.nx + i;
    if (j < g.ny) {
      const T pc = p[idx];
      const T pxm = p[idx - i + (i == 0 ? g.nx - 1 : i - 1)];
      const T pzm = p[(size_t)j * plane + (size_t)(k == 0 ? g.nz - 1 : k - 1) * g.nx + i];
      u[idx] -= cx * (pc - pxm);
      w[idx] -= cz * (pc - pzm);
    }
    if (j >= 1 && j <= g.ny - 1) {
      const T cy = dt * inv_h[j];
      v[idx] -= cy * (p[idx] - p[idx - plane]);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_adj_epi(Geometry g, const T* __restrict__ pp_, T* __restrict__ gu,
                                                 T* __restrict__ gv, T* __restrict__ gw,
                                                 const double* __restrict__ dy) {
  const size_t plane = (size_t)g.nz * g.nx;
  const int nlines = (g.ny + 1) * g.nz;
  const T ix = T(1.0 / g.dx), iz = T(1.0 / g.dz);
  for (int line = blockIdx.x; line < nlines; line += gridDim.x)
  for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
    const int j = line / g.nz, k = line - j * g.nz;
    const size_t idx = (size_t)line * g.nx + i;
    if (j < g.ny) {
      const T dyj = T(dy[j]);
      const T pc = pp_[idx];
      const T pxm = pp_[idx - i + (i == 0 ? g.nx - 1 : i - 1)];
      const T pzm = pp_[(size_t)j * plane + (size_t)(k == 0 ? g.nz - 1 : k - 1) * g.nx + i];
      gu[idx] -= dyj * (pxm - pc) * ix;
      gw[idx] -= dyj * (pzm - pc) * iz;
    }
    // (D_y^T q)_f = q_{f-1}/dy_{f-1} - q_f/dy_f = p'_{f-1} - p'_f  (terms outside 0..ny-1 vanish)
    T t = T(0);
    if (j >= 1) t += pp_[idx - plane];
    if (j <= g.ny - 1) t -= pp_[idx];
    gv[idx] -= t;
  }
}

// out[j][k][i] = in[j][k][i] * s_j with s_j = 1/dy_j (to_weighted = false) or dy_j (true): the
// diagonal volume weights W^-1 and W of the transposed solve (L_h^T = W L_h W^-1).
template <typename T>
__global__ void __launch_bounds__(256) k_scale_planes(Geometry g, const T* __restrict__ in, T* __restrict__ out,
                                                      const double* __restrict__ dy, int to_weighted) {
  const int nlines = g.ny * g.nz;
  for (int line = blockIdx.x; line < nlines; line += gridDim.x) {
    const int j = line / g.nz;
    const T sj = to_weighted ? T(dy[j]) : T(1.0 / dy[j]);
    const size_t base = (size_t)line * g.nx;
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x) out[base + i] = in[base + i] * sj;
  }
}

// q[j][k][i] = dy_j (hi + lo): the FP64 value of the refined solve's FP32 pair, weighted.
__global__ void __launch_bounds__(256) k_weighted_pair(Geometry g, const float* __restrict__ hi,
                                                       const float* __restrict__ lo, double* __restrict__ q,
                                                       const double* __restrict__ dy) {
  const int nlines = g.ny * g.nz;
  for (int line = blockIdx.x; line < nlines; line += gridDim.x) {
    const double w = dy[line / g.nz];
    const size_t base = (size_t)line * g.nx;
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x)
      q[base + i] = w * f32_add_to_f64(hi[base + i], lo ? lo[base + i] : 0.0f);
  }
}

template <typename T>
__global__ void k_check_finite(const T* __restrict__ x, size_t n, int* status) {
  bool bad = false;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    bad |= !isfinite(x[i]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch(status, (int)DEV_NONFINITE);
}

template <typename T>
__global__ void __launch_bounds__(256) k_divergence(Geometry g, const T* __restrict__ u, const T* __restrict__ v,
                                                    const T* __restrict__ w, T* __restrict__ f,
                                                    const T* __restrict__ inv_dy, T inv_dt) {
  const size_t plane = (size_t)g.nz * g.nx;
  const int nlines = g.ny * g.nz;
  const T ix = T(1.0 / g.dx), iz = T(1.0 / g.dz);
  for (int line = blockIdx.x; line < nlines; line += gridDim.x) {
    const int j = line / g.nz, k = line - j * g.nz;
    const T iy = inv_dy[j];
    const size_t row = (size_t)line * g.nx;
    const size_t rkp = (size_t)j * plane + (size_t)(k + 1 == g.nz ? 0 : k + 1) * g.nx;
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
      const size_t idx = row + i;
      const T dux = u[row + (i + 1 == g.nx ? 0 : i + 1)] - u[idx];
      const T dvy = v[idx + plane] - v[idx];
      const T dwz = w[rkp + i] - w[idx];
      f[idx] = (dux * ix + dvy * iy + dwz * iz) * inv_dt;
    }
  }
}

static int stream_grid(size_t total) {
  size_t blocks = (total + 255) / 256;
  const size_t cap = 152 * 16;
  return (int)(blocks < cap ? (blocks ? blocks : 1) : cap);
}

// Line-wise launch of the face stencils: one CTA per x-line at a time (grid-stride over the
// (ny+1) nz lines), threads over x, so no per-element 64-bit index division.
static int line_grid(const Geometry& g) {
  const int nlines = (g.ny + 1) * g.nz;
  const int cap = 152 * 16;
  return nlines < cap ? nlines : cap;
}
static int line_block(const Geometry& g) { return g.nx >= 256 ? 256 : (g.nx + 31) / 32 * 32; }

template <typename T> static const T* inv_h_table(const DevTables& tb);
template <> const double* inv_h_table<double>(const DevTables& tb) { return tb.d.inv_h; }
template <> const float* inv_h_table<float>(const DevTables& tb) { return tb.f.inv_h; }

template <typename T>
cudaError_t launch_gradient(const Geometry& g, const DevTables& tb, const T* p, T* u, T* v, T* w, double dt,
                            cudaStream_t st, int jlo, int jhi) {
  if (jhi < 0) jhi = g.ny;
  if (jlo < 0 || jhi > g.ny || jhi <= jlo) return cudaErrorInvalidValue;
  const int lbeg = jlo * g.nz, lend = (jhi == g.ny ? g.ny + 1 : jhi) * g.nz;
  const int cap = line_grid(g);
  k_gradient<T><<<lend - lbeg < cap ? lend - lbeg : cap, line_block(g), 0, st>>>(g, p, u, v, w, inv_h_table<T>(tb),
                                                                                  T(dt), lbeg, lend);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adjoint_epilogue(const Geometry& g, const DevTables& tb, const T* q, T* gu, T* gv, T* gw,
                                    cudaStream_t st) {
  k_adj_epi<T><<<line_grid(g), line_block(g), 0, st>>>(g, q, gu, gv, gw, tb.dy);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scale_planes(const Geometry& g, const DevTables& tb, const T* in, T* out, bool to_weighted,
                                cudaStream_t st) {
  const int nlines = g.ny * g.nz, cap = 152 * 16;
  k_scale_planes<T><<<nlines < cap ? nlines : cap, line_block(g), 0, st>>>(g, in, out, tb.dy, to_weighted ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_weighted_pair(const Geometry& g, const DevTables& tb, const float* hi, const float* lo, double* q,
                                 cudaStream_t st) {
  const int nlines = g.ny * g.nz, cap = 152 * 16;
  k_weighted_pair<<<nlines < cap ? nlines : cap, line_block(g), 0, st>>>(g, hi, lo, q, tb.dy);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_divergence(const Geometry& g, const DevTables& tb, const T* u, const T* v, const T* w, T* f,
                              double dt, cudaStream_t st) {
  const int nlines = g.ny * g.nz, cap = 152 * 16;
  const T* inv_dy = sizeof(T) == 8 ? (const T*)tb.d.inv_dy : (const T*)tb.f.inv_dy;
  k_divergence<T><<<nlines < cap ? nlines : cap, line_block(g), 0, st>>>(g, u, v, w, f, inv_dy, T(1.0 / dt));
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_check_finite(const T* x, size_t n, int* status, cudaStream_t st) {
  k_check_finite<T><<<stream_grid(n), 256, 0, st>>>(x, n, status);
  return cudaGetLastError();
}

template cudaError_t launch_gradient<double>(const Geometry&, const DevTables&, const double*, double*, double*,
                                             double*, double, cudaStream_t, int, int);
template cudaError_t launch_gradient<float>(const Geometry&, const DevTables&, const float*, float*, float*, float*,
                                            double, cudaStream_t, int, int);
template cudaError_t launch_adjoint_epilogue<double>(const Geometry&, const DevTables&, const double*, double*,
                                                     double*, double*, cudaStream_t);
template cudaError_t launch_adjoint_epilogue<float>(const Geometry&, const DevTables&, const float*, float*, float*,
                                                    float*, cudaStream_t);
template cudaError_t launch_scale_planes<double>(const Geometry&, const DevTables&, const double*, double*, bool,
                                                 cudaStream_t);
template cudaError_t launch_scale_planes<float>(const Geometry&, const DevTables&, const float*, float*, bool,
                                                cudaStream_t);
template cudaError_t launch_divergence<double>(const Geometry&, const DevTables&, const double*, const double*,
                                               const double*, double*, double, cudaStream_t);
template cudaError_t launch_divergence<float>(const Geometry&, const DevTables&, const float*, const float*,
                                              const float*, float*, double, cudaStream_t);
template cudaError_t launch_check_finite<double>(const double*, size_t, int*, cudaStream_t);
template cudaError_t launch_check_finite<float>(const float*, size_t, int*, cudaStream_t);

}  // namespace pp

// ---- FP64 FMA throughput (diagnostics) --------------------------------------------------------
// Each thread runs 8 independent chains of dependent FMAs (enough in flight per warp to fill the
// FP64 pipe); the sum is stored so that the chains are not removed.
namespace pp {
__global__ void __launch_bounds__(256) k_fp64_fma_rate(double* __restrict__ out, int iters, double a, double b) {
  double x0 = threadIdx.x * 1e-9, x1 = x0 + 1e-3, x2 = x0 + 2e-3, x3 = x0 + 3e-3;
  double x4 = x0 + 4e-3, x5 = x0 + 5e-3, x6 = x0 + 6e-3, x7 = x0 + 7e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
}
}  // namespace pp

extern "C" poisson_status poisson_fp64_fma_rate(void* scratch, size_t bytes, void* stream, double* gflops) {
  if (!scratch || !gflops) return PS_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PS_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PS_ECUDA;
  const int blocks = sms * 8, threads = 256, iters = 512;
  if (bytes < (size_t)blocks * threads * sizeof(double)) return PS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return PS_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return PS_ECUDA;
  }
  poisson_status s = PS_OK;
  float best = 0.f;
  for (int rep = 0; rep < 4 && s == PS_OK; ++rep) {   // the first launch warms up
    cudaEventRecord(e0, st);
    pp::k_fp64_fma_rate<<<blocks, threads, 0, st>>>((double*)scratch, iters, 0.9999999, 1e-7);
    cudaEventRecord(e1, st);
    float ms = 0.f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
      s = PS_ECUDA;
    else if (rep > 0 && (best == 0.f || ms < best))
      best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != PS_OK) return s;
  const double fmas = (double)blocks * threads * iters * 16.0 * 8.0;
  *gflops = 2.0 * fmas / (best * 1e-3) / 1e9;
  return PS_OK;
}
