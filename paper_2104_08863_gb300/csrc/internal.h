// Host-side plan and kernel launchers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <vector>

#include "../../include/poisson.h"
#include "fft.cuh"

namespace pp {

// Device-side table pointers for one arithmetic type T.
template <typename T> struct Tables {
  const cplx<T>* tw_m;     // e^{-2 pi i t / M}, t < M   (half-length complex FFT in x)
  const cplx<T>* tw_post;  // e^{-2 pi i k / Nx}, k <= M (real-to-complex packing)
  const cplx<T>* tw_z;     // e^{-2 pi i t / Nz}, t < Nz
  const T* a;              // wall-normal sub-diagonal a_j  (0 for j = 0)
  const T* c;              // wall-normal super-diagonal c_j (0 for j = ny-1)
  const T* inv_dy;         // 1 / dy_j
  const T* inv_h;          // 1 / h_j for interior faces j = 1..ny-1, 0 on the walls
  const T* a_lo;           // FP32 tables only: a_j - (float)a_j, so (a, a_lo) is a double-float
  const T* c_lo;           // FP32 tables only: c_j - (float)c_j
};

// Per-mode PDD factors, built once by k_tridiag_setup (layout [row][system]
// and [block][system], system = kz * (Nx/2+1) + kx).  For block rows r0..r1 of one system:
//   mult_j = a_j / beta_{j-1} (0 at r0), rb_j = 1 / beta_j, gv_j = forward-eliminated spike
//   a_{r0} e_1, kappa_j = rb_j prod_{r0<=l<j} c_l rb_l (so x~_{r0} = sum_j kappa_j g_j);
//   vF, vL, wF, wL = first/last-row values of the spikes v = A_i^-1 a e_1, w = A_i^-1 c e_m.
// FP32 plans keep only rb and gv per row (mult and kappa are recomputed in the sweep).
template <typename T> struct TriFactors {
  T *mult, *kappa, *rb, *gv;
  T *vF, *vL, *wF, *wL;
  int nsys;   // 0 when the plan has no factors of this precision
};

struct DevTables {
  Tables<double> d;
  Tables<float> f;
  const double* lamx;      // lambda_x(kx), kx = 0..M   (Eq. 9 eigenvalues)
  const double* lamz;      // lambda_z(kz), kz = 0..nz-1
  const double* dy;        // cell heights dy_j
  const double* h;         // centre distances across face j (j = 1..ny-1; h[0], h[ny] = 0)
  int* status;             // device status word
  double* acc;             // accumulators of the refined solve: [0] <f>, [1] sum_jki dy_j p_jki
  TriFactors<double> tri_d;  // FP64 plans
  TriFactors<float> tri_f;   // FP32 and FP32-refined plans
  const float* red_f;        // FP32 register-kernel plans: per-mode LU of the reduced interface system
};

struct Geometry {
  int nx, ny, nz, M, ncols, pitch;
  double dx, dz;
  int generic_fft;   // 1: use the runtime-generic FFT kernels (POISSON_GENERIC_FFT)
  int selftest_wait; // 1: the bulk-copy-staged x-transform skips its first copy (POISSON_SELFTEST_WAIT)
};

struct LaunchCount {
  int n = 0;
};

// Raise a kernel's dynamic shared-memory limit to at least `bytes`, once per kernel (a registry
// keyed by the kernel's address), so that the attribute call does not recur inside stream capture.
cudaError_t ensure_smem_limit(const void* kernel, size_t bytes);

// --- launchers (return cudaGetLastError() after the launch) --------------------------
enum FwdMode { FWD_PLAIN = 0, FWD_DIV = 1, FWD_RESID = 2, FWD_GRADT = 3 };
// INV_FINAL (FP32 spectrum, FP64 output): out = hi + (lo + v) assembled exactly in FP64,
// with hi, lo the FP32 pair that carries the refined pressure (lo may be null).
enum InvMode { INV_STORE = 0, INV_ACCUM = 1, INV_FINAL = 2 };

struct FwdArgs {
  const void* in;        // FWD_PLAIN / FWD_RESID: rhs field
  const void* u;         // FWD_DIV / FWD_GRADT: face fields
  const void* v;
  const void* w;
  const void* p;         // FWD_RESID: the FP32 pressure field the residual is formed of
  double in_scale;       // FWD_DIV: 1/dt; FWD_PLAIN: 1 (ignored for FP64 input to FP32)
  float idx2h, idx2l;    // FWD_RESID: 1/dx^2 and 1/dz^2 as double-floats
  float idz2h, idz2l;
  // FWD_RESID, later corrections: r = rin - L_h p with rin a stored residual (one FP32 pair per
  // cell) in place of (f - <f>); null for the first.  rout (may be null): the residual is also
  // stored there as an FP32 pair.
  const void* rin;
  void* rout;
};

// Pointers of the FP32 pressure pair used by INV_FINAL.
struct PairArgs {
  const float* hi;
  const float* lo;
};

template <typename T, typename TI>
cudaError_t launch_fwd_x(const Geometry& g, const DevTables& tb, const FftFactors& fm, FwdMode mode,
                         const FwdArgs& args, cplx<T>* spec, cudaStream_t st);

// accumulate: also add sum_jki dy_j out_jki (of this pass's contribution) to tb.acc[1].
template <typename T, typename TO>
cudaError_t launch_inv_x(const Geometry& g, const DevTables& tb, const FftFactors& fm, InvMode mode,
                         const cplx<T>* spec, TO* out, double scale, bool accumulate, cudaStream_t st,
                         PairArgs pair = PairArgs{nullptr, nullptr});

template <typename T>
cudaError_t launch_fft_z(const Geometry& g, const DevTables& tb, const FftFactors& fz, int sign, cplx<T>* spec,
                         cudaStream_t st);

// Specialised x-transforms for Nx/2 in {16, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024}
// (cudaErrorNotSupported otherwise).  Suffix: spectral type, field type (d = double, f = float).
cudaError_t launch_fwd_x_fast_dd(const Geometry& g, const DevTables& tb, FwdMode mode, const FwdArgs& args,
                                 cplx<double>* spec, cudaStream_t st);
cudaError_t launch_fwd_x_fast_ff(const Geometry& g, const DevTables& tb, FwdMode mode, const FwdArgs& args,
                                 cplx<float>* spec, cudaStream_t st);
cudaError_t launch_fwd_x_fast_fd(const Geometry& g, const DevTables& tb, FwdMode mode, const FwdArgs& args,
                                 cplx<float>* spec, cudaStream_t st);
cudaError_t launch_inv_x_fast_dd(const Geometry& g, const DevTables& tb, InvMode mode, const cplx<double>* spec,
                                 double* out, double scale, bool accumulate, cudaStream_t st, PairArgs pair);
cudaError_t launch_inv_x_fast_ff(const Geometry& g, const DevTables& tb, InvMode mode, const cplx<float>* spec,
                                 float* out, double scale, bool accumulate, cudaStream_t st, PairArgs pair);
cudaError_t launch_inv_x_fast_fd(const Geometry& g, const DevTables& tb, InvMode mode, const cplx<float>* spec,
                                 double* out, double scale, bool accumulate, cudaStream_t st, PairArgs pair);

// Specialised z-transform for Nz in {16, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024};
// returns cudaErrorNotSupported for other lengths.  [kx_lo, kx_hi): the kx columns transformed
// (kx_hi < 0: all; kx_lo a multiple of fft_z_fast_tile).
template <typename T>
cudaError_t launch_fft_z_fast(const Geometry& g, const Tables<T>& tt, int sign, cplx<T>* spec, cudaStream_t st,
                              int kx_lo = 0, int kx_hi = -1);
template <typename T>
int fft_z_fast_tile(const Geometry& g);

template <typename TD, typename TC>
cudaError_t launch_tridiag(const Geometry& g, const DevTables& tb, int parts, int low_modes, bool low_list,
                           cplx<TD>* spec, cudaStream_t st);

template <>
cudaError_t launch_tridiag<double, double>(const Geometry& g, const DevTables& tb, int parts, int low_modes,
                                           bool low_list, cplx<double>* spec, cudaStream_t st);
template <>
cudaError_t launch_tridiag<float, float>(const Geometry& g, const DevTables& tb, int parts, int low_modes,
                                         bool low_list, cplx<float>* spec, cudaStream_t st);

// PDD with the precomputed factors tb.tri_d / tb.tri_f (setup once per plan, then per solve).
cudaError_t launch_tridiag_setup(const Geometry& g, const DevTables& tb, int parts, cudaStream_t st);
// trunc: the truncated reduced system of Sec. 2.2 (framed coupling entries dropped).
cudaError_t launch_tridiag_factored(const Geometry& g, const DevTables& tb, int parts, bool trunc, cplx<double>* spec,
                                    cudaStream_t st);
cudaError_t launch_tridiag_factored_f32(const Geometry& g, const DevTables& tb, int parts, int low_modes, bool trunc,
                                        cplx<float>* spec, cudaStream_t st);

// FP32 PDD with each block of m = ny/P rows held in one thread's registers and its factors
// computed on the fly (no factor tables): m in {1, 2, 3, 4, 6, 8, 12, 16, 24}, P <= 256, S = 256/P
// systems per CTA (at least 1).  Other (ny, P) use the factored kernel with tables.
__host__ __device__ inline bool reg_tridiag_ok(int ny, int P) {
  if (P < 1 || P > 256 || ny % P) return false;
  const int m = ny / P;
  return m == 1 || m == 2 || m == 3 || m == 4 || m == 6 || m == 8 || m == 12 || m == 16 || m == 24;
}
__host__ __device__ inline int reg_systems_per_cta(int P) { return P >= 256 ? 1 : 256 / P; }
// [kx_lo, kx_hi): the kx columns solved (kx_hi < 0: all); a partial range is supported by the
// warp-scan variant only (P a power of two <= 32), with kx_lo a multiple of
// reg_systems_per_cta(P), and is refused (cudaErrorNotSupported) otherwise.
cudaError_t launch_tridiag_reg_f32(const Geometry& g, const DevTables& tb, int parts, int low_modes,
                                   cplx<float>* spec, cudaStream_t st, int kx_lo = 0, int kx_hi = -1);
__host__ __device__ inline bool scan_tridiag_ok(int ny, int P) { return reg_tridiag_ok(ny, P) && P <= 32 && (P & (P - 1)) == 0; }
// Bytes of the reduced-system table of the register kernel, and its FP64 set-up (once per plan).
size_t reduced_table_bytes(const Geometry& g, int parts);
cudaError_t launch_reduced_setup(const Geometry& g, const DevTables& tb, int parts, bool trunc, float* tab,
                                 cudaStream_t st);

// FP64 re-solve of the low-mode list on FP32 spectral data (intermediates in FP64 scratch).
cudaError_t launch_tridiag_low64(const Geometry& g, const DevTables& tb, int parts, int low_modes,
                                 cplx<float>* spec, cplx<double>* scratch, cudaStream_t st);

// Gauge modes of the (0, 0) solve: plain zero weighted mean; GAUGE_STORE_MEAN also stores the
// rhs mean <f> in tb.acc[0]; GAUGE_OFFSET shifts the result so that the running pressure
// total (weighted sum tb.acc[1]) plus this correction has zero weighted mean.
enum GaugeMode { GAUGE_ZERO = 0, GAUGE_STORE_MEAN = 1, GAUGE_OFFSET = 2 };
template <typename TD>
cudaError_t launch_mode00(const Geometry& g, const DevTables& tb, GaugeMode gauge, cplx<TD>* spec,
                          cudaStream_t st);

template <typename T>
cudaError_t launch_gradient(const Geometry& g, const DevTables& tb, const T* p, T* u, T* v, T* w, double dt,
                            cudaStream_t st, int jlo = 0, int jhi = -1);   // rows [jlo, jhi) (+ the top wall faces)

template <typename T>
cudaError_t launch_adjoint_epilogue(const Geometry& g, const DevTables& tb, const T* q, T* gu, T* gv, T* gw,
                                    cudaStream_t st);

// out = in * (1/dy_j) or in * dy_j per y-plane j (in == out allowed), and q = dy_j (hi + lo) in FP64.
template <typename T>
cudaError_t launch_scale_planes(const Geometry& g, const DevTables& tb, const T* in, T* out, bool to_weighted,
                                cudaStream_t st);
cudaError_t launch_weighted_pair(const Geometry& g, const DevTables& tb, const float* hi, const float* lo, double* q,
                                 cudaStream_t st);

template <typename T>
cudaError_t launch_check_finite(const T* x, size_t n, int* status, cudaStream_t st);

// f = D(u)/dt (Eq. 7) as a cell field, in T arithmetic.
template <typename T>
cudaError_t launch_divergence(const Geometry& g, const DevTables& tb, const T* u, const T* v, const T* w, T* f,
                              double dt, cudaStream_t st);

// One stage of Heun's RK2 momentum predictor (csrc/k_momentum.cu):
//   out = alpha * base + beta * s + bdt * R(s),  R = -div(s s) + nu lap(s) + (fx, 0, 0).
// base may be null (alpha = 0); out may alias base but not s.
template <typename T> struct MomArgs {
  const T *su, *sv, *sw;
  const T *bu, *bv, *bw;
  T *ou, *ov, *ow;
  double alpha, beta, bdt, nu, fx;
};
// Rows [jlo, jhi) of the cell fields and the v faces jlo .. jhi-1 (plus the wall faces 0 and ny
// when the range touches them); jhi < 0: up to ny.  A range reads the rows jlo-1 .. jhi.
template <typename T>
cudaError_t launch_momentum(const Geometry& g, const DevTables& tb, const MomArgs<T>& a, cudaStream_t st,
                            int jlo = 0, int jhi = -1);

// The FP64-accurate timestep on FP32 units (csrc/k_refined_ts.cu): the state as FP32 pairs
// (hi, lo) in the FP64 buffers, double-float momentum stages, divergence and gradient.
struct MomArgsDF {
  const float2 *su, *sv, *sw;
  const float2 *bu, *bv, *bw;
  float2 *ou, *ov, *ow;
  double alpha, beta, bdt, nu, fx;
};
cudaError_t launch_to_pairs(double* x, size_t n, cudaStream_t st);
cudaError_t launch_from_pairs(double* x, size_t n, cudaStream_t st);
cudaError_t launch_momentum_df(const Geometry& g, const DevTables& tb, const MomArgsDF& a, cudaStream_t st);
cudaError_t launch_divergence_df(const Geometry& g, const DevTables& tb, const float2* u, const float2* v,
                                 const float2* w, double dt, double* f, cudaStream_t st);
// u = u* - dt G p with p = hi + lo (the refined solve's FP32 pair); p_out (may be null) receives
// p in FP64.
cudaError_t launch_gradient_pairs(const Geometry& g, const DevTables& tb, const float* hi, const float* lo, double* u,
                                  double* v, double* w, double* p_out, double dt, cudaStream_t st);

// Row chunks of the host-buffer timestep's input copies (projection_timestep_host).
constexpr int HOST_CHUNKS = 8;

}  // namespace pp

// Host plan (opaque to callers of include/poisson.h).
struct poisson_plan_s {
  pp::Geometry g;
  double lx, lz;
  int precision, tridiag, parts, low, refine;
  unsigned flags;
  pp::FftFactors fm, fz;
  std::vector<double> faces, dy, h, a, c, lamx, lamz;
  std::vector<unsigned char> host_tables;   // staging image of the device tables
  // workspace layout (byte offsets)
  size_t off_spec, off_pbuf, off_pbuf2, off_r1, off_scratch, off_tables, off_status, off_acc, off_tri, off_red,
      ws_bytes;
  bool has_tri;   // per-mode PDD factor tables in the workspace (FP64 plans; FP32 plans with m = ny/P outside the register kernel's set)
  size_t tab_offsets[32];
  unsigned char* ws;
  pp::DevTables dt;
  int launches;
  // kx-slab chain of the FP32 spectral middle (poisson_plan_set_chain): slab width in columns
  // (0: one pass over the whole spectrum), streams (1 or 2), the second stream and its events
  int slab_cols = 0;
  int chain_streams = 1;
  cudaStream_t chain_st = nullptr;
  cudaEvent_t chain_ev[2] = {nullptr, nullptr};
  // host-buffer timestep: the stream of its copies and per row chunk the events of the input
  // copies, the pressure and the corrected velocity (+ a start event)
  cudaStream_t copy_st = nullptr;
  cudaEvent_t copy_ev[3 * pp::HOST_CHUNKS + 1] = {};
  // POISSON_TIMING: one event pair around every launch of the last call
  std::vector<cudaEvent_t> ev;
  std::vector<const char*> ev_names;
  int nev;
  // batched plans (poisson_plan_batched): sub-plans, fork streams and the cached graph
  std::vector<poisson_plan_s*> children;
  std::vector<cudaStream_t> forks;
  std::vector<cudaEvent_t> fork_ev;
  cudaGraphExec_t gexec = nullptr;
  std::vector<const void*> g_rhs;
  std::vector<void*> g_p;
  bool warmed = false;
  // persistent batched launch (batch_persistent.cu): on when POISSON_BATCH_PERSISTENT is set and
  // every instance is supported; byte offsets of its regions after the instances' workspaces
  bool persistent = false;
  bool selftest = false;
  size_t off_bstatus = 0, off_inst = 0, off_items = 0, off_ctl = 0, ctl_bytes = 0, off_lowscr = 0;
  int nitems = 0;
  std::vector<unsigned char> inst_host;   // host image of the instance table
};

namespace pp {
// Table pointers of a plan inside a workspace that starts at `base`.
DevTables bind_tables(const poisson_plan_s* pl, unsigned char* base);
// poisson_solve's pipeline on an explicit workspace (no timing events).
poisson_status solve_on_workspace(poisson_plan_s* pl, unsigned char* ws, const DevTables& dt, const void* rhs,
                                  void* p, cudaStream_t st);
// Batched plans (csrc/batch.cu).
poisson_status set_batch_workspace(poisson_plan_s* pl, unsigned char* ws, void* stream);
void destroy_batch(poisson_plan_s* pl);
}  // namespace pp
