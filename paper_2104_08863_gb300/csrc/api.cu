// Host planner and C ABI of the pressure-Poisson library (include/poisson.h).
//
// poisson_plan_create validates the descriptor and computes, in FP64 on the host: the
// stretched-grid metrics (Sec. 2; cell heights dy_j, centre distances h_j, the wall-normal
// coefficients a_j = 1/(dy_j h_j), c_j = 1/(dy_j h_{j+1})), the modified wavenumbers of
// Eq. 9 (lambda = -(4/d^2) sin^2(pi k / N)), the FFT factorisations and twiddles.  The solve
// entry points run the pipeline of Sec. 3.2 steps (1)-(8) as a sequence of kernels on the
// caller's stream.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "internal.h"

using namespace pp;

// struct poisson_plan_s is defined in internal.h (shared with the static-workspace entry point).

namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

bool factor(int L, FftFactors& f) {
  f.L = L;
  f.nst = 0;
  int r = L;
  while (r % 8 == 0 && r > 4) { f.rad[f.nst++] = 8; r /= 8; }
  while (r % 4 == 0) { f.rad[f.nst++] = 4; r /= 4; }
  while (r % 2 == 0) { f.rad[f.nst++] = 2; r /= 2; }
  while (r % 3 == 0) { f.rad[f.nst++] = 3; r /= 3; }
  if (f.nst > 12) return false;
  if (r != 1) return false;
  if (f.nst == 0) { f.rad[f.nst++] = 1; }  // L == 1 is rejected by validation
  return true;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Automatic PDD partition.  FP64 (factored kernel, FP64-issue bound): the most blocks with at
// least 48 rows each.  FP32 (register kernel): blocks of the largest supported height <= 24.
int auto_parts(int ny, int precision) {
  if (precision != PP_FP64) {
    for (int P = 1; P <= 256; ++P)
      if (ny % P == 0 && ny / P <= 24 && pp::reg_tridiag_ok(ny, P)) return P;
  }
  int best = 1;
  for (int P = 2; P <= 32; ++P)
    if (ny % P == 0 && ny / P >= 48) best = P;
  return best;
}

template <typename T>
void put_cplx_table(std::vector<unsigned char>& img, size_t off, const std::vector<double>& re,
                    const std::vector<double>& im) {
  T* p = reinterpret_cast<T*>(img.data() + off);
  for (size_t i = 0; i < re.size(); ++i) { p[2 * i] = (T)re[i]; p[2 * i + 1] = (T)im[i]; }
}
template <typename T>
void put_real_table(std::vector<unsigned char>& img, size_t off, const std::vector<double>& v) {
  T* p = reinterpret_cast<T*>(img.data() + off);
  for (size_t i = 0; i < v.size(); ++i) p[i] = (T)v[i];
}

bool spec_is_fp64(const poisson_plan_s* pl) { return pl->precision == PP_FP64; }

}  // namespace

namespace pp {
cudaError_t ensure_smem_limit(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::unordered_map<const void*, size_t> granted;
  if (bytes <= 48 * 1024) return cudaSuccess;
  std::lock_guard<std::mutex> lock(mu);
  auto it = granted.find(kernel);
  if (it != granted.end() && it->second >= bytes) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) granted[kernel] = bytes;
  return e;
}

DevTables bind_tables(const poisson_plan_s* pl, unsigned char* base) {
  DevTables dt;
  unsigned char* tb = base + pl->off_tables;
  const size_t* to = pl->tab_offsets;
  dt.d.tw_m = (const cplx<double>*)(tb + to[0]);
  dt.d.tw_post = (const cplx<double>*)(tb + to[1]);
  dt.d.tw_z = (const cplx<double>*)(tb + to[2]);
  dt.d.a = (const double*)(tb + to[3]);
  dt.d.c = (const double*)(tb + to[4]);
  dt.f.tw_m = (const cplx<float>*)(tb + to[5]);
  dt.f.tw_post = (const cplx<float>*)(tb + to[6]);
  dt.f.tw_z = (const cplx<float>*)(tb + to[7]);
  dt.f.a = (const float*)(tb + to[8]);
  dt.f.c = (const float*)(tb + to[9]);
  dt.lamx = (const double*)(tb + to[10]);
  dt.lamz = (const double*)(tb + to[11]);
  dt.dy = (const double*)(tb + to[12]);
  dt.h = (const double*)(tb + to[13]);
  dt.d.inv_dy = (const double*)(tb + to[14]);
  dt.d.inv_h = (const double*)(tb + to[15]);
  dt.f.inv_dy = (const float*)(tb + to[16]);
  dt.f.inv_h = (const float*)(tb + to[17]);
  dt.f.a_lo = (const float*)(tb + to[18]);
  dt.f.c_lo = (const float*)(tb + to[19]);
  dt.d.a_lo = nullptr;
  dt.d.c_lo = nullptr;
  dt.red_f = pl->has_tri ? nullptr : (const float*)(base + pl->off_red);
  dt.status = (int*)(base + pl->off_status);
  dt.acc = (double*)(base + pl->off_acc);
  dt.tri_d = TriFactors<double>{};
  dt.tri_f = TriFactors<float>{};
  {
    const size_t nsys = (size_t)pl->g.nz * pl->g.ncols;
    const size_t rows = nsys * pl->g.ny, blks = nsys * pl->parts;
    if (pl->precision == PP_FP64) {
      double* t = (double*)(base + pl->off_tri);
      TriFactors<double>& f = dt.tri_d;
      f.mult = t; f.kappa = t + rows; f.rb = t + 2 * rows; f.gv = t + 3 * rows;
      f.vF = t + 4 * rows; f.vL = f.vF + blks; f.wF = f.vL + blks; f.wL = f.wF + blks;
      f.nsys = (int)nsys;
    } else if (pl->has_tri) {
      float* t = (float*)(base + pl->off_tri);
      TriFactors<float>& f = dt.tri_f;
      f.mult = nullptr; f.kappa = nullptr; f.rb = t; f.gv = t + rows;
      f.vF = t + 2 * rows; f.vL = f.vF + blks; f.wF = f.vL + blks; f.wL = f.wF + blks;
      f.nsys = (int)nsys;
    }
  }
  return dt;
}
}  // namespace pp

extern "C" {

const char* poisson_status_string(poisson_status s) {
  switch (s) {
    case PS_OK: return "ok";
    case PS_EINVAL: return "invalid argument";
    case PS_EUNSUPPORTED: return "unsupported size or option";
    case PS_ENOMEM: return "host allocation failed";
    case PS_ECUDA: return "CUDA error";
    case PS_ETIMEOUT: return "device wait timed out";
    case PS_ENONFINITE: return "non-finite input";
    case PS_ENOWORKSPACE: return "workspace not set";
  }
  return "unknown status";
}

poisson_status poisson_plan_create(const poisson_desc* d, poisson_plan_t* out) {
  if (!d || !out) return PS_EINVAL;
  *out = nullptr;
  if (d->nx < 4 || d->ny < 2 || d->nz < 2 || (d->nx & 1)) return PS_EINVAL;
  if (!(d->lx > 0.0) || !(d->lz > 0.0) || !d->y_faces) return PS_EINVAL;
  if (d->precision < PP_FP64 || d->precision > PP_FP32_REFINED) return PS_EINVAL;
  if (d->tridiag < PT_AUTO || d->tridiag > PT_PDD_TRUNCATED) return PS_EINVAL;
  if ((long long)d->nx * d->ny * d->nz > (1LL << 34)) return PS_EUNSUPPORTED;
  if (d->ny > 8192) return PS_EUNSUPPORTED;
  if ((long long)(d->ny + 1) * d->nz >= (1LL << 31)) return PS_EUNSUPPORTED;   // line counts are int
  for (int j = 0; j <= d->ny; ++j)
    if (!isfinite(d->y_faces[j]) || (j > 0 && !(d->y_faces[j] > d->y_faces[j - 1]))) return PS_EINVAL;
  poisson_plan_s* pl = new (std::nothrow) poisson_plan_s();
  if (!pl) return PS_ENOMEM;
  Geometry& g = pl->g;
  g.nx = d->nx; g.ny = d->ny; g.nz = d->nz;
  g.M = d->nx / 2;
  g.ncols = g.M + 1;
  const int cpad = d->precision == PP_FP64 ? 4 : 8;   // 64-byte aligned spectral rows
  g.pitch = (g.ncols + cpad - 1) / cpad * cpad;
  g.dx = d->lx / d->nx;
  g.dz = d->lz / d->nz;
  g.generic_fft = (d->flags & POISSON_GENERIC_FFT) ? 1 : 0;
  g.selftest_wait = (d->flags & POISSON_SELFTEST_WAIT) ? 1 : 0;
  pl->lx = d->lx; pl->lz = d->lz;
  pl->precision = d->precision;
  pl->tridiag = d->tridiag;
  pl->flags = d->flags;
  if (!factor(g.M, pl->fm) || !factor(g.nz, pl->fz) || g.M < 2) { delete pl; return PS_EUNSUPPORTED; }
  int P = 1;
  if (d->tridiag == PT_THOMAS) P = 1;
  else if (d->pdd_parts > 0) P = d->pdd_parts;
  else P = auto_parts(g.ny, d->precision);
  if (g.ny % P != 0 || (P > 32 && !(d->precision != PP_FP64 && pp::reg_tridiag_ok(g.ny, P)))) {
    delete pl;
    return PS_EUNSUPPORTED;
  }
  pl->parts = P;
  int L = -1;
  if (d->precision != PP_FP64) {
    L = d->fp64_low_modes < 0 ? 0 : d->fp64_low_modes;
    if (L > g.M) L = g.M;
    if (2 * L + 1 > g.nz) L = (g.nz - 1) / 2;
  }
  pl->low = L;
  pl->refine = d->precision == PP_FP32_REFINED ? (d->refine_steps > 0 ? d->refine_steps : 1) : 0;

  // --- grid metrics (FP64) ---
  const int ny = g.ny;
  pl->faces.assign(d->y_faces, d->y_faces + ny + 1);
  pl->dy.resize(ny);
  std::vector<double> yc(ny);
  for (int j = 0; j < ny; ++j) {
    pl->dy[j] = pl->faces[j + 1] - pl->faces[j];
    yc[j] = 0.5 * (pl->faces[j] + pl->faces[j + 1]);
  }
  pl->h.assign(ny + 1, 0.0);
  for (int j = 1; j < ny; ++j) pl->h[j] = yc[j] - yc[j - 1];
  pl->a.assign(ny, 0.0);
  pl->c.assign(ny, 0.0);
  for (int j = 1; j < ny; ++j) pl->a[j] = 1.0 / (pl->dy[j] * pl->h[j]);
  for (int j = 0; j < ny - 1; ++j) pl->c[j] = 1.0 / (pl->dy[j] * pl->h[j + 1]);
  pl->lamx.resize(g.ncols);
  for (int k = 0; k < g.ncols; ++k) {
    const double s = sin(M_PI * k / g.nx);
    pl->lamx[k] = -(4.0 / (g.dx * g.dx)) * s * s;
  }
  pl->lamz.resize(g.nz);
  for (int k = 0; k < g.nz; ++k) {
    const double s = sin(M_PI * k / g.nz);
    pl->lamz[k] = -(4.0 / (g.dz * g.dz)) * s * s;
  }
  // --- twiddles (FP64 trig, index-reduced angles) ---
  auto twid = [](int L, int n, std::vector<double>& re, std::vector<double>& im) {
    re.resize(n); im.resize(n);
    for (int t = 0; t < n; ++t) {
      const double ang = -2.0 * M_PI * (double)t / (double)L;
      re[t] = cos(ang); im[t] = sin(ang);
    }
  };
  std::vector<double> twm_r, twm_i, twp_r, twp_i, twz_r, twz_i;
  twid(g.M, g.M, twm_r, twm_i);
  twid(g.nx, g.M + 1, twp_r, twp_i);
  twid(g.nz, g.nz, twz_r, twz_i);

  // --- table image: double tables then float tables ---
  size_t off = 0;
  size_t* to = pl->tab_offsets;
  auto slot = [&](int id, size_t bytes) { to[id] = off; off = align_up(off + bytes, 256); };
  slot(0, 16 * (size_t)g.M);  slot(1, 16 * (size_t)(g.M + 1)); slot(2, 16 * (size_t)g.nz);
  slot(3, 8 * (size_t)ny);    slot(4, 8 * (size_t)ny);
  slot(5, 8 * (size_t)g.M);   slot(6, 8 * (size_t)(g.M + 1)); slot(7, 8 * (size_t)g.nz);
  slot(8, 4 * (size_t)ny);    slot(9, 4 * (size_t)ny);
  slot(10, 8 * (size_t)g.ncols); slot(11, 8 * (size_t)g.nz);
  slot(12, 8 * (size_t)ny);   slot(13, 8 * (size_t)(ny + 1));
  slot(14, 8 * (size_t)ny);   slot(15, 8 * (size_t)(ny + 1));
  slot(16, 4 * (size_t)ny);   slot(17, 4 * (size_t)(ny + 1));
  slot(18, 4 * (size_t)ny);   slot(19, 4 * (size_t)ny);
  const size_t tab_bytes = off;
  pl->host_tables.assign(tab_bytes, 0);
  auto& img = pl->host_tables;
  put_cplx_table<double>(img, to[0], twm_r, twm_i);
  put_cplx_table<double>(img, to[1], twp_r, twp_i);
  put_cplx_table<double>(img, to[2], twz_r, twz_i);
  put_real_table<double>(img, to[3], pl->a);
  put_real_table<double>(img, to[4], pl->c);
  put_cplx_table<float>(img, to[5], twm_r, twm_i);
  put_cplx_table<float>(img, to[6], twp_r, twp_i);
  put_cplx_table<float>(img, to[7], twz_r, twz_i);
  put_real_table<float>(img, to[8], pl->a);
  put_real_table<float>(img, to[9], pl->c);
  put_real_table<double>(img, to[10], pl->lamx);
  put_real_table<double>(img, to[11], pl->lamz);
  put_real_table<double>(img, to[12], pl->dy);
  put_real_table<double>(img, to[13], pl->h);
  std::vector<double> inv_dy(ny), inv_h(ny + 1, 0.0);
  for (int j = 0; j < ny; ++j) inv_dy[j] = 1.0 / pl->dy[j];
  for (int j = 1; j < ny; ++j) inv_h[j] = 1.0 / pl->h[j];
  put_real_table<double>(img, to[14], inv_dy);
  put_real_table<double>(img, to[15], inv_h);
  put_real_table<float>(img, to[16], inv_dy);
  put_real_table<float>(img, to[17], inv_h);
  {   // low parts of the double-float coefficients (a, c) used by the refinement residual
    std::vector<double> alo(ny), clo(ny);
    for (int j = 0; j < ny; ++j) {
      alo[j] = pl->a[j] - (double)(float)pl->a[j];
      clo[j] = pl->c[j] - (double)(float)pl->c[j];
    }
    put_real_table<float>(img, to[18], alo);
    put_real_table<float>(img, to[19], clo);
  }

  // --- workspace layout ---
  const size_t csz = spec_is_fp64(pl) ? 16 : 8;
  const size_t rsz = spec_is_fp64(pl) ? 8 : 4;
  off = 0;
  pl->off_spec = off;  off = align_up(off + csz * (size_t)ny * g.nz * g.pitch, 256);
  pl->off_pbuf = off;  off = align_up(off + rsz * (size_t)ny * g.nz * g.nx, 256);
  pl->off_pbuf2 = off;   // low FP32 part of the refined pressure
  if (d->precision == PP_FP32_REFINED) off = align_up(off + 4 * (size_t)ny * g.nz * g.nx, 256);
  pl->off_r1 = off;      // the first correction's residual (FP32 pair per cell) for the later ones
  if (pl->refine >= 2) off = align_up(off + 8 * (size_t)ny * g.nz * g.nx, 256);
  pl->off_scratch = off;
  if (L >= 0) off = align_up(off + 16 * (size_t)ny * (L + 1) * (2 * L + 1), 256);
  pl->off_tables = off; off = align_up(off + tab_bytes, 256);
  pl->off_status = off; off = align_up(off + 256, 256);
  pl->off_acc = off;    off = align_up(off + 256, 256);
  {   // per-mode PDD factors: FP64 plans 4 per row + 4 per block; FP32 plans 2 per row + 4 per block
    const size_t nsys = (size_t)g.nz * g.ncols;
    pl->off_tri = off;
    // FP32 plans whose blocks fit in registers build their factors on the fly (no tables)
    pl->has_tri = d->precision == PP_FP64 || !pp::reg_tridiag_ok(ny, P);
    if (d->precision == PP_FP64) off = align_up(off + 8 * nsys * (4 * (size_t)ny + 4 * (size_t)P), 256);
    else if (pl->has_tri) off = align_up(off + 4 * nsys * (2 * (size_t)ny + 4 * (size_t)P), 256);
    pl->off_red = off;
    if (!pl->has_tri) off = align_up(off + pp::reduced_table_bytes(g, P), 256);
  }
  pl->ws_bytes = off;
  pl->ws = nullptr;
  pl->launches = 0;
  pl->nev = 0;
  pl->nev = 0;
  *out = pl;
  return PS_OK;
}

poisson_status poisson_workspace_size(poisson_plan_t pl, size_t* bytes) {
  if (!pl || !bytes) return PS_EINVAL;
  *bytes = pl->ws_bytes;   // batched plans: the sum of their sub-plans' aligned workspaces
  return PS_OK;
}

poisson_status poisson_set_workspace(poisson_plan_t pl, void* ws, size_t bytes, void* stream) {
  if (!pl || !ws) return PS_EINVAL;
  if (bytes < pl->ws_bytes || ((uintptr_t)ws & 255u)) return PS_EINVAL;
  if (!pl->children.empty()) return pp::set_batch_workspace(pl, (unsigned char*)ws, stream);
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* base = (unsigned char*)ws;
  cudaError_t e = cudaMemcpyAsync(base + pl->off_tables, pl->host_tables.data(), pl->host_tables.size(),
                                  cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return PS_ECUDA;
  e = cudaMemsetAsync(base + pl->off_status, 0, 256, st);
  if (e != cudaSuccess) return PS_ECUDA;
  // The host image must outlive the copy; synchronise once here (set-up, not the hot path).
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return PS_ECUDA;
  pl->ws = base;
  pl->dt = pp::bind_tables(pl, base);
  if (!pl->has_tri && pl->parts > 1) {
    if (launch_reduced_setup(pl->g, pl->dt, pl->parts, pl->tridiag == PT_PDD_TRUNCATED, (float*)(base + pl->off_red),
                             st) != cudaSuccess)
      return PS_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return PS_ECUDA;
  }
  if (pl->has_tri) {
    if (launch_tridiag_setup(pl->g, pl->dt, pl->parts, st) != cudaSuccess) return PS_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return PS_ECUDA;
  }
  return PS_OK;
}

}  // extern "C"

namespace {

// Execution context of one call: the plan, the workspace it runs on and its table pointers.
struct Exec {
  poisson_plan_s* pl;
  unsigned char* ws;
  DevTables dt;
  cudaStream_t st;
  bool timing;
};

bool timer_begin(Exec& ex) {
  poisson_plan_s* pl = ex.pl;
  if (!ex.timing || pl->nev >= 64) return false;
  while ((int)pl->ev.size() < 2 * (pl->nev + 1)) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return false;
    pl->ev.push_back(e);
  }
  return cudaEventRecord(pl->ev[2 * pl->nev], ex.st) == cudaSuccess;
}

void timer_end(Exec& ex, const char* name) {
  poisson_plan_s* pl = ex.pl;
  cudaEventRecord(pl->ev[2 * pl->nev + 1], ex.st);
  if ((int)pl->ev_names.size() <= pl->nev) pl->ev_names.resize(pl->nev + 1);
  pl->ev_names[pl->nev] = name;
  ++pl->nev;
}

#define PP_TRY_N(name, expr)                              \
  do {                                                    \
    const bool _t = timer_begin(ex);                      \
    cudaError_t _e = (expr);                              \
    if (_t) timer_end(ex, name);                          \
    ++ex.pl->launches;                                    \
    if (_e != cudaSuccess) return PS_ECUDA;               \
  } while (0)

#define PP_RET(expr)                     \
  do {                                   \
    poisson_status _s = (expr);          \
    if (_s != PS_OK) return _s;          \
  } while (0)

// A launch inside a region that is timed as a whole (no event pair of its own).
#define PP_TRY_Q(expr)                                    \
  do {                                                    \
    cudaError_t _e = (expr);                              \
    ++ex.pl->launches;                                    \
    if (_e != cudaSuccess) return PS_ECUDA;               \
  } while (0)

// Spectral middle of a solve on the x-transformed spectral buffer (Sec. 3.2 steps (4)-(6)):
// forward z-transform, wall-normal systems, the (0, 0) mode, inverse z-transform.
template <typename T>
poisson_status spectral_mid(Exec& ex, cplx<T>* spec, GaugeMode gauge);

template <>
poisson_status spectral_mid<double>(Exec& ex, cplx<double>* spec, GaugeMode gauge) {
  const poisson_plan_s* pl = ex.pl;
  const Geometry& g = pl->g;
  cudaStream_t st = ex.st;
  PP_TRY_N("fft_z_fwd", launch_fft_z<double>(g, ex.dt, pl->fz, -1, spec, st));
  PP_TRY_N("tridiag_pdd", launch_tridiag_factored(g, ex.dt, pl->parts, pl->tridiag == PT_PDD_TRUNCATED, spec, st));
  PP_TRY_N("mode00", launch_mode00<double>(g, ex.dt, gauge, spec, st));
  PP_TRY_N("fft_z_inv", launch_fft_z<double>(g, ex.dt, pl->fz, +1, spec, st));
  return PS_OK;
}

// The FP32 spectral middle in kx slabs (poisson_plan_set_chain): for each slab of slab_cols
// columns the forward z-transform, the wall-normal solves and the inverse z-transform run back
// to back, so the slab (ny nz slab_cols complex values) is still in L2 when the next pass reads
// it and the spectrum crosses HBM once in each direction for the three passes.  Slabs are
// independent (disjoint columns); with two streams, odd slabs run on the plan's second stream
// (forked from and joined back into the caller's stream by events), which fills the tail of one
// slab's launch with the next slab's work.  The low modes and the (0, 0) mode lie in slab 0.
poisson_status spectral_chain_f32(Exec& ex, cplx<float>* spec, GaugeMode gauge) {
  const poisson_plan_s* pl = ex.pl;
  const Geometry& g = pl->g;
  cudaStream_t st = ex.st;
  const int sw = pl->slab_cols;
  const bool two = pl->chain_streams > 1 && pl->chain_st != nullptr;
  cplx<double>* scr = (cplx<double>*)(ex.ws + pl->off_scratch);
  const bool timed = timer_begin(ex);
  if (two) {
    if (cudaEventRecord(pl->chain_ev[0], st) != cudaSuccess) return PS_ECUDA;
    if (cudaStreamWaitEvent(pl->chain_st, pl->chain_ev[0], 0) != cudaSuccess) return PS_ECUDA;
  }
  for (int k = 0, lo = 0; lo < g.ncols; ++k, lo += sw) {
    const int hi = lo + sw < g.ncols ? lo + sw : g.ncols;
    cudaStream_t s = (two && (k & 1)) ? pl->chain_st : st;
    PP_TRY_Q(launch_fft_z_fast<float>(g, ex.dt.f, -1, spec, s, lo, hi));
    PP_TRY_Q(launch_tridiag_reg_f32(g, ex.dt, pl->parts, pl->low, spec, s, lo, hi));
    if (lo == 0) {
      if (pl->low >= 0) PP_TRY_Q(launch_tridiag_low64(g, ex.dt, pl->parts, pl->low, spec, scr, s));
      PP_TRY_Q(launch_mode00<float>(g, ex.dt, gauge, spec, s));
    }
    PP_TRY_Q(launch_fft_z_fast<float>(g, ex.dt.f, +1, spec, s, lo, hi));
  }
  if (two) {
    if (cudaEventRecord(pl->chain_ev[1], pl->chain_st) != cudaSuccess) return PS_ECUDA;
    if (cudaStreamWaitEvent(st, pl->chain_ev[1], 0) != cudaSuccess) return PS_ECUDA;
  }
  if (timed) timer_end(ex, "z_pdd_z_chain");
  return PS_OK;
}

template <>
poisson_status spectral_mid<float>(Exec& ex, cplx<float>* spec, GaugeMode gauge) {
  const poisson_plan_s* pl = ex.pl;
  const Geometry& g = pl->g;
  cudaStream_t st = ex.st;
  if (pl->slab_cols > 0) return spectral_chain_f32(ex, spec, gauge);
  PP_TRY_N("fft_z_fwd", launch_fft_z<float>(g, ex.dt, pl->fz, -1, spec, st));
  if (pl->has_tri)
    PP_TRY_N("tridiag_pdd", launch_tridiag_factored_f32(g, ex.dt, pl->parts, pl->low, pl->tridiag == PT_PDD_TRUNCATED,
                                                        spec, st));
  else PP_TRY_N("tridiag_pdd", launch_tridiag_reg_f32(g, ex.dt, pl->parts, pl->low, spec, st));
  if (pl->low >= 0) {
    cplx<double>* scr = (cplx<double>*)(ex.ws + pl->off_scratch);
    PP_TRY_N("tridiag_low64", launch_tridiag_low64(g, ex.dt, pl->parts, pl->low, spec, scr, st));
  }
  PP_TRY_N("mode00", launch_mode00<float>(g, ex.dt, gauge, spec, st));
  PP_TRY_N("fft_z_inv", launch_fft_z<float>(g, ex.dt, pl->fz, +1, spec, st));
  return PS_OK;
}

// Forward x-transform of the right-hand side of `mode`, then the spectral middle (which ends
// with the inverse z-transform).
template <typename T, typename TI>
poisson_status forward_and_core(Exec& ex, FwdMode mode, const FwdArgs& args, GaugeMode gauge) {
  cplx<T>* spec = (cplx<T>*)(ex.ws + ex.pl->off_spec);
  cudaStream_t st = ex.st;
  static const char* const fwd_names[] = {"fwd_x", "fwd_x_div", "fwd_x_resid", "fwd_x_gradt"};
  PP_TRY_N(fwd_names[mode], (launch_fwd_x<T, TI>(ex.pl->g, ex.dt, ex.pl->fm, mode, args, spec, st)));
  return spectral_mid<T>(ex, spec, gauge);
}

// Inverse x-transform of the spectral buffer (already inverse z-transformed) into `out` with
// the epilogue `mode`.
template <typename T, typename TO>
poisson_status inverse_x(Exec& ex, InvMode mode, TO* out, bool accumulate, PairArgs pair = PairArgs{nullptr, nullptr}) {
  cplx<T>* spec = (cplx<T>*)(ex.ws + ex.pl->off_spec);
  const double scale = 1.0 / ((double)ex.pl->g.nx * (double)ex.pl->g.nz);
  cudaStream_t st = ex.st;
  static const char* const inv_names[] = {"inv_x", "inv_x_accum", "inv_x_final"};
  PP_TRY_N(inv_names[mode], (launch_inv_x<T, TO>(ex.pl->g, ex.dt, ex.pl->fm, mode, spec, out, scale, accumulate, st,
                                                 pair)));
  return PS_OK;
}

void split_f32(double x, float& hi, float& lo) {
  hi = (float)x;
  lo = (float)(x - (double)hi);
}

size_t cell_count(const poisson_plan_s* pl) { return (size_t)pl->g.ny * pl->g.nz * pl->g.nx; }
size_t vface_count(const poisson_plan_s* pl) { return (size_t)(pl->g.ny + 1) * pl->g.nz * pl->g.nx; }

template <typename T>
poisson_status check_finite(Exec& ex, const void* x, size_t n) {
  if (!(ex.pl->flags & POISSON_CHECK_FINITE)) return PS_OK;
  cudaStream_t st = ex.st;
  PP_TRY_N("check_finite", launch_check_finite<T>((const T*)x, n, ex.dt.status, st));
  return PS_OK;
}

// POISSON_CHECK_FINITE on a velocity triple (u, w cell-sized, v with its ny+1 face planes).
template <typename T>
poisson_status check_finite_uvw(Exec& ex, const void* u, const void* v, const void* w) {
  PP_RET(check_finite<T>(ex, u, cell_count(ex.pl)));
  PP_RET(check_finite<T>(ex, v, vface_count(ex.pl)));
  return check_finite<T>(ex, w, cell_count(ex.pl));
}

// The solve of poisson_solve on any workspace (caller-owned or the library's static one).
//
// PP_FP32_REFINED keeps the pressure as an FP32 pair p = hi + lo in the workspace and never
// issues per-point FP64 arithmetic (slow on GB300):
//   hi = S32 f;  then for each of refine_steps corrections
//   r = (f - <f>) - L_h (hi + lo) in double-float arithmetic (from the second correction on as
//   r1 - L_h lo, r1 the first correction's residual kept as an FP32 pair);  d = S32 r;
//   lo = d (first) or lo += d, and on the last correction p = hi + (lo + d) is written in FP64
//   (both FP32 terms widened exactly, one FP64 addition).
// <f> is taken from the first solve's (0, 0) mode so that the FP32 transform of r carries no
// large constant; the dy-weighted sum of p is accumulated by every inverse pass and each
// correction's (0, 0) mode cancels it, so the gauge error of the FP32 transforms (invisible to
// the residual) does not persist.
// pair_out (PP_FP32_REFINED only): leave the result as the FP32 pair (hi, lo) in the workspace's
// pressure buffers (the last correction accumulated into lo) instead of writing FP64 p.
poisson_status solve_impl(Exec& ex, const void* rhs, void* p, bool pair_out = false) {
  const poisson_plan_s* pl = ex.pl;
  FwdArgs args = {};
  args.in = rhs;
  args.in_scale = 1.0;
  if (pl->precision == PP_FP64) {
    PP_RET(check_finite<double>(ex, rhs, cell_count(pl)));
    PP_RET((forward_and_core<double, double>(ex, FWD_PLAIN, args, GAUGE_ZERO)));
    PP_RET((inverse_x<double, double>(ex, INV_STORE, (double*)p, false)));
  } else if (pl->precision == PP_FP32) {
    PP_RET(check_finite<float>(ex, rhs, cell_count(pl)));
    PP_RET((forward_and_core<float, float>(ex, FWD_PLAIN, args, GAUGE_ZERO)));
    PP_RET((inverse_x<float, float>(ex, INV_STORE, (float*)p, false)));
  } else {
    float* hi = (float*)(ex.ws + pl->off_pbuf);
    float* lo = (float*)(ex.ws + pl->off_pbuf2);
    PP_RET(check_finite<double>(ex, rhs, cell_count(pl)));
    if (cudaMemsetAsync(ex.dt.acc, 0, 2 * sizeof(double), ex.st) != cudaSuccess) return PS_ECUDA;
    PP_RET((forward_and_core<float, double>(ex, FWD_PLAIN, args, GAUGE_STORE_MEAN)));
    PP_RET((inverse_x<float, float>(ex, INV_STORE, hi, true)));
    FwdArgs ra = {};
    ra.in = rhs;
    ra.p = hi;
    ra.in_scale = 1.0;
    split_f32(1.0 / (pl->g.dx * pl->g.dx), ra.idx2h, ra.idx2l);
    split_f32(1.0 / (pl->g.dz * pl->g.dz), ra.idz2h, ra.idz2l);
    // The first correction forms r1 = (f - <f>) - L_h hi (and, when more follow, stores it as an
    // FP32 pair); correction r then forms r1 - L_h lo, lo the sum of the corrections so far:
    // the same f - <f> - L_h (hi + lo) by linearity, without re-reading f and hi.
    float2* r1 = pl->refine >= 2 ? (float2*)(ex.ws + pl->off_r1) : nullptr;
    for (int r = 1; r <= pl->refine; ++r) {
      ra.p = r == 1 ? hi : lo;
      ra.rin = r == 1 ? nullptr : r1;
      ra.rout = r == 1 ? r1 : nullptr;
      PP_RET((forward_and_core<float, double>(ex, FWD_RESID, ra, GAUGE_OFFSET)));
      if (r < pl->refine) {
        PP_RET((inverse_x<float, float>(ex, r == 1 ? INV_STORE : INV_ACCUM, lo, true)));
      } else if (pair_out) {
        PP_RET((inverse_x<float, float>(ex, r == 1 ? INV_STORE : INV_ACCUM, lo, false)));
      } else {
        PairArgs pair{hi, r >= 2 ? lo : nullptr};   // the last pass: no pressure total needed
        PP_RET((inverse_x<float, double>(ex, INV_FINAL, (double*)p, false, pair)));
      }
    }
  }
  return PS_OK;
}

// Eqs. 4 and 7 on u, v, w in place (validated by the caller): divergence fused into the forward
// x-transform, the solve, the gradient correction.
poisson_status projection_impl(Exec& ex, void* u, void* v, void* w, void* p_out, double dt) {
  const poisson_plan_s* pl = ex.pl;
  cudaStream_t st = ex.st;
  FwdArgs args = {};
  args.u = u; args.v = v; args.w = w;
  args.in_scale = 1.0 / dt;
  if (pl->precision == PP_FP64) {
    double* p = p_out ? (double*)p_out : (double*)(pl->ws + pl->off_pbuf);
    PP_RET(check_finite_uvw<double>(ex, u, v, w));
    PP_RET((forward_and_core<double, double>(ex, FWD_DIV, args, GAUGE_ZERO)));
    PP_RET((inverse_x<double, double>(ex, INV_STORE, p, false)));
    PP_TRY_N("gradient", launch_gradient<double>(pl->g, ex.dt, p, (double*)u, (double*)v, (double*)w, dt, st));
  } else {
    float* p = p_out ? (float*)p_out : (float*)(pl->ws + pl->off_pbuf);
    PP_RET(check_finite_uvw<float>(ex, u, v, w));
    PP_RET((forward_and_core<float, float>(ex, FWD_DIV, args, GAUGE_ZERO)));
    PP_RET((inverse_x<float, float>(ex, INV_STORE, p, false)));
    PP_TRY_N("gradient", launch_gradient<float>(pl->g, ex.dt, p, (float*)u, (float*)v, (float*)w, dt, st));
  }
  return PS_OK;
}

// The projection of PP_FP32_REFINED plans (Eqs. 4 and 7) without per-point FP64 arithmetic:
// u, v, w converted in place to FP32 pairs, f = D(u)/dt assembled in FP64 into p_out (the
// solve's right-hand side), the refined solve into the workspace's pressure pair, then
// u = u - dt G p written in FP64 over the pairs and p (FP64) over f in p_out.
poisson_status projection_pairs(Exec& ex, void* u, void* v, void* w, void* p_out, double dt) {
  const poisson_plan_s* pl = ex.pl;
  PP_RET(check_finite_uvw<double>(ex, u, v, w));
  PP_TRY_N("to_pairs", launch_to_pairs((double*)u, cell_count(pl), ex.st));
  PP_TRY_N("to_pairs", launch_to_pairs((double*)v, vface_count(pl), ex.st));
  PP_TRY_N("to_pairs", launch_to_pairs((double*)w, cell_count(pl), ex.st));
  double* f = (double*)p_out;
  PP_TRY_N("divergence_df", launch_divergence_df(pl->g, ex.dt, (const float2*)u, (const float2*)v,
                                                 (const float2*)w, dt, f, ex.st));
  PP_RET(solve_impl(ex, f, nullptr, true));
  const float* hi = (const float*)(ex.ws + pl->off_pbuf);
  const float* lo = (const float*)(ex.ws + pl->off_pbuf2);
  PP_TRY_N("gradient_pairs", launch_gradient_pairs(pl->g, ex.dt, hi, lo, (double*)u, (double*)v, (double*)w,
                                                   (double*)p_out, dt, ex.st));
  return PS_OK;
}

poisson_status check_timestep_args(const poisson_plan_s* pl, const void* u, const void* v, const void* w,
                                   const void* ub, const void* vb, const void* wb, const void* p_out, double dt,
                                   double nu, double fx) {
  if (!pl || !u || !v || !w || !ub || !vb || !wb) return PS_EINVAL;
  if (!pl->children.empty()) return PS_EINVAL;
  if (!pl->ws) return PS_ENOWORKSPACE;
  if (!(dt > 0.0) || !isfinite(dt) || !(nu >= 0.0) || !isfinite(nu) || !isfinite(fx)) return PS_EINVAL;
  const void* all[7] = {u, v, w, ub, vb, wb, p_out};
  for (int a = 0; a < 7; ++a) {
    if (all[a] && !aligned16(all[a])) return PS_EINVAL;
    for (int b = 0; b < a; ++b)
      if (all[a] && all[a] == all[b]) return PS_EINVAL;   // every buffer distinct
  }
  return PS_OK;
}

// The predictor of PP_FP32_REFINED plans: u, v, w converted in place to FP32 pairs, the two Heun
// stages in double-float; u, v, w hold u_star as pairs on return.
poisson_status predictor_pairs(Exec& ex, void* u, void* v, void* w, void* ub, void* vb, void* wb, double dt,
                               double nu, double fx) {
  const poisson_plan_s* pl = ex.pl;
  PP_RET(check_finite_uvw<double>(ex, u, v, w));
  PP_TRY_N("to_pairs", launch_to_pairs((double*)u, cell_count(pl), ex.st));
  PP_TRY_N("to_pairs", launch_to_pairs((double*)v, vface_count(pl), ex.st));
  PP_TRY_N("to_pairs", launch_to_pairs((double*)w, cell_count(pl), ex.st));
  MomArgsDF s1{(const float2*)u, (const float2*)v, (const float2*)w, nullptr, nullptr, nullptr,
               (float2*)ub, (float2*)vb, (float2*)wb, 0.0, 1.0, dt, nu, fx};
  PP_TRY_N("momentum_df_1", launch_momentum_df(pl->g, ex.dt, s1, ex.st));
  MomArgsDF s2{(const float2*)ub, (const float2*)vb, (const float2*)wb, (const float2*)u, (const float2*)v,
               (const float2*)w, (float2*)u, (float2*)v, (float2*)w, 0.5, 0.5, 0.5 * dt, nu, fx};
  PP_TRY_N("momentum_df_2", launch_momentum_df(pl->g, ex.dt, s2, ex.st));
  return PS_OK;
}

// Heun's RK2 (Eqs. 5-6) in two launches: (ub, vb, wb) = u + dt R(u), then in place
// u = (u + ub + dt R(ub)) / 2.
poisson_status predictor_impl(Exec& ex, void* u, void* v, void* w, void* ub, void* vb, void* wb, double dt,
                              double nu, double fx) {
  const poisson_plan_s* pl = ex.pl;
  if (pl->precision == PP_FP64) {
    PP_RET(check_finite_uvw<double>(ex, u, v, w));
    MomArgs<double> s1{(const double*)u, (const double*)v, (const double*)w, nullptr, nullptr, nullptr,
                       (double*)ub, (double*)vb, (double*)wb, 0.0, 1.0, dt, nu, fx};
    PP_TRY_N("momentum_1", launch_momentum<double>(pl->g, ex.dt, s1, ex.st));
    MomArgs<double> s2{(const double*)ub, (const double*)vb, (const double*)wb, (const double*)u,
                       (const double*)v, (const double*)w, (double*)u, (double*)v, (double*)w,
                       0.5, 0.5, 0.5 * dt, nu, fx};
    PP_TRY_N("momentum_2", launch_momentum<double>(pl->g, ex.dt, s2, ex.st));
  } else {
    PP_RET(check_finite_uvw<float>(ex, u, v, w));
    MomArgs<float> s1{(const float*)u, (const float*)v, (const float*)w, nullptr, nullptr, nullptr,
                      (float*)ub, (float*)vb, (float*)wb, 0.0, 1.0, dt, nu, fx};
    PP_TRY_N("momentum_1", launch_momentum<float>(pl->g, ex.dt, s1, ex.st));
    MomArgs<float> s2{(const float*)ub, (const float*)vb, (const float*)wb, (const float*)u,
                      (const float*)v, (const float*)w, (float*)u, (float*)v, (float*)w,
                      0.5, 0.5, 0.5 * dt, nu, fx};
    PP_TRY_N("momentum_2", launch_momentum<float>(pl->g, ex.dt, s2, ex.st));
  }
  return PS_OK;
}

// The inverse x-transform (STORE) of the wall-normal rows [j0, j1): the lines of those rows are
// one contiguous stretch of the spectrum and of the output, so the launch takes them as a grid of
// j1 - j0 rows (the STORE form depends on nothing else of the row index).
template <typename T>
poisson_status inverse_x_rows(Exec& ex, T* out, int j0, int j1) {
  const Geometry& g = ex.pl->g;
  Geometry gs = g;
  gs.ny = j1 - j0;
  cplx<T>* spec = (cplx<T>*)(ex.ws + ex.pl->off_spec) + (size_t)j0 * g.nz * g.pitch;
  const double scale = 1.0 / ((double)g.nx * (double)g.nz);
  PP_TRY_N("inv_x", (launch_inv_x<T, T>(gs, ex.dt, ex.pl->fm, INV_STORE, spec, out + (size_t)j0 * g.nz * g.nx, scale,
                                        false, ex.st, PairArgs{nullptr, nullptr})));
  return PS_OK;
}

// projection_timestep_host of PP_FP64 and PP_FP32 plans with its copies overlapped.  The rows of
// u, w and the v faces go over in HOST_CHUNKS row chunks on the plan's copy stream, and momentum
// stage 1 of a chunk (Eqs. 5-6) starts on the caller's stream once the chunk and the row above it
// have arrived (a stage-1 row reads its neighbours j-1 and j+1).  Stage 2 and the solve follow as
// in projection_timestep; the inverse x-transform and the gradient correction (Eq. 4) then run
// chunk by chunk, and each chunk of p (final after its inverse transform) and of u, v, w (final
// after its gradient, which reads p rows j-1 and j) goes back to the host while the next chunk is
// computed.  The results are those of projection_timestep bit for bit.
template <typename T>
poisson_status timestep_overlapped(poisson_plan_s* pl, const void* u_h, const void* v_h, const void* w_h, void* p_h,
                                   T* u, T* v, T* w, T* ub, T* vb, T* wb, T* p_dev, double dt, double nu, double fx,
                                   cudaStream_t st) {
  const Geometry& g = pl->g;
  constexpr int C = pp::HOST_CHUNKS;
  if (!pl->copy_st) {
    if (cudaStreamCreateWithFlags(&pl->copy_st, cudaStreamNonBlocking) != cudaSuccess) return PS_ECUDA;
    for (cudaEvent_t& e : pl->copy_ev)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return PS_ECUDA;
  }
  cudaStream_t cp = pl->copy_st;
  cudaEvent_t* ev_in = pl->copy_ev;             // input chunk c has arrived
  cudaEvent_t ev_start = pl->copy_ev[C];
  cudaEvent_t* ev_p = pl->copy_ev + C + 1;      // p rows of chunk c are final
  cudaEvent_t* ev_g = pl->copy_ev + 2 * C + 1;  // u, v, w rows of chunk c are final
  // the copies start after the caller's earlier work on these buffers
  if (cudaEventRecord(ev_start, st) != cudaSuccess) return PS_ECUDA;
  if (cudaStreamWaitEvent(cp, ev_start, 0) != cudaSuccess) return PS_ECUDA;
  const size_t plane = (size_t)g.nz * g.nx;
  int rows[C + 1];
  for (int c = 0; c <= C; ++c) rows[c] = (int)((long long)g.ny * c / C);
  // chunk c: cell rows [rows[c], rows[c+1]); v faces the same, plus the top wall face in the last
  auto cells = [&](int c) { return (size_t)(rows[c + 1] - rows[c]) * plane; };
  auto faces = [&](int c) { return (size_t)((c == C - 1 ? g.ny + 1 : rows[c + 1]) - rows[c]) * plane; };
  for (int c = 0; c < C; ++c) {
    const size_t o = (size_t)rows[c] * plane;
    if (cudaMemcpyAsync(u + o, (const T*)u_h + o, cells(c) * sizeof(T), cudaMemcpyHostToDevice, cp) != cudaSuccess ||
        cudaMemcpyAsync(w + o, (const T*)w_h + o, cells(c) * sizeof(T), cudaMemcpyHostToDevice, cp) != cudaSuccess ||
        cudaMemcpyAsync(v + o, (const T*)v_h + o, faces(c) * sizeof(T), cudaMemcpyHostToDevice, cp) != cudaSuccess)
      return PS_ECUDA;
    if (cudaEventRecord(ev_in[c], cp) != cudaSuccess) return PS_ECUDA;
  }
  pl->launches = 0;
  pl->nev = 0;
  Exec ex{pl, pl->ws, pl->dt, st, false};
  for (int c = 0; c < C; ++c) {
    if (cudaStreamWaitEvent(st, ev_in[c + 1 < C ? c + 1 : C - 1], 0) != cudaSuccess) return PS_ECUDA;
    MomArgs<T> s1{u, v, w, nullptr, nullptr, nullptr, ub, vb, wb, 0.0, 1.0, dt, nu, fx};
    PP_TRY_N("momentum_1", launch_momentum<T>(g, ex.dt, s1, st, rows[c], rows[c + 1]));
  }
  MomArgs<T> s2{ub, vb, wb, u, v, w, u, v, w, 0.5, 0.5, 0.5 * dt, nu, fx};
  PP_TRY_N("momentum_2", launch_momentum<T>(g, ex.dt, s2, st));
  FwdArgs args = {};
  args.u = u; args.v = v; args.w = w;
  args.in_scale = 1.0 / dt;
  T* p = p_dev ? p_dev : (T*)(pl->ws + pl->off_pbuf);
  PP_RET((forward_and_core<T, T>(ex, FWD_DIV, args, GAUGE_ZERO)));
  for (int c = 0; c < C; ++c) {
    const size_t o = (size_t)rows[c] * plane;
    PP_RET(inverse_x_rows<T>(ex, p, rows[c], rows[c + 1]));
    if (p_h) {
      if (cudaEventRecord(ev_p[c], st) != cudaSuccess || cudaStreamWaitEvent(cp, ev_p[c], 0) != cudaSuccess ||
          cudaMemcpyAsync((T*)p_h + o, p + o, cells(c) * sizeof(T), cudaMemcpyDeviceToHost, cp) != cudaSuccess)
        return PS_ECUDA;
    }
    PP_TRY_N("gradient", launch_gradient<T>(g, ex.dt, p, u, v, w, dt, st, rows[c], rows[c + 1]));
    if (cudaEventRecord(ev_g[c], st) != cudaSuccess || cudaStreamWaitEvent(cp, ev_g[c], 0) != cudaSuccess)
      return PS_ECUDA;
    if (cudaMemcpyAsync((T*)u_h + o, u + o, cells(c) * sizeof(T), cudaMemcpyDeviceToHost, cp) != cudaSuccess ||
        cudaMemcpyAsync((T*)w_h + o, w + o, cells(c) * sizeof(T), cudaMemcpyDeviceToHost, cp) != cudaSuccess ||
        cudaMemcpyAsync((T*)v_h + o, v + o, faces(c) * sizeof(T), cudaMemcpyDeviceToHost, cp) != cudaSuccess)
      return PS_ECUDA;
  }
  if (cudaStreamSynchronize(cp) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return PS_ECUDA;
  return PS_OK;
}

}  // namespace

namespace pp {
poisson_status solve_on_workspace(poisson_plan_s* pl, unsigned char* ws, const DevTables& dt, const void* rhs,
                                  void* p, cudaStream_t st) {
  Exec ex{pl, ws, dt, st, false};
  pl->launches = 0;
  pl->nev = 0;
  return solve_impl(ex, rhs, p);
}
}  // namespace pp

extern "C" {

poisson_status poisson_solve(poisson_plan_t pl, const void* rhs, void* p, void* stream) {
  if (!pl || !rhs || !p) return PS_EINVAL;
  if (!pl->children.empty()) return PS_EINVAL;   // batched plans use poisson_solve_batched
  if (!pl->ws) return PS_ENOWORKSPACE;
  if (!aligned16(rhs) || !aligned16(p)) return PS_EINVAL;
  if (pl->precision == PP_FP32_REFINED && rhs == p) return PS_EINVAL;  // the residual re-reads rhs
  pl->launches = 0;
  pl->nev = 0;
  Exec ex{pl, pl->ws, pl->dt, (cudaStream_t)stream, (pl->flags & POISSON_TIMING) != 0};
  return solve_impl(ex, rhs, p);
}

// S^T g for the gauged solve S of poisson_solve: since L_h^T = W L_h W^-1 (W = diag(dy_j)) and the
// mean removal and the gauge of S transpose into each other, S^T g = W S(W^-1 g).
poisson_status poisson_solve_adjoint(poisson_plan_t pl, const void* g, void* q, void* stream) {
  if (!pl || !g || !q) return PS_EINVAL;
  if (!pl->children.empty()) return PS_EINVAL;
  if (!pl->ws) return PS_ENOWORKSPACE;
  if (!aligned16(g) || !aligned16(q)) return PS_EINVAL;
  pl->launches = 0;
  pl->nev = 0;
  Exec ex{pl, pl->ws, pl->dt, (cudaStream_t)stream, (pl->flags & POISSON_TIMING) != 0};
  const Geometry& geo = pl->g;
  cudaStream_t st = ex.st;
  if (pl->precision == PP_FP32) {
    PP_TRY_N("scale_in", launch_scale_planes<float>(geo, ex.dt, (const float*)g, (float*)q, false, st));
    PP_RET(solve_impl(ex, q, q));
    PP_TRY_N("scale_out", launch_scale_planes<float>(geo, ex.dt, (const float*)q, (float*)q, true, st));
  } else if (pl->precision == PP_FP64) {
    PP_TRY_N("scale_in", launch_scale_planes<double>(geo, ex.dt, (const double*)g, (double*)q, false, st));
    PP_RET(solve_impl(ex, q, q));
    PP_TRY_N("scale_out", launch_scale_planes<double>(geo, ex.dt, (const double*)q, (double*)q, true, st));
  } else {
    // the refined solve re-reads its rhs: solve into the workspace's pressure pair, then weight it
    PP_TRY_N("scale_in", launch_scale_planes<double>(geo, ex.dt, (const double*)g, (double*)q, false, st));
    PP_RET(solve_impl(ex, q, nullptr, true));
    const float* hi = (const float*)(ex.ws + pl->off_pbuf);
    const float* lo = (const float*)(ex.ws + pl->off_pbuf2);
    PP_TRY_N("weighted_pair", launch_weighted_pair(geo, ex.dt, hi, lo, (double*)q, st));
  }
  return PS_OK;
}

poisson_status projection_step(poisson_plan_t pl, void* u, void* v, void* w, void* p_out, double dt,
                               void* stream) {
  if (!pl || !u || !v || !w) return PS_EINVAL;
  if (!pl->ws) return PS_ENOWORKSPACE;
  if (!(dt > 0.0) || !isfinite(dt)) return PS_EINVAL;
  if (!aligned16(u) || !aligned16(v) || !aligned16(w) || (p_out && !aligned16(p_out))) return PS_EINVAL;
  if (!pl->children.empty()) return PS_EINVAL;
  if (pl->precision == PP_FP32_REFINED) {
    // p_out carries the FP64 right-hand side during the solve, so it is required here
    if (!p_out) return PS_EINVAL;
    const void* all[4] = {u, v, w, p_out};
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < a; ++b)
        if (all[a] == all[b]) return PS_EINVAL;
  }
  pl->launches = 0;
  pl->nev = 0;
  Exec ex{pl, pl->ws, pl->dt, (cudaStream_t)stream, (pl->flags & POISSON_TIMING) != 0};
  if (pl->precision == PP_FP32_REFINED) return projection_pairs(ex, u, v, w, p_out, dt);
  return projection_impl(ex, u, v, w, p_out, dt);
}

poisson_status momentum_predictor(poisson_plan_t pl, void* u, void* v, void* w, void* ub, void* vb, void* wb,
                                  double dt, double nu, double fx, void* stream) {
  PP_RET(check_timestep_args(pl, u, v, w, ub, vb, wb, nullptr, dt, nu, fx));
  pl->launches = 0;
  pl->nev = 0;
  Exec ex{pl, pl->ws, pl->dt, (cudaStream_t)stream, (pl->flags & POISSON_TIMING) != 0};
  if (pl->precision != PP_FP32_REFINED) return predictor_impl(ex, u, v, w, ub, vb, wb, dt, nu, fx);
  PP_RET(predictor_pairs(ex, u, v, w, ub, vb, wb, dt, nu, fx));
  PP_TRY_N("from_pairs", launch_from_pairs((double*)u, cell_count(pl), ex.st));
  PP_TRY_N("from_pairs", launch_from_pairs((double*)v, vface_count(pl), ex.st));
  PP_TRY_N("from_pairs", launch_from_pairs((double*)w, cell_count(pl), ex.st));
  return PS_OK;
}

poisson_status projection_timestep(poisson_plan_t pl, void* u, void* v, void* w, void* ub, void* vb, void* wb,
                                   void* p_out, double dt, double nu, double fx, void* stream) {
  PP_RET(check_timestep_args(pl, u, v, w, ub, vb, wb, p_out, dt, nu, fx));
  pl->launches = 0;
  pl->nev = 0;
  Exec ex{pl, pl->ws, pl->dt, (cudaStream_t)stream, (pl->flags & POISSON_TIMING) != 0};
  if (pl->precision != PP_FP32_REFINED) {
    PP_RET(predictor_impl(ex, u, v, w, ub, vb, wb, dt, nu, fx));
    return projection_impl(ex, u, v, w, p_out, dt);
  }
  // refined: u_star as pairs; f = D(u_star)/dt into ub (FP64); the refined solve into p_out or
  // vb; then the FP64 correction u = u_star - dt G p written over the pairs
  PP_RET(predictor_pairs(ex, u, v, w, ub, vb, wb, dt, nu, fx));
  double* f = (double*)ub;
  PP_TRY_N("divergence_df", launch_divergence_df(pl->g, ex.dt, (const float2*)u, (const float2*)v,
                                                 (const float2*)w, dt, f, ex.st));
  PP_RET(solve_impl(ex, f, nullptr, true));   // p = hi + lo in the workspace
  const float* hi = (const float*)(pl->ws + pl->off_pbuf);
  const float* lo = (const float*)(pl->ws + pl->off_pbuf2);
  PP_TRY_N("gradient_pairs", launch_gradient_pairs(pl->g, ex.dt, hi, lo, (double*)u, (double*)v, (double*)w,
                                                   (double*)p_out, dt, ex.st));
  return PS_OK;
}

poisson_status projection_step_adjoint(poisson_plan_t pl, void* gu, void* gv, void* gw, void* stream) {
  if (!pl || !gu || !gv || !gw) return PS_EINVAL;
  if (!pl->ws) return PS_ENOWORKSPACE;
  if (!aligned16(gu) || !aligned16(gv) || !aligned16(gw)) return PS_EINVAL;
  if (pl->precision == PP_FP32_REFINED) return PS_EUNSUPPORTED;
  pl->launches = 0;
  pl->nev = 0;
  Exec ex{pl, pl->ws, pl->dt, (cudaStream_t)stream, (pl->flags & POISSON_TIMING) != 0};
  cudaStream_t st = ex.st;
  FwdArgs args = {};
  args.u = gu; args.v = gv; args.w = gw;
  args.in_scale = 1.0;
  if (pl->precision == PP_FP64) {
    double* q = (double*)(pl->ws + pl->off_pbuf);
    PP_RET((forward_and_core<double, double>(ex, FWD_GRADT, args, GAUGE_ZERO)));
    PP_RET((inverse_x<double, double>(ex, INV_STORE, q, false)));
    PP_TRY_N("adj_epilogue",
             launch_adjoint_epilogue<double>(pl->g, ex.dt, q, (double*)gu, (double*)gv, (double*)gw, st));
  } else {
    float* q = (float*)(pl->ws + pl->off_pbuf);
    PP_RET((forward_and_core<float, float>(ex, FWD_GRADT, args, GAUGE_ZERO)));
    PP_RET((inverse_x<float, float>(ex, INV_STORE, q, false)));
    PP_TRY_N("adj_epilogue",
             launch_adjoint_epilogue<float>(pl->g, ex.dt, q, (float*)gu, (float*)gv, (float*)gw, st));
  }
  return PS_OK;
}

poisson_status projection_step_host(poisson_plan_t pl, void* u_h, void* v_h, void* w_h, void* p_h, void* u_d,
                                    void* v_d, void* w_d, void* p_d, double dt, void* stream) {
  if (!pl || !u_h || !v_h || !w_h || !u_d || !v_d || !w_d) return PS_EINVAL;
  if (p_h && !p_d) return PS_EINVAL;
  if (pl->precision == PP_FP32_REFINED && !p_d) return PS_EINVAL;   // the solve's right-hand side
  cudaStream_t st = (cudaStream_t)stream;
  const size_t es = pl->precision == PP_FP32 ? 4 : 8;
  const size_t nc = cell_count(pl) * es, nv = vface_count(pl) * es;
  if (cudaMemcpyAsync(u_d, u_h, nc, cudaMemcpyHostToDevice, st) != cudaSuccess) return PS_ECUDA;
  if (cudaMemcpyAsync(v_d, v_h, nv, cudaMemcpyHostToDevice, st) != cudaSuccess) return PS_ECUDA;
  if (cudaMemcpyAsync(w_d, w_h, nc, cudaMemcpyHostToDevice, st) != cudaSuccess) return PS_ECUDA;
  void* pd = (p_h || pl->precision == PP_FP32_REFINED) ? p_d : nullptr;
  PP_RET(projection_step(pl, u_d, v_d, w_d, pd, dt, stream));
  if (cudaMemcpyAsync(u_h, u_d, nc, cudaMemcpyDeviceToHost, st) != cudaSuccess) return PS_ECUDA;
  if (cudaMemcpyAsync(v_h, v_d, nv, cudaMemcpyDeviceToHost, st) != cudaSuccess) return PS_ECUDA;
  if (cudaMemcpyAsync(w_h, w_d, nc, cudaMemcpyDeviceToHost, st) != cudaSuccess) return PS_ECUDA;
  if (p_h && cudaMemcpyAsync(p_h, p_d, nc, cudaMemcpyDeviceToHost, st) != cudaSuccess) return PS_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return PS_ECUDA;
  return PS_OK;
}

poisson_status projection_timestep_host(poisson_plan_t pl, void* u_h, void* v_h, void* w_h, void* p_h, void* u_d,
                                        void* v_d, void* w_d, void* p_d, void* ub, void* vb, void* wb, double dt,
                                        double nu, double fx, void* stream) {
  if (!u_h || !v_h || !w_h) return PS_EINVAL;
  if (p_h && !p_d) return PS_EINVAL;
  PP_RET(check_timestep_args(pl, u_d, v_d, w_d, ub, vb, wb, p_h ? p_d : nullptr, dt, nu, fx));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t es = pl->precision == PP_FP32 ? 4 : 8;
  const size_t nc = cell_count(pl) * es, nv = vface_count(pl) * es;
  const bool overlap = pl->precision != PP_FP32_REFINED && !(pl->flags & (POISSON_CHECK_FINITE | POISSON_TIMING)) &&
                       pl->g.ny >= 2 * pp::HOST_CHUNKS;
  if (overlap) {
    if (pl->precision == PP_FP64)
      return timestep_overlapped<double>(pl, u_h, v_h, w_h, p_h, (double*)u_d, (double*)v_d, (double*)w_d,
                                         (double*)ub, (double*)vb, (double*)wb, p_h ? (double*)p_d : nullptr, dt, nu,
                                         fx, st);
    return timestep_overlapped<float>(pl, u_h, v_h, w_h, p_h, (float*)u_d, (float*)v_d, (float*)w_d, (float*)ub,
                                      (float*)vb, (float*)wb, p_h ? (float*)p_d : nullptr, dt, nu, fx, st);
  }
  if (cudaMemcpyAsync(u_d, u_h, nc, cudaMemcpyHostToDevice, st) != cudaSuccess) return PS_ECUDA;
  if (cudaMemcpyAsync(v_d, v_h, nv, cudaMemcpyHostToDevice, st) != cudaSuccess) return PS_ECUDA;
  if (cudaMemcpyAsync(w_d, w_h, nc, cudaMemcpyHostToDevice, st) != cudaSuccess) return PS_ECUDA;
  PP_RET(projection_timestep(pl, u_d, v_d, w_d, ub, vb, wb, p_h ? p_d : nullptr, dt, nu, fx, stream));
  if (cudaMemcpyAsync(u_h, u_d, nc, cudaMemcpyDeviceToHost, st) != cudaSuccess) return PS_ECUDA;
  if (cudaMemcpyAsync(v_h, v_d, nv, cudaMemcpyDeviceToHost, st) != cudaSuccess) return PS_ECUDA;
  if (cudaMemcpyAsync(w_h, w_d, nc, cudaMemcpyDeviceToHost, st) != cudaSuccess) return PS_ECUDA;
  if (p_h && cudaMemcpyAsync(p_h, p_d, nc, cudaMemcpyDeviceToHost, st) != cudaSuccess) return PS_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return PS_ECUDA;
  return PS_OK;
}

poisson_status poisson_divergence(poisson_plan_t pl, const void* u, const void* v, const void* w, void* f, double dt,
                                  void* stream) {
  if (!pl || !u || !v || !w || !f) return PS_EINVAL;
  if (!pl->children.empty()) return PS_EINVAL;
  if (!pl->ws) return PS_ENOWORKSPACE;
  if (!(dt > 0.0) || !isfinite(dt)) return PS_EINVAL;
  if (!aligned16(u) || !aligned16(v) || !aligned16(w) || !aligned16(f)) return PS_EINVAL;
  if (f == u || f == v || f == w) return PS_EINVAL;
  pl->launches = 0;
  pl->nev = 0;
  Exec ex{pl, pl->ws, pl->dt, (cudaStream_t)stream, (pl->flags & POISSON_TIMING) != 0};
  if (pl->precision == PP_FP32)
    PP_TRY_N("divergence", launch_divergence<float>(pl->g, ex.dt, (const float*)u, (const float*)v, (const float*)w,
                                                    (float*)f, dt, ex.st));
  else
    PP_TRY_N("divergence", launch_divergence<double>(pl->g, ex.dt, (const double*)u, (const double*)v,
                                                     (const double*)w, (double*)f, dt, ex.st));
  return PS_OK;
}

poisson_status poisson_plan_set_chain(poisson_plan_t pl, int slab_cols, int streams) {
  if (!pl || !pl->children.empty() || slab_cols < 0 || streams < 1 || streams > 2) return PS_EINVAL;
  if (slab_cols == 0) {
    pl->slab_cols = 0;
    pl->chain_streams = 1;
    return PS_OK;
  }
  const Geometry& g = pl->g;
  const int wz = pp::fft_z_fast_tile<float>(g);
  const bool path_ok = pl->precision != PP_FP64 && !pl->has_tri && pp::scan_tridiag_ok(g.ny, pl->parts) &&
                       !g.generic_fft && wz > 0;
  if (!path_ok) return PS_EUNSUPPORTED;
  const int step = wz > pp::reg_systems_per_cta(pl->parts) ? wz : pp::reg_systems_per_cta(pl->parts);
  if (slab_cols % step || slab_cols <= pl->low) return PS_EUNSUPPORTED;
  if (streams == 2 && !pl->chain_st) {
    if (cudaStreamCreateWithFlags(&pl->chain_st, cudaStreamNonBlocking) != cudaSuccess) return PS_ECUDA;
    for (cudaEvent_t& e : pl->chain_ev)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return PS_ECUDA;
  }
  pl->slab_cols = slab_cols;
  pl->chain_streams = streams;
  return PS_OK;
}

poisson_status poisson_device_status(poisson_plan_t pl, void* stream) {
  if (!pl) return PS_EINVAL;
  if (!pl->ws || !pl->dt.status) return PS_ENOWORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  int h = 0;
  if (cudaMemcpyAsync(&h, pl->dt.status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return PS_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return PS_ECUDA;
  if (cudaMemsetAsync(pl->dt.status, 0, sizeof(int), st) != cudaSuccess) return PS_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return PS_ECUDA;
  return (poisson_status)h;
}

int poisson_last_launch_count(poisson_plan_t pl) { return pl ? pl->launches : -1; }

int poisson_stage_times(poisson_plan_t pl, float* ms, const char** names, int max) {
  if (!pl || !(pl->flags & POISSON_TIMING)) return -1;
  const int n = pl->nev;
  if (n == 0) return 0;
  if (cudaEventSynchronize(pl->ev[2 * n - 1]) != cudaSuccess) return -1;
  for (int i = 0; i < n && i < max; ++i) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, pl->ev[2 * i], pl->ev[2 * i + 1]) != cudaSuccess) return -1;
    if (ms) ms[i] = t;
    if (names) names[i] = pl->ev_names[i];
  }
  return n;
}

poisson_status poisson_plan_destroy(poisson_plan_t pl) {
  if (pl) {
    for (cudaEvent_t e : pl->ev) cudaEventDestroy(e);
    if (pl->chain_st) cudaStreamDestroy(pl->chain_st);
    if (pl->copy_st) cudaStreamDestroy(pl->copy_st);
    for (cudaEvent_t e : pl->copy_ev)
      if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : pl->chain_ev)
      if (e) cudaEventDestroy(e);
    pp::destroy_batch(pl);
  }
  delete pl;
  return PS_OK;
}

}  // extern "C"
