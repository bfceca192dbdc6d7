// poisson_solve_static_ws: poisson_solve without caller-provided device workspace.
//
// Some callers cannot call cudaMalloc at the point where they need a pressure solve: a host
// application whose own memory pool owns the device and forbids allocations from libraries,
// or a time-critical loop where the implicit device synchronisation and latency of
// cudaMalloc / cudaFree are not acceptable.  For them this entry point runs the same kernels
// as poisson_solve, with the workspace (spectral buffer, tables, status word) placed in one
// file-scope device array of fixed size instead of caller memory.  It calls no allocator.
//
// The array lives in every GPU that loads the library until the process exits.  In host code
// its name only stands for the device object; the device address is obtained once per device
// with cudaGetSymbolAddress (with that device current) and passed to the kernels.
#include "internal.h"

namespace {

constexpr size_t kStaticWorkspaceBytes = (size_t)POISSON_STATIC_WS_MAX_BYTES;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_ws[kStaticWorkspaceBytes];

unsigned char* g_static_ptr[kMaxDevices] = {};   // device address of g_static_ws, per device

poisson_status static_workspace_address(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PS_ECUDA;
  if (!g_static_ptr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_static_ws) != cudaSuccess || !ptr) return PS_ECUDA;
    g_static_ptr[dev] = (unsigned char*)ptr;
  }
  *out = g_static_ptr[dev];
  return PS_OK;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

#define PP_CHECK(expr)                                 \
  do {                                                 \
    if ((expr) != cudaSuccess) return PS_ECUDA;        \
  } while (0)

template <typename T>
poisson_status core(const poisson_plan_s* pl, const pp::DevTables& dt, unsigned char* ws, cudaStream_t st) {
  using namespace pp;
  const Geometry& g = pl->g;
  cplx<T>* spec = (cplx<T>*)(ws + pl->off_spec);
  PP_CHECK(launch_fft_z<T>(g, dt, pl->fz, -1, spec, st));
  if constexpr (sizeof(T) == 8) {
    PP_CHECK((launch_tridiag<double, double>(g, dt, pl->parts, -1, false, spec, st)));
  } else {
    PP_CHECK((launch_tridiag<float, float>(g, dt, pl->parts, pl->low, false, spec, st)));
    if (pl->low >= 0)
      PP_CHECK(launch_tridiag_low64(g, dt, pl->parts, pl->low, spec, (cplx<double>*)(ws + pl->off_scratch), st));
  }
  PP_CHECK(launch_mode00<T>(g, dt, false, spec, st));
  PP_CHECK(launch_fft_z<T>(g, dt, pl->fz, +1, spec, st));
  return PS_OK;
}

template <typename T, typename TIO>
poisson_status solve_pass(const poisson_plan_s* pl, const pp::DevTables& dt, unsigned char* ws, pp::FwdMode mode,
                          const pp::FwdArgs& args, pp::InvMode imode, TIO* out, cudaStream_t st) {
  using namespace pp;
  cplx<T>* spec = (cplx<T>*)(ws + pl->off_spec);
  PP_CHECK((launch_fwd_x<T, TIO>(pl->g, dt, pl->fm, mode, args, spec, st)));
  poisson_status s = core<T>(pl, dt, ws, st);
  if (s != PS_OK) return s;
  const double scale = 1.0 / ((double)pl->g.nx * (double)pl->g.nz);
  PP_CHECK((launch_inv_x<T, TIO>(pl->g, dt, pl->fm, imode, spec, out, scale, st)));
  return PS_OK;
}

}  // namespace

extern "C" poisson_status poisson_solve_static_ws(poisson_plan_t pl, const void* rhs, void* p, void* stream) {
  using namespace pp;
  if (!pl || !rhs || !p) return PS_EINVAL;
  if (!aligned16(rhs) || !aligned16(p)) return PS_EINVAL;
  if (pl->ws_bytes > kStaticWorkspaceBytes) return PS_EUNSUPPORTED;   // grid too large for the array
  if (pl->precision == PP_FP32_REFINED && rhs == p) return PS_EINVAL;
  unsigned char* ws = nullptr;
  poisson_status s = static_workspace_address(&ws);
  if (s != PS_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  // The array keeps whatever the previous call left: reload this plan's tables and clear the
  // status word (the only region that must start at zero) on every call.
  PP_CHECK(cudaMemcpyAsync(ws + pl->off_tables, pl->host_tables.data(), pl->host_tables.size(),
                           cudaMemcpyHostToDevice, st));
  PP_CHECK(cudaMemsetAsync(ws + pl->off_status, 0, 256, st));
  unsigned char* tb = ws + pl->off_tables;
  const size_t* to = pl->tab_offsets;
  DevTables dt;
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
  dt.status = (int*)(ws + pl->off_status);
  FwdArgs args = {};
  args.in = rhs;
  args.in_scale = 1.0;
  if (pl->precision == PP_FP64)
    return solve_pass<double, double>(pl, dt, ws, FWD_PLAIN, args, INV_STORE, (double*)p, st);
  if (pl->precision == PP_FP32)
    return solve_pass<float, float>(pl, dt, ws, FWD_PLAIN, args, INV_STORE, (float*)p, st);
  s = solve_pass<float, double>(pl, dt, ws, FWD_PLAIN, args, INV_STORE, (double*)p, st);
  for (int r = 0; s == PS_OK && r < pl->refine; ++r) {
    FwdArgs ra = {};
    ra.in = rhs;
    ra.p = p;
    ra.in_scale = 1.0;
    s = solve_pass<float, double>(pl, dt, ws, FWD_RESID, ra, INV_ACCUM, (double*)p, st);
  }
  return s;
}
