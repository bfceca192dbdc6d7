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
// with cudaGetSymbolAddress (with that device current, under a lock) and passed to the kernels.
#include <mutex>

#include "internal.h"

namespace {

constexpr size_t kStaticWorkspaceBytes = (size_t)POISSON_STATIC_WS_MAX_BYTES;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_ws[kStaticWorkspaceBytes];

std::mutex g_static_mu;                          // guards the per-device address cache
unsigned char* g_static_ptr[kMaxDevices] = {};   // device address of g_static_ws, per device

poisson_status static_workspace_address(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PS_ECUDA;
  std::lock_guard<std::mutex> lock(g_static_mu);   // first calls from several threads look it up once
  if (!g_static_ptr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_static_ws) != cudaSuccess || !ptr) return PS_ECUDA;
    g_static_ptr[dev] = (unsigned char*)ptr;
  }
  *out = g_static_ptr[dev];
  return PS_OK;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

extern "C" poisson_status poisson_solve_static_ws(poisson_plan_t pl, const void* rhs, void* p, void* stream) {
  if (!pl || !rhs || !p) return PS_EINVAL;
  if (!pl->children.empty()) return PS_EINVAL;   // batched plans have no geometry of their own
  if (!aligned16(rhs) || !aligned16(p)) return PS_EINVAL;
  if (pl->ws_bytes > kStaticWorkspaceBytes) return PS_EUNSUPPORTED;   // grid too large for the array
  if (pl->precision == PP_FP32_REFINED && rhs == p) return PS_EINVAL;
  unsigned char* ws = nullptr;
  poisson_status s = static_workspace_address(&ws);
  if (s != PS_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  // The array keeps whatever the previous call left: reload this plan's tables, rebuild its
  // PDD factors and clear the status word (the only region that must start at zero).  The
  // table image is ordinary (pageable) host memory, so this copy returns only once the stream
  // has reached it.
  if (cudaMemcpyAsync(ws + pl->off_tables, pl->host_tables.data(), pl->host_tables.size(),
                      cudaMemcpyHostToDevice, st) != cudaSuccess)
    return PS_ECUDA;
  if (cudaMemsetAsync(ws + pl->off_status, 0, 256, st) != cudaSuccess) return PS_ECUDA;
  const pp::DevTables dt = pp::bind_tables(pl, ws);
  if (pl->has_tri && pp::launch_tridiag_setup(pl->g, dt, pl->parts, st) != cudaSuccess) return PS_ECUDA;
  if (!pl->has_tri && pp::launch_reduced_setup(pl->g, dt, pl->parts, pl->tridiag == PT_PDD_TRUNCATED,
                                               (float*)(ws + pl->off_red), st) != cudaSuccess)
    return PS_ECUDA;
  return pp::solve_on_workspace(pl, ws, dt, rhs, p, st);
}
