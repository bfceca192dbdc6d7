// Batched solves of independent, uneven-size problems in one graph launch, and the autotuner.
//
// A batched plan holds one sub-plan per instance and carves their workspaces out of one caller
// allocation.  poisson_solve_batched captures, once, a CUDA graph in which every instance's
// kernel sequence (the same pipeline as poisson_solve) is a branch forked from the caller's
// stream, so that small instances run concurrently and the host pays one graph launch per
// batch instead of ~7 launches per instance; later calls with the same pointers replay it.
//
// poisson_autotune picks, per grid, the PDD partition count and the FFT tiling (compile-time
// specialised or generic kernels) by timing the actual solve on the device.
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "internal.h"

namespace {

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

void drop_graph(poisson_plan_s* pl) {
  if (pl->gexec) cudaGraphExecDestroy(pl->gexec);
  pl->gexec = nullptr;
  pl->g_rhs.clear();
  pl->g_p.clear();
}

}  // namespace

namespace pp {

poisson_status set_batch_workspace(poisson_plan_s* pl, unsigned char* ws, void* stream) {
  size_t off = 0;
  for (poisson_plan_s* c : pl->children) {
    const poisson_status s = poisson_set_workspace(c, ws + off, c->ws_bytes, stream);
    if (s != PS_OK) return s;
    off += align256(c->ws_bytes);
  }
  pl->ws = ws;
  drop_graph(pl);
  pl->warmed = false;
  return PS_OK;
}

void destroy_batch(poisson_plan_s* pl) {
  drop_graph(pl);
  for (cudaStream_t s : pl->forks) cudaStreamDestroy(s);
  for (cudaEvent_t e : pl->fork_ev) cudaEventDestroy(e);
  for (poisson_plan_s* c : pl->children) poisson_plan_destroy(c);
  pl->children.clear();
}

}  // namespace pp

extern "C" {

poisson_status poisson_plan_batched(const poisson_desc* descs, int count, poisson_plan_t* out) {
  if (!descs || !out || count <= 0) return PS_EINVAL;
  *out = nullptr;
  poisson_plan_s* pl = new (std::nothrow) poisson_plan_s();
  if (!pl) return PS_ENOMEM;
  size_t total = 0;
  for (int i = 0; i < count; ++i) {
    poisson_plan_t c = nullptr;
    const poisson_status s = poisson_plan_create(&descs[i], &c);
    if (s != PS_OK) {
      pp::destroy_batch(pl);
      delete pl;
      return s;
    }
    pl->children.push_back(c);
    total += align256(c->ws_bytes);
  }
  pl->ws_bytes = total;
  pl->ws = nullptr;
  pl->launches = 0;
  pl->nev = 0;
  pl->precision = -1;
  *out = pl;
  return PS_OK;
}

poisson_status poisson_solve_batched(poisson_plan_t pl, const void* const* rhs, void* const* p, void* stream) {
  if (!pl || !rhs || !p || pl->children.empty()) return PS_EINVAL;
  if (!pl->ws) return PS_ENOWORKSPACE;
  const int n = (int)pl->children.size();
  for (int i = 0; i < n; ++i) {
    if (!rhs[i] || !p[i] || ((uintptr_t)rhs[i] & 15u) || ((uintptr_t)p[i] & 15u)) return PS_EINVAL;
    if (pl->children[i]->precision == PP_FP32_REFINED && rhs[i] == p[i]) return PS_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  bool same = pl->gexec && (int)pl->g_rhs.size() == n;
  for (int i = 0; same && i < n; ++i) same = pl->g_rhs[i] == rhs[i] && pl->g_p[i] == p[i];
  if (!same) {
    drop_graph(pl);
    while ((int)pl->forks.size() < n + 1) {   // n branches + the capture stream
      cudaStream_t s;
      cudaEvent_t e;
      if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return PS_ECUDA;
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return PS_ECUDA;
      pl->forks.push_back(s);
      pl->fork_ev.push_back(e);
    }
    if (pl->fork_ev.size() < (size_t)n + 1) {
      cudaEvent_t e;
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return PS_ECUDA;
      pl->fork_ev.push_back(e);
    }
    if (!pl->warmed) {   // one plain pass: kernel attributes are set outside capture
      for (int i = 0; i < n; ++i) {
        poisson_plan_s* c = pl->children[i];
        const poisson_status s = pp::solve_on_workspace(c, c->ws, c->dt, rhs[i], p[i], st);
        if (s != PS_OK) return s;
      }
      pl->warmed = true;
    }
    // Capture on a library stream (the caller's may be the legacy default stream, which cannot
    // be captured); the graph is then launched on the caller's stream.
    cudaEvent_t e0 = pl->fork_ev[n];
    cudaStream_t cap = pl->forks[n];
    if (cudaStreamSynchronize(st) != cudaSuccess) return PS_ECUDA;
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return PS_ECUDA;
    poisson_status s = PS_OK;
    if (cudaEventRecord(e0, cap) != cudaSuccess) s = PS_ECUDA;
    for (int i = 0; s == PS_OK && i < n; ++i) {
      poisson_plan_s* c = pl->children[i];
      cudaStream_t fs = pl->forks[i];
      if (cudaStreamWaitEvent(fs, e0, 0) != cudaSuccess) { s = PS_ECUDA; break; }
      s = pp::solve_on_workspace(c, c->ws, c->dt, rhs[i], p[i], fs);
      if (s != PS_OK) break;
      if (cudaEventRecord(pl->fork_ev[i], fs) != cudaSuccess || cudaStreamWaitEvent(cap, pl->fork_ev[i], 0) != cudaSuccess)
        s = PS_ECUDA;
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(cap, &graph);
    if (s != PS_OK || ec != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return s != PS_OK ? s : PS_ECUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(&pl->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      pl->gexec = nullptr;
      return PS_ECUDA;
    }
    pl->g_rhs.assign(rhs, rhs + n);
    pl->g_p.assign(p, p + n);
  }
  int launches = 0;
  for (poisson_plan_s* c : pl->children) launches += c->launches;
  pl->launches = launches;
  return cudaGraphLaunch(pl->gexec, st) == cudaSuccess ? PS_OK : PS_ECUDA;
}

poisson_status poisson_autotune(const poisson_desc* desc, void* stream, int* pdd_parts, unsigned* flags, float* ms) {
  if (!desc || !pdd_parts || !flags) return PS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int> cands{1};
  for (int P = 2; P <= 256; ++P) {
    if (desc->ny % P) continue;
    const bool factored = P <= 32 && desc->ny / P >= 4;
    const bool reg = desc->precision != PP_FP64 && pp::reg_tridiag_ok(desc->ny, P);
    if (factored || reg) cands.push_back(P);
  }
  const size_t cells = (size_t)desc->nx * desc->ny * desc->nz;
  const size_t es = desc->precision == PP_FP32 ? 4 : 8;
  unsigned char* io = nullptr;
  if (cudaMalloc(&io, 2 * cells * es + 512) != cudaSuccess) return PS_ECUDA;
  cudaMemsetAsync(io, 0, 2 * cells * es + 512, st);
  void* rhs = io;
  void* out = io + align256(cells * es);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = -1.f;
  int bestP = cands[0];
  unsigned bestF = 0;
  poisson_status status = PS_OK;
  for (int tiling = 0; tiling < 2 && status == PS_OK; ++tiling) {
    for (int P : cands) {
      poisson_desc d = *desc;
      d.tridiag = P == 1 ? PT_THOMAS : PT_PDD_EXACT;
      d.pdd_parts = P;
      d.flags = (desc->flags & ~(POISSON_GENERIC_FFT | POISSON_TIMING)) | (tiling ? POISSON_GENERIC_FFT : 0u);
      poisson_plan_t pl = nullptr;
      if (poisson_plan_create(&d, &pl) != PS_OK) continue;
      size_t bytes = 0;
      poisson_workspace_size(pl, &bytes);
      void* ws = nullptr;
      if (cudaMalloc(&ws, bytes) != cudaSuccess) {
        poisson_plan_destroy(pl);
        status = PS_ECUDA;
        break;
      }
      float t = -1.f;
      if (poisson_set_workspace(pl, ws, bytes, stream) == PS_OK && poisson_solve(pl, rhs, out, stream) == PS_OK) {
        const int reps = 3;
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps; ++r) poisson_solve(pl, rhs, out, stream);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) == cudaSuccess) {
          cudaEventElapsedTime(&t, e0, e1);
          t /= reps;
        }
      }
      cudaStreamSynchronize(st);
      cudaFree(ws);
      poisson_plan_destroy(pl);
      if (t >= 0.f && (best < 0.f || t < best)) {
        best = t;
        bestP = P;
        bestF = tiling ? POISSON_GENERIC_FFT : 0u;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(io);
  if (status != PS_OK) return status;
  if (best < 0.f) return PS_EUNSUPPORTED;
  *pdd_parts = bestP;
  *flags = bestF;
  if (ms) *ms = best;
  return PS_OK;
}

}  // extern "C"
