// Batched solves of independent, uneven-size problems in one graph launch, and the autotuner.
//
// A batched plan holds one sub-plan per instance and carves their workspaces out of one caller
// allocation.  poisson_solve_batched captures, once, a CUDA graph and replays it while the
// pointers stay the same.  The graph holds either one branch per instance, forked from the
// caller's stream and holding that instance's kernel sequence (the same pipeline as
// poisson_solve), so that small instances run concurrently and the host pays one graph launch
// per batch instead of ~7 launches per instance; or (POISSON_BATCH_PERSISTENT, every instance
// supported) one persistent kernel over a device work list (batch_persistent.cu).
//
// poisson_autotune picks, per grid, the PDD partition count and the FFT tiling (compile-time
// specialised or generic kernels) by timing the actual solve on the device.
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "batch_persistent.h"
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

// Instance table and work list of the persistent launch, built once per workspace.  Items are
// ordered pass by pass; within a pass the instances go largest first.
static poisson_status build_persistent(poisson_plan_s* pl, unsigned char* ws, cudaStream_t st) {
  const int n = (int)pl->children.size();
  std::vector<BatchInst> inst(n);
  std::vector<int> order(n);
  size_t lowoff = pl->off_lowscr;
  for (int i = 0; i < n; ++i) {
    poisson_plan_s* c = pl->children[i];
    BatchInst& b = inst[i];
    memset(&b, 0, sizeof(b));
    b.g = c->g;
    b.dt = c->dt;
    b.spec = (cplx<float>*)(c->ws + c->off_spec);
    b.parts = c->parts;
    b.low = c->low;
    if (!batch_persistent_ok(c, b.xsel, b.zsel, b.msel)) return PS_EUNSUPPORTED;
    b.zcols = batch_zcols(c);
    batch_tiles(c, b.zcols, b.ntiles);
    const size_t nlow = c->low >= 0 ? (size_t)(c->low + 1) * (2 * c->low + 1) : 0;
    b.low_piv = (double*)(ws + lowoff);
    lowoff = align256(lowoff + 8 * nlow * c->g.ny);
    b.low_y = (cplx<double>*)(ws + lowoff);
    lowoff = align256(lowoff + 16 * nlow * c->g.ny);
    order[i] = i;
  }
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    const size_t px = (size_t)inst[x].g.nx * inst[x].g.ny * inst[x].g.nz;
    const size_t py = (size_t)inst[y].g.nx * inst[y].g.ny * inst[y].g.nz;
    return px > py;
  });
  std::vector<BatchItem> items;
  for (int pass = 0; pass < BP_N; ++pass)
    for (int i : order) {
      const int grp = batch_group(pl->children[i], pass, inst[i].zcols);
      for (int t = 0; t < inst[i].ntiles[pass]; t += grp)
        items.push_back(BatchItem{i, pass, t, std::min(grp, inst[i].ntiles[pass] - t)});
    }
  pl->nitems = (int)items.size();
  pl->inst_host.assign((unsigned char*)inst.data(), (unsigned char*)inst.data() + n * sizeof(BatchInst));
  if (cudaMemcpyAsync(ws + pl->off_items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice,
                      st) != cudaSuccess)
    return PS_ECUDA;
  if (cudaMemsetAsync(ws + pl->off_bstatus, 0, 256, st) != cudaSuccess) return PS_ECUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? PS_OK : PS_ECUDA;
}

poisson_status set_batch_workspace(poisson_plan_s* pl, unsigned char* ws, void* stream) {
  size_t off = 0;
  for (poisson_plan_s* c : pl->children) {
    const poisson_status s = poisson_set_workspace(c, ws + off, c->ws_bytes, stream);
    if (s != PS_OK) return s;
    off += align256(c->ws_bytes);
  }
  pl->ws = ws;
  pl->dt = DevTables{};
  pl->dt.status = (int*)(ws + pl->off_bstatus);
  drop_graph(pl);
  pl->warmed = false;
  if (cudaMemsetAsync(ws + pl->off_bstatus, 0, 256, (cudaStream_t)stream) != cudaSuccess) return PS_ECUDA;
  if (pl->persistent) return build_persistent(pl, ws, (cudaStream_t)stream);
  return cudaStreamSynchronize((cudaStream_t)stream) == cudaSuccess ? PS_OK : PS_ECUDA;
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
  const bool branches = (descs[0].flags & POISSON_BATCH_PERSISTENT) == 0;
  for (int i = 0; i < count; ++i) {
    poisson_desc d = descs[i];
    // the persistent launch's PDD tiles take blocks of at most 16 rows (register budget): an
    // automatic partition becomes the smallest power of two P <= 32 with ny / P <= 16
    if (!branches && d.precision == PP_FP32 && d.pdd_parts == 0 && d.tridiag == PT_AUTO) {
      for (int P = 1; P <= 32; P *= 2)
        if (d.ny % P == 0 && d.ny / P <= 16 && pp::reg_tridiag_ok(d.ny, P)) {
          d.pdd_parts = P;
          d.tridiag = P == 1 ? PT_THOMAS : PT_PDD_EXACT;
          break;
        }
    }
    poisson_plan_t c = nullptr;
    const poisson_status s = poisson_plan_create(&d, &c);
    if (s != PS_OK) {
      pp::destroy_batch(pl);
      delete pl;
      return s;
    }
    pl->children.push_back(c);
    total += align256(c->ws_bytes);
  }
  // the batch's own regions after the instances' workspaces: status word, then (persistent
  // launch) the instance table, the work list, the control block and the low modes' scratch
  pl->off_bstatus = total;
  total += 256;
  bool ok = !branches;
  size_t nitems = 0, lowscr = 0;
  for (int i = 0; ok && i < count; ++i) {
    poisson_plan_s* c = pl->children[i];
    int xs, zs, ms;
    if (!pp::batch_persistent_ok(c, xs, zs, ms)) {
      ok = false;
      break;
    }
    int nt[pp::BP_N];
    pp::batch_tiles(c, pp::batch_zcols(c), nt);
    for (int k = 0; k < pp::BP_N; ++k) nitems += (size_t)nt[k];
    const size_t nlow = c->low >= 0 ? (size_t)(c->low + 1) * (2 * c->low + 1) : 0;
    lowscr += align256(8 * nlow * c->g.ny) + align256(16 * nlow * c->g.ny);
  }
  if (ok && nitems < (size_t)1 << 30) {
    pl->persistent = true;
    pl->selftest = (descs[0].flags & POISSON_SELFTEST_WAIT) != 0;
    pl->off_inst = total;
    total += align256((size_t)count * sizeof(pp::BatchInst));
    pl->off_items = total;
    total += align256(nitems * sizeof(pp::BatchItem));
    pl->off_ctl = total;
    pl->ctl_bytes = sizeof(pp::BatchCtl) + sizeof(unsigned) * ((size_t)count * pp::BP_N);
    total += align256(pl->ctl_bytes);
    pl->off_lowscr = total;
    total += lowscr;
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
  if (pl->persistent) {
    if (!same) {
      drop_graph(pl);
      if (pl->forks.empty()) {
        cudaStream_t s;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return PS_ECUDA;
        pl->forks.push_back(s);
      }
      pp::BatchInst* inst = (pp::BatchInst*)pl->inst_host.data();
      for (int i = 0; i < n; ++i) {
        inst[i].rhs = (const float*)rhs[i];
        inst[i].out = (float*)p[i];
      }
      unsigned char* ws = pl->ws;
      if (cudaMemcpyAsync(ws + pl->off_inst, pl->inst_host.data(), pl->inst_host.size(), cudaMemcpyHostToDevice,
                          st) != cudaSuccess)
        return PS_ECUDA;
      auto launch = [&](cudaStream_t s) {
        return pp::launch_batch_persistent((const pp::BatchInst*)(ws + pl->off_inst),
                                           (const pp::BatchItem*)(ws + pl->off_items), pl->nitems,
                                           (pp::BatchCtl*)(ws + pl->off_ctl), pl->ctl_bytes,
                                           (int*)(ws + pl->off_bstatus), pl->selftest ? 1 : 0, s);
      };
      if (!pl->warmed) {   // one plain launch: kernel attributes and the grid size are set outside capture
        if (launch(st) != cudaSuccess) return PS_ECUDA;
        pl->warmed = true;
      }
      if (cudaStreamSynchronize(st) != cudaSuccess) return PS_ECUDA;
      cudaStream_t cap = pl->forks[0];
      if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return PS_ECUDA;
      const cudaError_t el = launch(cap);
      cudaGraph_t graph = nullptr;
      const cudaError_t ec = cudaStreamEndCapture(cap, &graph);
      if (el != cudaSuccess || ec != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return PS_ECUDA;
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
    pl->launches = 1;
    return cudaGraphLaunch(pl->gexec, st) == cudaSuccess ? PS_OK : PS_ECUDA;
  }
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
