// Many independent FP32 solves of uneven sizes in ONE persistent launch.
//
// The work of a batch is a list of items (instance, pass, tile) over the passes of the FP32 solve
// (Sec. 3.2 steps (2)-(8)): forward x-transform tiles, forward z-transform tiles, PDD tiles (Sec.
// 2.2), one item for the FP64 low modes and the (0, 0) mode, inverse z- and x-transform tiles.  The
// list is ordered pass by pass (all instances' tiles of one pass before the next pass), and a
// resident grid of CTAs takes items in list order from an atomic ticket.  An item of pass p of
// instance i first waits (one thread, acquire loads) until every tile of pass p-1 of instance i
// has been counted done; a CTA only ever waits for items with smaller tickets, which are held by
// running CTAs or finished, so the launch cannot deadlock.  Each wait is bounded (about a second of
// clock cycles): when it runs out the CTA writes PS_ETIMEOUT into the batch's status word and
// raises an abort flag that makes every CTA return at its next wait or ticket.  A finished item is
// published by a barrier, a fence and an atomic increment of its (instance, pass) counter.
//
// The tile functions are those of the standalone kernels (z_reg.cuh, k_fft_x_reg.cuh,
// tridiag_scan.cuh), specialised for the batch sizes Nx/2 in {32, 48, 64, 96, 128, 192}, Nz in
// {64, 96, 128, 192, 256, 384} and PDD blocks of {2, 3, 4, 6, 8, 12, 16, 24} rows (P a power of two
// <= 32); other batches run as a graph of per-instance kernel branches (batch.cu).
#include "batch_persistent.h"
#include "k_fft_x_reg.cuh"
#include "tridiag_scan.cuh"
#include "z_reg.cuh"

namespace pp {

namespace {

constexpr int kBatchM[] = {32, 48, 64, 96, 128, 192};
constexpr int kBatchNz[] = {64, 96, 128, 192, 256, 384};
constexpr int kBatchRows[] = {2, 3, 4, 6, 8, 12, 16};

template <int N>
int index_of(const int (&a)[N], int v) {
  for (int i = 0; i < N; ++i)
    if (a[i] == v) return i;
  return -1;
}

constexpr int cmax(int a, int b) { return a > b ? a : b; }

constexpr int scan_smem_bytes(int m) {   // P * (m S + 1) float2 + 2 P (m | 1) floats, S = 256 / P, worst P
  int worst = 0;
  for (int P = 1; P <= 32; P *= 2) {
    const int S = 256 / P;
    const int b = P * (m * S + 1) * 8 + 2 * P * (m | 1) * 4;
    worst = cmax(worst, b);
  }
  return worst;
}

constexpr int batch_smem() {
  int s = 0;
  s = cmax(s, XReg<32>::SMEM); s = cmax(s, XReg<48>::SMEM); s = cmax(s, XReg<64>::SMEM);
  s = cmax(s, XReg<96>::SMEM); s = cmax(s, XReg<128>::SMEM); s = cmax(s, XReg<192>::SMEM);
  s = cmax(s, ZReg<float, 64>::SMEM); s = cmax(s, ZReg<float, 96>::SMEM); s = cmax(s, ZReg<float, 128>::SMEM);
  s = cmax(s, ZReg<float, 192>::SMEM); s = cmax(s, ZReg<float, 256>::SMEM); s = cmax(s, ZReg<float, 384>::SMEM);
  for (int m : kBatchRows) s = cmax(s, scan_smem_bytes(m));
  s = cmax(s, 2 * 256 * 8);   // the (0, 0) mode's work area (ny <= 256)
  return s;
}
constexpr int kBatchSmem = batch_smem();
constexpr int kBatchThreads = 256;

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Bounded wait (thread 0) for *ctr >= target: false when the abort flag rises or about a second
// of clock cycles (2^31 at ~2 GHz; at most 2^22 polls) has passed.
__device__ bool wait_count(const unsigned* ctr, unsigned target, const unsigned* abort_flag) {
  const long long t0 = clock64();
  unsigned ns = 64;
  for (int it = 0; it < (1 << 22); ++it) {
    if (ld_acquire(ctr) >= target) return true;
    if (ld_acquire(abort_flag)) return false;
    if (clock64() - t0 > (1LL << 31)) return false;
    __nanosleep(ns);
    if (ns < 1024) ns *= 2;
  }
  return false;
}

// FP64 low modes (|kx|, |kz| <= L, not (0, 0)) of one instance: one thread per system, the Thomas
// algorithm with the margin recurrence e_j = sigma + a_j e_{j-1} / beta_{j-1}, beta_j = c_j + e_j
// on the FP32 spectrum's values, forward values and pivots kept in FP64 scratch.
__device__ __forceinline__ void low_modes(const BatchInst& in, int q) {
  const Geometry& g = in.g;
  const int L = in.low, nl = 2 * L + 1;
  if (L < 0 || q >= (L + 1) * nl) return;
  const int kx = q / nl, r = q - kx * nl;
  const int kz = r <= L ? r : g.nz - (r - L);
  if (kx > g.M || (kx == 0 && kz == 0) || kz < 0 || kz >= g.nz) return;
  const double* a = in.dt.d.a;
  const double* c = in.dt.d.c;
  const double sigma = -(in.dt.lamx[kx] + in.dt.lamz[kz]);
  const size_t rstride = (size_t)g.nz * g.pitch;
  cplx<float>* col = in.spec + (size_t)kz * g.pitch + kx;
  const int nlow = (L + 1) * nl;
  double e = sigma, rbp = 0.0, yr = 0.0, yi = 0.0;
  for (int j = 0; j < g.ny; ++j) {
    if (j > 0) e = sigma + a[j] * e * rbp;
    const double rb = 1.0 / (c[j] + e);
    const cplx<float> F = ld_c_cg(col + (size_t)j * rstride);
    yr = (-(double)F.x + a[j] * yr) * rb;
    yi = (-(double)F.y + a[j] * yi) * rb;
    in.low_piv[(size_t)j * nlow + q] = rb;
    in.low_y[(size_t)j * nlow + q] = mk<double>(yr, yi);
    rbp = rb;
  }
  double xr = yr, xi = yi;
  st_c(col + (size_t)(g.ny - 1) * rstride, mk<float>(float(xr), float(xi)));
  for (int j = g.ny - 2; j >= 0; --j) {
    const double cr = c[j] * in.low_piv[(size_t)j * nlow + q];
    const cplx<double> y = in.low_y[(size_t)j * nlow + q];
    xr = y.x + cr * xr;
    xi = y.y + cr * xi;
    st_c(col + (size_t)j * rstride, mk<float>(float(xr), float(xi)));
  }
}

#define PP_SEL_M(F) F(0, 32) F(1, 48) F(2, 64) F(3, 96) F(4, 128) F(5, 192)
#define PP_SEL_NZ(F) F(0, 64) F(1, 96) F(2, 128) F(3, 192) F(4, 256) F(5, 384)
#define PP_SEL_ROWS(F) F(0, 2) F(1, 3) F(2, 4) F(3, 6) F(4, 8) F(5, 12) F(6, 16)

__device__ __forceinline__ void run_item(const BatchInst& in, int pass, int tile, unsigned char* smem) {
  const Geometry& g = in.g;
  switch (pass) {
    case BP_XF: {
      FwdArgs args = {};
      args.in = in.rhs;
      args.in_scale = 1.0;
      const int nlines = g.ny * g.nz;
      switch (in.xsel) {
#define PP_XF(I, MV) \
        case I: fwd_x_reg_tile<float, MV, FWD_PLAIN>(g, args, in.dt.f, in.dt, in.spec, nlines, tile, smem); break;
        PP_SEL_M(PP_XF)
#undef PP_XF
      }
      break;
    }
    case BP_ZF:
    case BP_ZI: {
      const int bx = tile % in.zcols, j = tile / in.zcols;
      switch (in.zsel) {
#define PP_Z(I, NZV)                                                                              \
        case I:                                                                                   \
          if (pass == BP_ZF) z_reg_tile<float, NZV, -1>(g, in.dt.f, in.spec, 0, g.ncols, bx, j, smem); \
          else z_reg_tile<float, NZV, 1>(g, in.dt.f, in.spec, 0, g.ncols, bx, j, smem);            \
          break;
        PP_SEL_NZ(PP_Z)
#undef PP_Z
      }
      break;
    }
    case BP_TRI: {
      const int S = reg_systems_per_cta(in.parts);
      switch (in.msel) {
#define PP_T(I, MM)                                                                                          \
        case I:                                                                                              \
          tridiag_scan_tile<MM>(g, in.parts, S, in.low, in.dt.f.a, in.dt.f.c, in.dt.lamx, in.dt.lamz, in.dt.red_f, \
                                in.spec, 0, g.ncols, tile, smem);                                            \
          break;
        PP_SEL_ROWS(PP_T)
#undef PP_T
      }
      break;
    }
    case BP_LOW: {
      if (threadIdx.x < 32) mode00_warp<float>(g, in.dt.dy, in.dt.h, in.spec, in.dt.acc, GAUGE_ZERO,
                                               reinterpret_cast<double*>(smem));
      else low_modes(in, threadIdx.x - 32);
      break;
    }
    case BP_XI: {
      const int nlines = g.ny * g.nz;
      const double scale = 1.0 / ((double)g.nx * (double)g.nz);
      switch (in.xsel) {
#define PP_XI(I, MV)                                                                                      \
        case I:                                                                                           \
          inv_x_reg_tile<float, MV, INV_STORE, false>(g, in.dt.f, in.spec, in.out, scale, nlines, in.dt.dy, \
                                                      in.dt.acc, PairArgs{nullptr, nullptr}, tile, smem); \
          break;
        PP_SEL_M(PP_XI)
#undef PP_XI
      }
      break;
    }
  }
}

// Four CTAs per SM (64 registers per thread): the kernel holds every tile kind, so its register
// budget sets the occupancy of all of them; 4 CTAs/SM measured 3.4 ms on the 64-instance batch
// against 6.0 / 4.1 / 3.4 ms at 1 / 2 / 3 CTAs/SM (the spills cost less than the lost warps).
__global__ void __launch_bounds__(kBatchThreads, 4)
    k_batch_persistent(const BatchInst* __restrict__ inst, const BatchItem* __restrict__ items, int nitems,
                       BatchCtl* ctl, int* status, int selftest) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_item;
  __shared__ __align__(16) BatchInst s_inst;   // the current item's instance record
  // thread 0 holds the next ticket while the CTA works on the current item, so the atomic's latency
  // is hidden (a CTA holding two tickets still only ever waits on smaller ones)
  int next = threadIdx.x == 0 ? (int)atomicAdd(&ctl->ticket, 1u) : 0;
  for (;;) {
    if (threadIdx.x == 0) {
      int t = next;
      if (t >= nitems || ld_acquire(&ctl->abort)) {
        t = -1;
      } else {
        next = (int)atomicAdd(&ctl->ticket, 1u);
        const BatchItem it = items[t];
        if (it.pass > 0) {
          const unsigned need = (unsigned)inst[it.inst].ntiles[it.pass - 1];
          if (!wait_count(&ctl->done[it.inst * BP_N + it.pass - 1], need, &ctl->abort)) {
            if (!ld_acquire(&ctl->abort)) {   // this CTA's own wait ran out (not a propagated abort)
              atomicExch(status, (int)DEV_TIMEOUT);
              atomicExch(&ctl->abort, 1u);
            }
            t = -1;
          }
        }
      }
      s_item = t;
    }
    __syncthreads();
    const int t = s_item;
    if (t < 0) break;
    const BatchItem it = items[t];
    {
      const int* src = reinterpret_cast<const int*>(inst + it.inst);
      int* dst = reinterpret_cast<int*>(&s_inst);
      for (int k = threadIdx.x; k < (int)(sizeof(BatchInst) / sizeof(int)); k += blockDim.x) dst[k] = src[k];
    }
    __syncthreads();
    for (int k = 0; k < it.count; ++k) {
      run_item(s_inst, it.pass, it.tile + k, smem);
      __syncthreads();   // stores issued and shared memory free before the next tile or the count
    }
    if (threadIdx.x == 0) {
      // POISSON_SELFTEST_WAIT: the first x-transform item of instance 0 is never counted, so the
      // waits of that instance's next pass run out
      const bool skip = selftest && it.inst == 0 && it.pass == BP_XF && it.tile == 0;
      if (!skip) {
        __threadfence();
        atomicAdd(&ctl->done[it.inst * BP_N + it.pass], (unsigned)it.count);
      }
    }
  }
}

}  // namespace

int batch_persistent_smem() { return kBatchSmem; }

// Selectors of the specialised tile functions for one instance (false: not supported here).
bool batch_persistent_ok(const poisson_plan_s* c, int& xsel, int& zsel, int& msel) {
  if (c->precision != PP_FP32 || c->has_tri || c->g.generic_fft) return false;
  if (!scan_tridiag_ok(c->g.ny, c->parts) || c->g.ny > 256) return false;
  xsel = index_of(kBatchM, c->g.M);
  zsel = index_of(kBatchNz, c->g.nz);
  msel = index_of(kBatchRows, c->g.ny / c->parts);
  if (c->low >= 0 && (c->low + 1) * (2 * c->low + 1) > kBatchThreads - 32) return false;
  return xsel >= 0 && zsel >= 0 && msel >= 0;
}

// Tile counts of each pass of an instance (the grids of the standalone kernels).
void batch_tiles(const poisson_plan_s* c, int zcols, int ntiles[BP_N]) {
  const Geometry& g = c->g;
  int lpb = 0;
  switch (g.M) {
#define PP_L(I, MV) \
    case MV: lpb = XReg<MV>::LPB; break;
    PP_SEL_M(PP_L)
#undef PP_L
  }
  const int nlines = g.ny * g.nz;
  const int S = reg_systems_per_cta(c->parts);
  ntiles[BP_XF] = (nlines + lpb - 1) / lpb;
  ntiles[BP_ZF] = zcols * g.ny;
  ntiles[BP_TRI] = g.nz * ((g.ncols + S - 1) / S);
  ntiles[BP_LOW] = 1;
  ntiles[BP_ZI] = ntiles[BP_ZF];
  ntiles[BP_XI] = ntiles[BP_XF];
}

// Tiles per work item of a pass: enough that an item moves about 2 MB, so that the per-item cost
// of the queue (ticket, acquire, barriers, release) stays small against the tile work (measured:
// 4.7 / 4.2 / 4.1 ms for 128 KB / 512 KB / 2 MB items on the 64-instance batch).
int batch_group(const poisson_plan_s* c, int pass, int zcols) {
  const Geometry& g = c->g;
  size_t bytes = 0;
  int lpb = 1;
  switch (g.M) {
#define PP_L(I, MV) \
    case MV: lpb = XReg<MV>::LPB; break;
    PP_SEL_M(PP_L)
#undef PP_L
  }
  const int wz = (g.ncols + zcols - 1) / zcols;
  const int S = reg_systems_per_cta(c->parts);
  switch (pass) {
    case BP_XF: case BP_XI: bytes = (size_t)lpb * (4 * g.nx + 8 * (g.M + 1)); break;
    case BP_ZF: case BP_ZI: bytes = (size_t)16 * wz * g.nz; break;
    case BP_TRI: bytes = (size_t)16 * S * g.ny; break;
    default: return 1;
  }
  const size_t target = (size_t)2 << 20;
  const int grp = (int)((target + bytes - 1) / bytes);
  return grp < 1 ? 1 : (grp > 256 ? 256 : grp);
}

int batch_zcols(const poisson_plan_s* c) {
  const int w = fft_z_fast_tile<float>(c->g);
  return (c->g.ncols + w - 1) / w;
}

cudaError_t launch_batch_persistent(const BatchInst* inst, const BatchItem* items, int nitems, BatchCtl* ctl,
                                    size_t ctl_bytes, int* status, int selftest, cudaStream_t st) {
  cudaError_t e = ensure_smem_limit((const void*)k_batch_persistent, (size_t)kBatchSmem);
  if (e != cudaSuccess) return e;
  static int grid = 0;
  if (!grid) {
    int dev = 0, sms = 0, per = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_persistent, kBatchThreads,
                                                           (size_t)kBatchSmem)) != cudaSuccess)
      return e;
    if (per < 1) return cudaErrorInvalidConfiguration;
    grid = sms * per;
  }
  if ((e = cudaMemsetAsync(ctl, 0, ctl_bytes, st)) != cudaSuccess) return e;
  k_batch_persistent<<<grid, kBatchThreads, kBatchSmem, st>>>(inst, items, nitems, ctl, status, selftest);
  return cudaGetLastError();
}

}  // namespace pp
