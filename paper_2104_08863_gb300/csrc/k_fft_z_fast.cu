// Specialised z-transform kernel (step (4) / (6) of Sec. 3.2): a CTA transforms a tile of W
// adjacent kx columns of one y-plane along z (Nz points each).  The tile is loaded with
// coalesced row segments of W complex values, transformed in place in (padded) shared memory
// by the compile-time Stockham engine, and stored back.  W and the thread count are chosen so
// that each thread stages 16 (FP32) or 8 (FP64) complex values per stage, which keeps two
// CTAs resident per SM so that one CTA's loads overlap the other's arithmetic.  A launch may
// cover only the kx columns [kx_lo, kx_hi) (one slab of the spectrum; kx_lo a multiple of W).
#include "fft_static.cuh"
#include "internal.h"
#include "z_reg.cuh"

namespace pp {

template <typename T, int NZ> struct ZTile {
  static constexpr int E = sizeof(T) == 4 ? 16 : 8;               // complex values per thread
  static constexpr int WMIN = sizeof(T) == 4 ? 8 : 4;             // 64-byte row segments
  static constexpr int W0 = (E * 512) / NZ;
  static constexpr int W = W0 < WMIN ? WMIN : (W0 > 32 ? 32 : W0);
  static constexpr int T0 = W * NZ / E;
  static constexpr int THREADS = T0 < 64 ? 64 : (T0 > 512 ? 512 : T0);
  static constexpr int SMEM = padded_size<T>(W * NZ) * (int)sizeof(cplx<T>);
  static constexpr int MINB = 2;   // two CTAs per SM so one CTA's memory phase overlaps the other's math
};

template <typename T, int NZ, int SIGN>
__global__ void __launch_bounds__(ZTile<T, NZ>::THREADS, ZTile<T, NZ>::MINB) k_fft_z_fast(Geometry g, Tables<T> tt,
                                                                       cplx<T>* __restrict__ spec, int kx_lo,
                                                                       int kx_hi) {
  using C = ZTile<T, NZ>;
  constexpr int W = C::W, THREADS = C::THREADS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
  const int j = blockIdx.y;
  const int kx0 = kx_lo + blockIdx.x * W;
  cplx<T>* plane = spec + (size_t)j * NZ * g.pitch + kx0;
  const int ncol = min(W, kx_hi - kx0);
  {
    // every load of the thread is issued before its first shared-memory store
    constexpr int PER = (NZ * W + THREADS - 1) / THREADS;
    cplx<T> v[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int idx = threadIdx.x + q * THREADS;
      const int n = idx / W, c = idx % W;
      v[q] = (idx < NZ * W && c < ncol) ? ld_c(plane + (size_t)n * g.pitch + c) : mk<T>(T(0), T(0));
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int idx = threadIdx.x + q * THREADS;
      if (idx < NZ * W) buf[padi<T>(idx)] = v[q];
    }
  }
  __syncthreads();
  fft_static<T, NZ, SIGN, W, THREADS, W, 1, true>(buf, tt.tw_z);
#pragma unroll 4
  for (int idx = threadIdx.x; idx < NZ * W; idx += THREADS) {
    const int n = idx / W, c = idx % W;
    if (c < ncol) st_c(plane + (size_t)n * g.pitch + c, buf[padi<T>(idx)]);
  }
}

template <typename K>
static cudaError_t set_smem_once(K kernel, int smem) {
  return ensure_smem_limit((const void*)kernel, (size_t)smem);
}

template <typename T, int NZ>
static cudaError_t launch_z_reg(const Geometry& g, const Tables<T>& tt, int sign, cplx<T>* spec, cudaStream_t st,
                                int kx_lo, int kx_hi) {
  using C = ZReg<T, NZ>;
  if (kx_lo % C::W || kx_lo < 0 || kx_hi > g.ncols || kx_hi <= kx_lo) return cudaErrorInvalidValue;
  const dim3 grid((kx_hi - kx_lo + C::W - 1) / C::W, g.ny);
  cudaError_t e;
  if (sign < 0) {
    auto k = k_fft_z_reg<T, NZ, -1>;
    if ((e = set_smem_once(k, C::SMEM)) != cudaSuccess) return e;
    k<<<grid, C::THREADS, C::SMEM, st>>>(g, tt, spec, kx_lo, kx_hi);
  } else {
    auto k = k_fft_z_reg<T, NZ, 1>;
    if ((e = set_smem_once(k, C::SMEM)) != cudaSuccess) return e;
    k<<<grid, C::THREADS, C::SMEM, st>>>(g, tt, spec, kx_lo, kx_hi);
  }
  return cudaGetLastError();
}

template <typename T, int NZ>
static cudaError_t launch_z(const Geometry& g, const Tables<T>& tt, int sign, cplx<T>* spec, cudaStream_t st,
                            int kx_lo, int kx_hi) {
  if constexpr (sizeof(T) == 4) return launch_z_reg<T, NZ>(g, tt, sign, spec, st, kx_lo, kx_hi);
  using C = ZTile<T, NZ>;
  if (kx_lo % C::W || kx_lo < 0 || kx_hi > g.ncols || kx_hi <= kx_lo) return cudaErrorInvalidValue;
  const dim3 grid((kx_hi - kx_lo + C::W - 1) / C::W, g.ny);
  cudaError_t e;
  if (sign < 0) {
    auto k = k_fft_z_fast<T, NZ, -1>;
    if ((e = set_smem_once(k, C::SMEM)) != cudaSuccess) return e;
    k<<<grid, C::THREADS, C::SMEM, st>>>(g, tt, spec, kx_lo, kx_hi);
  } else {
    auto k = k_fft_z_fast<T, NZ, 1>;
    if ((e = set_smem_once(k, C::SMEM)) != cudaSuccess) return e;
    k<<<grid, C::THREADS, C::SMEM, st>>>(g, tt, spec, kx_lo, kx_hi);
  }
  return cudaGetLastError();
}

// Returns cudaErrorNotSupported when Nz has no specialisation (the caller then uses the
// generic kernel).  kx_hi < 0 means all columns.
template <typename T>
cudaError_t launch_fft_z_fast(const Geometry& g, const Tables<T>& tt, int sign, cplx<T>* spec, cudaStream_t st,
                              int kx_lo, int kx_hi) {
  if (kx_hi < 0) kx_hi = g.ncols;
  switch (g.nz) {
#define PP_Z_CASE(NZ) \
    case NZ: return launch_z<T, NZ>(g, tt, sign, spec, st, kx_lo, kx_hi);
    PP_Z_CASE(16) PP_Z_CASE(32) PP_Z_CASE(48) PP_Z_CASE(64) PP_Z_CASE(96) PP_Z_CASE(128) PP_Z_CASE(192)
    PP_Z_CASE(256) PP_Z_CASE(384) PP_Z_CASE(512) PP_Z_CASE(768) PP_Z_CASE(1024)
#undef PP_Z_CASE
    default: return cudaErrorNotSupported;
  }
}

// Column width of the specialised z tile for this Nz (0 when Nz has no specialisation).
template <typename T>
int fft_z_fast_tile(const Geometry& g) {
  switch (g.nz) {
#define PP_ZW_CASE(NZ) \
    case NZ: return sizeof(T) == 4 ? ZReg<T, NZ>::W : ZTile<T, NZ>::W;
    PP_ZW_CASE(16) PP_ZW_CASE(32) PP_ZW_CASE(48) PP_ZW_CASE(64) PP_ZW_CASE(96) PP_ZW_CASE(128) PP_ZW_CASE(192)
    PP_ZW_CASE(256) PP_ZW_CASE(384) PP_ZW_CASE(512) PP_ZW_CASE(768) PP_ZW_CASE(1024)
#undef PP_ZW_CASE
    default: return 0;
  }
}

template cudaError_t launch_fft_z_fast<float>(const Geometry&, const Tables<float>&, int, cplx<float>*, cudaStream_t,
                                              int, int);
template cudaError_t launch_fft_z_fast<double>(const Geometry&, const Tables<double>&, int, cplx<double>*,
                                               cudaStream_t, int, int);
template int fft_z_fast_tile<float>(const Geometry&);
template int fft_z_fast_tile<double>(const Geometry&);

}  // namespace pp
