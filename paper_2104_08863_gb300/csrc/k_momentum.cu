// Momentum predictor of the fully explicit projection method (Sec. 2, Eqs. 3, 5, 6).
//
// One launch evaluates one stage of Heun's RK2 on the staggered faces:
//   out = alpha * base + beta * s + bdt * R(s),   R(s) = -N(s) + nu lap(s) + (fx, 0, 0)
// stage 1: (alpha, beta, bdt) = (0, 1, dt)       -> u_bar = u + dt R(u)
// stage 2: (alpha, beta, bdt) = (1/2, 1/2, dt/2) -> u_star = (u + u_bar + dt R(u_bar)) / 2
//                                                 = u + dt/2 (R(u) + R(u_bar))
// The advection N is the divergence form with two-point face averages: each flux through a
// face of a momentum control volume is the product of the two averaged velocities there, and the
// fluxes through the no-slip walls vanish.  The diffusion is the three-point Laplacian; the walls
// enter u and w through the wall value 0 half a cell from the first node.  v's wall faces are
// boundary values and are copied (stage 1) or left unchanged (stage 2, in place).
//
// Every flux is shared by two momentum equations: the u-v edge flux (x-face i, y-face f) is the
// y-flux of u and the x-flux of v, likewise u-w (z of u, x of w) and v-w (y of w, z of v).  A
// thread owns one (k, i) column of a (32 x 8) tile and marches up the rows of its chunk, so the
// y-fluxes and the y-neighbours roll through registers; x/z neighbours come through L1.
// Per-row coefficients (stretched y, no-slip wall rows, the stage factors) are built once per CTA
// in shared memory from the plan's FP64 metric tables.
#include "internal.h"

namespace pp {

namespace {

constexpr int MTX = 32, MTZ = 8;

template <typename T>
struct RowCoef {    // u and w rows j, v faces f = j
  T c0, ca, cc, cay;         // centre, j-1, j+1 diffusion weights; y-advection scale
  T v0, va, vc, vay;         // the same for v at face j (j = 1..ny-1)
};

template <typename T>
__device__ __forceinline__ T ld(const T* p) { return __ldg(p); }

template <typename T>
__global__ void __launch_bounds__(MTX * MTZ) k_momentum(Geometry g, MomArgs<T> a,
                                                         const double* __restrict__ inv_dy,
                                                         const double* __restrict__ inv_h,
                                                         const double* __restrict__ lo,
                                                         const double* __restrict__ up, int jlo, int jhi,
                                                         int jc) {
  extern __shared__ unsigned char smem_raw[];
  RowCoef<T>* rc = reinterpret_cast<RowCoef<T>*>(smem_raw);
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int j0 = jlo + blockIdx.z * jc;
  const int j1 = min(jhi, j0 + jc);
  const double bdtnu = a.bdt * a.nu;
  const double cdx = bdtnu / (g.dx * g.dx), cdz = bdtnu / (g.dz * g.dz);
  for (int r = threadIdx.y * MTX + threadIdx.x; r < j1 - j0; r += MTX * MTZ) {
    const int j = j0 + r;
    RowCoef<T> c;
    const double A = j > 0 ? lo[j] : 2.0 * inv_dy[0] * inv_dy[0];
    const double C = j < ny - 1 ? up[j] : 2.0 * inv_dy[ny - 1] * inv_dy[ny - 1];
    c.c0 = T(a.beta - 2.0 * cdx - 2.0 * cdz - bdtnu * (A + C));
    c.ca = T(j > 0 ? bdtnu * lo[j] : 0.0);
    c.cc = T(j < ny - 1 ? bdtnu * up[j] : 0.0);
    c.cay = T(-0.25 * a.bdt * inv_dy[j]);
    if (j >= 1) {
      const double va = bdtnu * inv_h[j] * inv_dy[j - 1], vc = bdtnu * inv_h[j] * inv_dy[j];
      c.v0 = T(a.beta - 2.0 * cdx - 2.0 * cdz - va - vc);
      c.va = T(va);
      c.vc = T(vc);
      c.vay = T(-0.25 * a.bdt * inv_h[j]);
    } else {
      c.v0 = c.va = c.vc = c.vay = T(0);
    }
    rc[r] = c;
  }
  __syncthreads();
  const int i = blockIdx.x * MTX + threadIdx.x;
  const int k = blockIdx.y * MTZ + threadIdx.y;
  if (i >= nx || k >= nz) return;
  const T cDx = T(cdx), cDz = T(cdz);
  const T cAx = T(-0.25 * a.bdt / g.dx), cAz = T(-0.25 * a.bdt / g.dz);
  const T fterm = T(a.bdt * a.fx);
  const T alpha = T(a.alpha);
  const bool has_base = a.bu != nullptr;
  const size_t plane = (size_t)nz * nx;
  const int im = i == 0 ? nx - 1 : i - 1, ip = i == nx - 1 ? 0 : i + 1;
  const int km = k == 0 ? nz - 1 : k - 1, kp = k == nz - 1 ? 0 : k + 1;
  // column offsets within a plane
  const size_t oc = (size_t)k * nx + i, oxm = (size_t)k * nx + im, oxp = (size_t)k * nx + ip;
  const size_t ozm = (size_t)km * nx + i, ozp = (size_t)kp * nx + i;
  const size_t ozm_xp = (size_t)km * nx + ip, ozp_xm = (size_t)kp * nx + im;
  const T* su = a.su;
  const T* sv = a.sv;
  const T* sw = a.sw;

  // rolling state at the chunk's first row j0
  T u_m = T(0), w_m = T(0);                 // row j-1 (0 below the wall)
  T u_c = ld(su + (size_t)j0 * plane + oc), w_c = ld(sw + (size_t)j0 * plane + oc);
  T v_m = j0 > 0 ? ld(sv + (size_t)(j0 - 1) * plane + oc) : T(0);
  T v_c = ld(sv + (size_t)j0 * plane + oc);
  T u_m_xp = T(0), w_m_zp = T(0);           // u(j-1, k, i+1), w(j-1, k+1, i)
  T e_uv = T(0), e_vw = T(0);               // fluxes through face j0 (zero on the wall)
  if (j0 > 0) {
    const size_t pm = (size_t)(j0 - 1) * plane, pc = (size_t)j0 * plane;
    u_m = ld(su + pm + oc);
    w_m = ld(sw + pm + oc);
    u_m_xp = ld(su + pm + oxp);
    w_m_zp = ld(sw + pm + ozp);
    e_uv = (ld(sv + pc + oxm) + v_c) * (u_m + u_c);
    e_vw = (ld(sv + pc + ozm) + v_c) * (w_m + w_c);
  }
  T vs_m = v_m + v_c;                       // v(j-1) + v(j): twice v at cell centre j-1

  if (j0 == 0) {   // bottom wall face of v: boundary value
    a.ov[oc] = has_base ? a.bv[oc] : v_c;
  }
  for (int j = j0; j < j1; ++j) {
    const RowCoef<T> c = rc[j - j0];
    const size_t pc = (size_t)j * plane, pn = pc + plane;
    const bool top = j + 1 < ny;
    const T u_n = top ? ld(su + pn + oc) : T(0);
    const T w_n = top ? ld(sw + pn + oc) : T(0);
    const T v_n = ld(sv + pn + oc);
    // neighbours in row j
    const T u_xm = ld(su + pc + oxm), u_xp = ld(su + pc + oxp), u_zm = ld(su + pc + ozm), u_zp = ld(su + pc + ozp);
    const T u_zm_xp = ld(su + pc + ozm_xp);
    const T w_xm = ld(sw + pc + oxm), w_xp = ld(sw + pc + oxp), w_zm = ld(sw + pc + ozm), w_zp = ld(sw + pc + ozp);
    const T w_zp_xm = ld(sw + pc + ozp_xm);
    const T v_xm = ld(sv + pc + oxm), v_xp = ld(sv + pc + oxp), v_zm = ld(sv + pc + ozm), v_zp = ld(sv + pc + ozp);
    // fluxes through face j+1 (zero on the top wall)
    const T e_uv_n = top ? (ld(sv + pn + oxm) + v_n) * (u_c + u_n) : T(0);
    const T e_vw_n = top ? (ld(sv + pn + ozm) + v_n) * (w_c + w_n) : T(0);
    // u-w edge flux at (x-face i, z-face k): z-flux of u, x-flux of w
    const T e_uw = (w_xm + w_c) * (u_zm + u_c);

    // ---- u at (j, k, i)
    {
      T acc = fterm;
      if (has_base) acc = alpha * a.bu[pc + oc] + acc;
      acc = c.c0 * u_c + acc;
      const T sx = u_xp + u_xm;
      acc = cDx * sx + acc;
      acc = cAx * ((u_xp - u_xm) * (sx + T(2) * u_c)) + acc;
      acc = cDz * (u_zp + u_zm) + acc;
      acc = cAz * ((w_zp_xm + w_zp) * (u_c + u_zp) - e_uw) + acc;
      acc = c.cay * (e_uv_n - e_uv) + acc;
      acc = c.ca * u_m + acc;
      acc = c.cc * u_n + acc;
      a.ou[pc + oc] = acc;
    }
    // ---- w at (j, k, i)
    {
      T acc = has_base ? alpha * a.bw[pc + oc] : T(0);
      acc = c.c0 * w_c + acc;
      const T sz = w_zp + w_zm;
      acc = cDz * sz + acc;
      acc = cAz * ((w_zp - w_zm) * (sz + T(2) * w_c)) + acc;
      acc = cDx * (w_xp + w_xm) + acc;
      acc = cAx * ((w_c + w_xp) * (u_zm_xp + u_xp) - e_uw) + acc;
      acc = c.cay * (e_vw_n - e_vw) + acc;
      acc = c.ca * w_m + acc;
      acc = c.cc * w_n + acc;
      a.ow[pc + oc] = acc;
    }
    // ---- v at face j (interior faces only)
    if (j >= 1) {
      T acc = has_base ? alpha * a.bv[pc + oc] : T(0);
      acc = c.v0 * v_c + acc;
      const T vs = v_c + v_n;
      acc = c.vay * ((vs - vs_m) * (vs + vs_m)) + acc;
      acc = cDx * (v_xp + v_xm) + acc;
      acc = cAx * ((v_c + v_xp) * (u_m_xp + u_xp) - e_uv) + acc;
      acc = cDz * (v_zp + v_zm) + acc;
      acc = cAz * ((v_c + v_zp) * (w_m_zp + w_zp) - e_vw) + acc;
      acc = c.va * v_m + acc;
      acc = c.vc * v_n + acc;
      a.ov[pc + oc] = acc;
    }
    // roll
    vs_m = v_c + v_n;
    u_m = u_c; u_c = u_n;
    w_m = w_c; w_c = w_n;
    v_m = v_c; v_c = v_n;
    u_m_xp = u_xp;
    w_m_zp = w_zp;
    e_uv = e_uv_n;
    e_vw = e_vw_n;
  }
  if (j1 == ny) {   // top wall face of v: boundary value
    const size_t pw = (size_t)ny * plane + oc;
    a.ov[pw] = has_base ? a.bv[pw] : ld(sv + pw);
  }
}

}  // namespace

template <typename T>
cudaError_t launch_momentum(const Geometry& g, const DevTables& tb, const MomArgs<T>& a, cudaStream_t st, int jlo,
                            int jhi) {
  if (jhi < 0) jhi = g.ny;
  if (jlo < 0 || jhi > g.ny || jhi <= jlo) return cudaErrorInvalidValue;
  const int rows = jhi - jlo;
  const int tx = (g.nx + MTX - 1) / MTX, tz = (g.nz + MTZ - 1) / MTZ;
  // enough CTAs for about three waves of two CTAs per SM; chunks of at least 16 rows
  const long long tiles = (long long)tx * tz;
  int chunks = (int)((3LL * 2 * 152 + tiles - 1) / tiles);
  if (chunks > rows / 16) chunks = rows / 16;
  if (chunks < 1) chunks = 1;
  const int jc = (rows + chunks - 1) / chunks;
  chunks = (rows + jc - 1) / jc;
  const size_t smem = sizeof(RowCoef<T>) * (size_t)jc;
  const cudaError_t e = ensure_smem_limit((const void*)k_momentum<T>, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(tx, tz, chunks), block(MTX, MTZ);
  k_momentum<T><<<grid, block, smem, st>>>(g, a, tb.d.inv_dy, tb.d.inv_h, tb.d.a, tb.d.c, jlo, jhi, jc);
  return cudaGetLastError();
}

template cudaError_t launch_momentum<double>(const Geometry&, const DevTables&, const MomArgs<double>&, cudaStream_t,
                                             int, int);
template cudaError_t launch_momentum<float>(const Geometry&, const DevTables&, const MomArgs<float>&, cudaStream_t,
                                            int, int);

}  // namespace pp
