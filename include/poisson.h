/*
 * poisson.h -- C ABI of the GB300 (sm_103a) pressure-Poisson projection library.
 *
 * The library implements the pressure step of the fully explicit projection method of
 * Sec. 2 (Eqs. 4 and 7): on a staggered channel grid that is periodic in x and z and
 * wall-bounded and stretched in y, it solves the discrete Poisson equation of Eq. 8 by
 * real FFTs in x and z (Eq. 9), one wall-normal tridiagonal system per (kx, kz) solved by
 * the PDD algorithm of Sec. 2.2 (Eqs. 10-21, exact reduced system) or by Thomas, and the
 * inverse FFTs (steps (1)-(8) of Sec. 3.2).  The divergence of Eq. 7 and the velocity
 * correction of Eq. 4 are fused around the solve.
 *
 * Conventions (all fields C-ordered, x fastest, contiguous, 16-byte aligned device memory):
 *   cell fields (rhs, p)  : [ny][nz][nx]
 *   u, w (x- / z-faces)   : [ny][nz][nx]; u[j][k][i] on the face between cells i-1 and i
 *   v (y-faces)           : [ny+1][nz][nx]; v[0] and v[ny] are the two walls
 *   y_faces               : ny+1 strictly increasing wall-normal face coordinates
 * The discrete operator is L_h = D G (finite-volume form): homogeneous Neumann at the walls.
 * poisson_solve returns the p with L_h p = rhs - <rhs> (volume-weighted mean removed, the
 * compatibility condition) and zero volume-weighted mean (the gauge).
 *
 * Ownership: every device buffer, including the workspace, belongs to the caller; the plan
 * owns only host memory.  Calls are stream-ordered and asynchronous unless stated.
 * Errors: invalid arguments are reported synchronously as a poisson_status; launch errors
 * as PS_ECUDA; device-side conditions (non-finite input when checked) go to a status word
 * in the workspace, read by poisson_device_status.  The library never aborts or traps.
 */
#ifndef POISSON_H
#define POISSON_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct poisson_plan_s* poisson_plan_t;

typedef enum {
  PS_OK = 0,
  PS_EINVAL = 1,          /* bad argument: null pointer, bad size, misaligned buffer     */
  PS_EUNSUPPORTED = 2,    /* valid but unsupported: nx, nz not 2^a 3^b, pdd_parts !| ny  */
  PS_ENOMEM = 3,          /* host allocation failed                                      */
  PS_ECUDA = 4,           /* a CUDA call or kernel launch failed                         */
  PS_ETIMEOUT = 5,        /* a bounded device-side wait gave up                          */
  PS_ENONFINITE = 6,      /* non-finite input detected (POISSON_CHECK_FINITE)            */
  PS_ENOWORKSPACE = 7     /* poisson_set_workspace has not been called                   */
} poisson_status;

typedef enum {
  PP_FP64 = 0,            /* FP64 in, FP64 arithmetic, FP64 out                          */
  PP_FP32 = 1,            /* FP32 in/out; FP32 FFTs and sweeps; (0,0) and the lowest     */
                          /* |kx|,|kz| <= fp64_low_modes systems in FP64                 */
  PP_FP32_REFINED = 2     /* FP64 in/out; PP_FP32 solves plus refine_steps corrections   */
                          /* driven by an FP64-accurate residual                          */
} poisson_precision;

typedef enum {
  PT_AUTO = 0,            /* PDD (exact reduced system) with an automatic partition      */
  PT_THOMAS = 1,          /* one serial Thomas sweep per system (pdd_parts = 1)          */
  PT_PDD_EXACT = 2,       /* PDD with pdd_parts sub-blocks, exact reduced system Eq. 21  */
  PT_PDD_TRUNCATED = 3    /* PDD as in Sec. 2.2: the framed coupling entries of Eq. 21   */
                          /* dropped, each interface an independent 2x2 system (exact    */
                          /* only when the spikes have decayed across a block; the modes */
                          /* that PP_FP32* solve in FP64 stay exact)                     */
} poisson_tridiag;

#define POISSON_CHECK_FINITE 0x1u   /* flag: scan inputs, set PS_ENONFINITE on NaN/Inf     */
#define POISSON_TIMING       0x2u   /* flag: record CUDA events around every kernel launch */
#define POISSON_GENERIC_FFT  0x4u   /* flag: use the runtime-generic FFT kernels instead of the
                                       compile-time specialised ones (a tiling the autotuner tries) */
#define POISSON_BATCH_PERSISTENT 0x10u /* batched plans (flag of descs[0]): run the whole batch as ONE
                                       persistent kernel over a device work queue instead of one
                                       graph branch per instance (see poisson_solve_batched)      */
#define POISSON_SELFTEST_WAIT 0x8u  /* diagnostics flag: the x-transform that stages its FP64
                                       input by bulk copies (FP32 plans, Nx/2 >= 256) skips its
                                       first copy, so its bounded wait runs out (~2 s): the call
                                       returns, the result is undefined and the device status
                                       reads PS_ETIMEOUT.  For a persistent batched plan (flag of
                                       descs[0]) the first x-transform item of instance 0 is never
                                       counted done, so that instance's next waits run out
                                       (~1 s), the launch aborts and the batch's status word reads
                                       PS_ETIMEOUT.  For testing the failure path only.          */

typedef struct {
  int nx, ny, nz;           /* cells; nx even, nx/2 and nz of the form 2^a 3^b; ny >= 2 */
  double lx, lz;            /* periodic lengths                                          */
  const double* y_faces;    /* host pointer, ny+1 values; copied during poisson_plan_create */
  int precision;            /* poisson_precision                                         */
  int tridiag;              /* poisson_tridiag                                           */
  int pdd_parts;            /* PDD sub-blocks per system (divides ny; <= 32, or <= 256   */
                            /* for FP32 plans with ny/P in {1,2,3,4,6,8,12,16,24});      */
                            /* 0 = automatic                                             */
  int fp64_low_modes;       /* PP_FP32*: systems with kx <= L and |kz| <= L run in FP64  */
  int refine_steps;         /* PP_FP32_REFINED: number of residual corrections (>= 1)    */
  unsigned flags;           /* POISSON_CHECK_FINITE                                      */
} poisson_desc;

/* Build a plan (host only; no CUDA call).  Validates the descriptor, factors the FFT
 * lengths, computes the FP64 grid metrics (Sec. 2: stretched y), the modified wavenumbers
 * of Eq. 9 and the FFT twiddles.  *out receives an opaque handle owned by the library. */
poisson_status poisson_plan_create(const poisson_desc* desc, poisson_plan_t* out);

/* Bytes of device workspace the plan needs (spectral buffer, tables, status word; for
 * PP_FP32_REFINED the FP32 pressure pair, and with refine_steps >= 2 the first correction's
 * residual as an FP32 pair per cell, 8 bytes per point). */
poisson_status poisson_workspace_size(poisson_plan_t plan, size_t* bytes);

/* Attach caller-owned device workspace (>= poisson_workspace_size bytes, 256-byte aligned)
 * and upload the plan's tables with stream-ordered copies on `stream` (a cudaStream_t). */
poisson_status poisson_set_workspace(poisson_plan_t plan, void* workspace, size_t bytes,
                                     void* stream);

/* Solve L_h p = rhs - <rhs> with zero volume-weighted mean of p (Eqs. 7-9).
 * rhs, p: device [ny][nz][nx]; FP64 for PP_FP64 and PP_FP32_REFINED, FP32 for PP_FP32.
 * rhs == p (in place) is allowed for PP_FP64 and PP_FP32; PP_FP32_REFINED re-reads rhs for
 * its residual and returns PS_EINVAL when rhs == p. */
poisson_status poisson_solve(poisson_plan_t plan, const void* rhs, void* p, void* stream);

/* The transpose of poisson_solve as a linear map of rhs (its adjoint, for gradient-based
 * callers): q = S^T g.  Computed as W S(W^-1 g) with W = diag(dy_j) (L_h^T = W L_h W^-1, and the
 * removal of the rhs mean and the zero-mean gauge of S transpose into each other), so q solves
 * L_h^T q = g - omega sum(g) (omega_j = dy_j / (nx nz sum dy)) with sum(q) = 0.
 * g, q: device [ny][nz][nx] with the dtype of poisson_solve; g == q is allowed.  With
 * PP_FP32_REFINED the workspace's pressure pair is overwritten.  Errors as for poisson_solve. */
poisson_status poisson_solve_adjoint(poisson_plan_t plan, const void* g, void* q, void* stream);

/* One projection (Eqs. 4 and 7): p solves L_h p = D(u_star) / dt (made compatible), then
 * u = u_star - dt G p in place on u, v, w.  The wall faces of v are boundary values: they enter D
 * and are not modified.  p_out (device [ny][nz][nx], may be NULL) receives p.
 * Field dtype as for poisson_solve.  PP_FP32_REFINED (FP64 fields): u, v, w are converted in
 * place to FP32 pairs, D(u)/dt is assembled in FP64 into p_out, which is therefore REQUIRED
 * (PS_EINVAL when NULL or aliased with u, v or w), solved by the refined solve and replaced by
 * p; u, v, w are written back in FP64 (after a round trip through FP32 pairs, so the wall
 * faces of v keep their values to 2^-48 relative).  With POISSON_CHECK_FINITE, u, v and w are
 * scanned. */
poisson_status projection_step(poisson_plan_t plan, void* u, void* v, void* w, void* p_out,
                               double dt, void* stream);

/* The right-hand side of the pressure equation as a field: f = D(u)/dt (Eq. 7), the discrete
 * divergence of the staggered velocity at the cell centres, with the grid metrics of the plan.
 * u, w: device [ny][nz][nx]; v: device [ny+1][nz][nx]; f: device [ny][nz][nx], distinct from
 * u, v and w; dtype as for poisson_solve (FP64 for PP_FP64 and PP_FP32_REFINED, FP32 for
 * PP_FP32), computed in that precision.  dt > 0.  One kernel launch on `stream`. */
poisson_status poisson_divergence(poisson_plan_t plan, const void* u, const void* v, const void* w, void* f,
                                  double dt, void* stream);

/* Adjoint of the velocity map of projection_step (which does not depend on dt):
 * g <- g - D^T S^T G^T g in place, S the gauged solve.  Uses the same FFT and PDD kernels:
 * L_h^T = W L_h W^-1 with W = diag(dy_j), so the transposed solve is a forward solve of a
 * row-scaled right-hand side.  PP_FP64 and PP_FP32 plans; PP_FP32_REFINED plans return
 * PS_EUNSUPPORTED (an FP64-accurate adjoint is served by a PP_FP64 plan). */
poisson_status projection_step_adjoint(poisson_plan_t plan, void* gu, void* gv, void* gw,
                                       void* stream);

/* End-to-end variant of projection_step on HOST buffers: copies u, v, w to the device
 * staging buffers (caller-owned device memory of the field sizes), runs projection_step,
 * copies u, v, w (and p when p_host != NULL, using p_dev) back and synchronises `stream`.
 * PP_FP32_REFINED needs p_dev (see projection_step).  Host buffers should be page-locked for
 * asynchronous copies. */
poisson_status projection_step_host(poisson_plan_t plan, void* u_host, void* v_host,
                                    void* w_host, void* p_host, void* u_dev, void* v_dev,
                                    void* w_dev, void* p_dev, double dt, void* stream);

/* Momentum predictor of the fully explicit projection method (Sec. 2, Eqs. 3, 5, 6): Heun's
 * RK2 applied in place to u, v, w (same layouts and dtype as projection_step):
 *   u_bar = u + dt R(u),   u <- u_star = u + dt/2 (R(u) + R(u_bar)),
 *   R(u) = -div(u u) + nu lap(u) + (fx, 0, 0).
 * Second-order central differences on the staggered grid: the advection is the divergence form
 * with two-point face averages (no flux through the walls); the diffusion is the three-point
 * Laplacian with the no-slip wall value 0 half a cell from the first u and w nodes; fx is a
 * constant streamwise body force (the mean pressure gradient that drives the channel).  The
 * wall faces of v are boundary values and are not modified.
 * ub, vb, wb: caller-owned device scratch of the sizes of u, v, w (they receive u_bar).
 * All six buffers must be distinct; dt > 0, nu >= 0, fx finite.  PP_FP64 and PP_FP32 plans
 * compute in their precision; PP_FP32_REFINED plans (FP64 fields) run both stages in
 * double-float arithmetic on FP32 pairs (u, v, w and the scratch hold pairs in between) and
 * return u_star in FP64.  With POISSON_CHECK_FINITE, u, v and w are scanned. */
poisson_status momentum_predictor(poisson_plan_t plan, void* u, void* v, void* w, void* ub, void* vb,
                                  void* wb, double dt, double nu, double fx, void* stream);

/* One full timestep of the fully explicit projection method (Sec. 2, Eqs. 3-7): the RK2
 * predictor of momentum_predictor followed by projection_step (same dt) on u, v, w in place.
 * p_out (may be NULL) receives the pressure.  Arguments as for the two calls. */
poisson_status projection_timestep(poisson_plan_t plan, void* u, void* v, void* w, void* ub, void* vb,
                                   void* wb, void* p_out, double dt, double nu, double fx, void* stream);

/* End-to-end variant of projection_timestep on HOST buffers (as projection_step_host): copies
 * u, v, w to the device buffers u_dev, v_dev, w_dev, runs projection_timestep with the device
 * scratch ub, vb, wb, copies u, v, w (and p when p_host != NULL, through p_dev) back and
 * synchronises `stream`.  For PP_FP64 and PP_FP32 plans with Ny >= 16 (and neither
 * POISSON_CHECK_FINITE nor POISSON_TIMING) the copies go in 8 row chunks on a stream the plan
 * owns: the first momentum stage of each row chunk starts on `stream` once its rows and the row
 * above have arrived, and the inverse x-transform and the gradient correction run chunk by chunk
 * with each chunk of p, u, v, w copied back while the next is computed; the results are those of
 * projection_timestep bit for bit.  Host
 * buffers should be pinned (pageable memory is copied synchronously by CUDA and loses the
 * overlap).  The plan must not be used from two host threads at once. */
poisson_status projection_timestep_host(poisson_plan_t plan, void* u_host, void* v_host, void* w_host,
                                        void* p_host, void* u_dev, void* v_dev, void* w_dev, void* p_dev,
                                        void* ub, void* vb, void* wb, double dt, double nu, double fx,
                                        void* stream);

/* Capacity of the library's built-in device workspace used by poisson_solve_static_ws. */
#define POISSON_STATIC_WS_MAX_BYTES (8u * 1024u * 1024u)

/* poisson_solve without caller-provided workspace, for callers that cannot allocate device
 * memory when they solve (a host application whose memory pool owns the device and forbids
 * library allocations, or a time-critical loop that must not pay cudaMalloc's latency and
 * implicit synchronisation).  The paper has no counterpart: this is a deployment variant.
 * Same arguments, precisions and results as poisson_solve on `plan` (which must have been
 * created by poisson_plan_create; poisson_set_workspace is not needed).  The workspace is a
 * fixed device array of POISSON_STATIC_WS_MAX_BYTES inside the library, held by every GPU
 * that loads the library until the process exits; plans whose poisson_workspace_size exceeds
 * it are rejected with PS_EUNSUPPORTED, batched plans with PS_EINVAL.  No cudaMalloc, cudaFree
 * or other allocator is called.  The first call on each device looks up the array's device
 * address (with that device current; the lookup is serialised by a lock, so concurrent first
 * calls are safe), so make that first call before any stream capture.  The address is kept
 * for the life of the process: after cudaDeviceReset on a device, do not call this entry point
 * on that device again.  Every call reloads the plan's tables into the array from ordinary
 * (pageable) host memory, so the call returns only once `stream` has reached that copy, and
 * clears the array's status word; all calls share the one array per device, so calls that
 * overlap on the GPU (different streams, threads or plans) race: serialise them. */
poisson_status poisson_solve_static_ws(poisson_plan_t plan, const void* rhs, void* p, void* stream);

/* Batched form: `count` independent solves of possibly different sizes and precisions
 * (descs[i] as for poisson_plan_create).  poisson_workspace_size reports the sum of the
 * instances' workspaces and poisson_set_workspace carves one caller allocation.  The batch
 * is solved by poisson_solve_batched only (poisson_solve on it returns PS_EINVAL). */
poisson_status poisson_plan_batched(const poisson_desc* descs, int count, poisson_plan_t* out);

/* Solve every instance i of a batched plan: rhs[i] -> p[i] (host arrays of `count` device
 * pointers, laid out and typed as for poisson_solve).  All instances run in ONE CUDA graph
 * launch on `stream`.  By default each instance's kernel sequence is a branch of the graph, so
 * kernels of different instances run concurrently.  With POISSON_BATCH_PERSISTENT (descs[0].flags)
 * and every instance a PP_FP32 plan with Nx/2 in {32,48,64,96,128,192}, Nz in
 * {64,96,128,192,256,384}, ny <= 256 and a warp-scan PDD partition (pdd_parts a power of two <= 32
 * with ny/pdd_parts in {2,3,4,6,8,12,16}; an automatic partition is chosen so), the graph is ONE
 * persistent kernel that takes (instance, pass, tiles) work items from a device queue, with
 * bounded waits (about a second) for the pass each item depends on: a wait that runs out sets
 * PS_ETIMEOUT in the batch's status word (read by poisson_device_status on the batched plan) and
 * ends the launch.  The graph is captured on the first call and replayed while the pointer
 * arrays stay the same (a change of pointers re-captures it).  The first call also runs the batch
 * once outside capture; make it before capturing `stream` yourself. */
poisson_status poisson_solve_batched(poisson_plan_t plan, const void* const* rhs, void* const* p, void* stream);

/* Autotuner: for the grid of `desc`, time poisson_solve with every candidate PDD partition
 * count (1, the divisors P of ny with 2 <= P <= 32 and ny/P >= 4 and, for FP32 plans, the
 * divisors whose block height ny/P is one of 1, 2, 3, 4, 6, 8, 12, 16, 24) and both FFT tilings
 * (specialised, generic) on `stream`, and return the fastest in *pdd_parts and *flags (the
 * POISSON_GENERIC_FFT bit) with its time in *ms.  It allocates and frees its own device buffers
 * (set-up time, not the solve path) and synchronises `stream`. */
poisson_status poisson_autotune(const poisson_desc* desc, void* stream, int* pdd_parts, unsigned* flags,
                                float* ms);

/* Tuning of the FP32 spectral middle (Sec. 3.2 steps (4)-(6): forward z-transform, wall-normal
 * systems, inverse z-transform).  slab_cols > 0 runs the three passes one slab of slab_cols kx
 * columns at a time, so a slab (ny * nz * slab_cols complex values) stays in L2 between the
 * passes; streams = 2 alternates the slabs between the caller's stream and a second stream owned
 * by the plan (forked and joined with events, so the call stays stream-ordered on the caller's
 * stream).  slab_cols = 0 restores one pass over the whole spectrum.  Needs a PP_FP32 or
 * PP_FP32_REFINED plan whose blocks use the warp-scan PDD kernel (pdd_parts a power of two
 * <= 32 with ny/pdd_parts in {1,2,3,4,6,8,12,16,24}) and the specialised z-transform (nz in
 * {16,...,1024} of the form 2^a 3^b, no POISSON_GENERIC_FFT), slab_cols a multiple of the z tile
 * and of 256/pdd_parts and larger than fp64_low_modes (PS_EUNSUPPORTED otherwise).  Call with
 * the plan's device current (the second stream is created then); results are identical to the
 * whole-spectrum order. */
poisson_status poisson_plan_set_chain(poisson_plan_t plan, int slab_cols, int streams);

/* Diagnostics: the FP64 fused multiply-add throughput of the current device, in GFLOP/s (2 flops
 * per FMA), measured by a kernel of independent FMA chains on every SM, timed with events on
 * `stream` (best of three launches after one warm-up; synchronises `stream`).  It is the
 * denominator of the roofline of FP64-arithmetic-bound kernels.  scratch: caller-owned device
 * memory of at least 8 * 256 * 8 * (multiprocessor count) bytes (receives the chains' sums). */
poisson_status poisson_fp64_fma_rate(void* scratch, size_t bytes, void* stream, double* gflops);

/* Synchronise `stream` and read the device status word (PS_OK, PS_ENONFINITE, ...),
 * then clear it. */
poisson_status poisson_device_status(poisson_plan_t plan, void* stream);

/* Number of kernel launches the last call on this plan issued (for accounting). */
int poisson_last_launch_count(poisson_plan_t plan);

/* With POISSON_TIMING: device time (ms) of each kernel launch of the last call on this plan,
 * measured by events recorded on the launching stream.  Writes up to `max` entries of ms[]
 * and names[] (static strings; either may be NULL), waits for the last event, and returns
 * the number of launches timed (-1 when timing is off or an event query fails). */
int poisson_stage_times(poisson_plan_t plan, float* ms, const char** names, int max);

/* Free the host plan (does not touch the caller's workspace). NULL is accepted. */
poisson_status poisson_plan_destroy(poisson_plan_t plan);

/* Static, human-readable name of a status code. */
const char* poisson_status_string(poisson_status status);

#ifdef __cplusplus
}
#endif

#endif /* POISSON_H */
