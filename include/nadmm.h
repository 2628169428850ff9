/*
 * nadmm.h -- C ABI of the GB300 (sm_103a) Nesterov-accelerated ADMM
 * diffeomorphic registration library (arXiv 2109.12688).
 *
 * Method (paper sections):
 *   Sec. 2, Eq. 1 (N = 1) -- greedy composition phi <- phi o (Id + v), each
 *     outer step re-warping the ORIGINAL moving image and re-linearising;
 *   Eq. 2 -- model (1/s)||rho(v)||^s + (lambda/2)||grad^n v||^2,
 *     rho(v) = <grad I1, v> + I1 - I0, s in {1, 2};
 *   Eq. 5 -- Nesterov-accelerated ADMM (v, w, b, alpha, w_hat, b_hat),
 *     w_hat^0 = b_hat^0 = 0, alpha^0 = 1;
 *   Eq. 6 -- closed-form per-voxel v-step (s = 1 thresholding, s = 2
 *     Sherman-Morrison) and the w-step as a division in the 3D DFT spectrum.
 *
 * Readings of the paper this library implements (the FP64 oracle follows
 * the same ones):
 *   w-step  w = F^-1[ F(v + b_hat) / (1 + (lambda/theta) K^n) ],
 *           K = 2 (3 - cos 2pi p/M - cos 2pi q/N - cos 2pi r/H), periodic;
 *   J = grad(I1 o phi) by central differences with clamped indices;
 *   trilinear sampling with coordinates clamped to [0, dim - 1];
 *   velocity composed per outer step = s * w^K with the global bound
 *   s = min(1, kappa / max ||D w||_inf, delta / max |w|_inf)
 *   (kappa = delta = INFINITY is the paper-literal, unbounded form);
 *   ADMM state reset at every outer step.
 *
 * Conventions for every entry point:
 *   - Volumes are fp32, C-contiguous [nz][ny][nx] (x fastest); vector fields
 *     are SoA [3][nz][ny][nx] with component 0 along x.  (nx, ny, nz) are the
 *     paper's (M, N, H).  Displacements are in voxels, phi(x) = x + u(x).
 *   - "device" pointers are CUDA global-memory addresses on the current
 *     device, 16-byte aligned; "host" pointers are ordinary host memory.
 *     The library never allocates device memory: scratch comes from a
 *     caller-owned workspace (nadmm_workspace_size / nadmm_set_workspace),
 *     and the library never frees caller memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device work is enqueued asynchronously on it; host-detectable
 *     errors are returned before anything is enqueued.  Device-side faults
 *     of the numerics (non-finite values) are recorded in a status word read
 *     by nadmm_get_status.
 *   - A handle is not thread-safe; distinct handles are independent.
 *   - Every function returning nadmm_status sets a thread-local message
 *     (nadmm_last_error) on failure.
 */
#ifndef NADMM_H
#define NADMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum nadmm_status {
  NADMM_OK = 0,
  NADMM_ERR_INVALID_ARG = 1,      /* null pointer, bad parameter value         */
  NADMM_ERR_UNSUPPORTED_SIZE = 2, /* dim < 4, nx % 4, ny % 2, a prime factor
                                     > 509 or more than 5 factors > 7, nz > 256,
                                     or plane beyond shared memory.  Factors
                                     2, 3, 5, 7 use codelet FFT stages, other
                                     primes a direct-sum stage (O(p) per value) */
  NADMM_ERR_ALIGNMENT = 3,        /* device pointer not 16-byte aligned        */
  NADMM_ERR_NO_WORKSPACE = 4,     /* workspace missing or too small            */
  NADMM_ERR_CUDA = 5,             /* a CUDA runtime call failed                */
  NADMM_ERR_NONFINITE = 6,        /* device status: NaN/Inf met in a bound step */
  NADMM_ERR_TIMEOUT = 7,          /* device status: a kernel's bounded wait for its
                                     own bulk copies expired; the kernel returned */
  NADMM_ERR_NO_SAVED_FORWARD = 8  /* nadmm_backward without a saved forward pass   */
} nadmm_status;

/* flags */
#define NADMM_FLAG_NO_GRAPH 1u    /* launch kernels directly instead of replaying
                                     a captured CUDA graph                      */
#define NADMM_FLAG_SAVE_FOR_BACKWARD 2u /* keep what nadmm_backward needs: u at the
                                     start of every outer step (outer_iters x 3V
                                     floats) plus the reverse-sweep scratch
                                     (2 inner_iters + 16 vector fields); single
                                     and batched handles                        */
/* FFT plan choice per axis (bits 2-3 x, 4-5 y, 6-7 z): an axis of n = R1 R2
 * with both R2 = 8 and R2 = 16 available is split with the R2 chosen here;
 * 0 keeps the library default (x 8, y 16, z 8).  nadmm_autotune picks them. */
#define NADMM_FLAG_LANE_SHIFT(axis) (2u + 2u * (axis))   /* axis 0 x, 1 y, 2 z */
#define NADMM_FLAG_LANE8(axis)  (1u << NADMM_FLAG_LANE_SHIFT(axis))
#define NADMM_FLAG_LANE16(axis) (2u << NADMM_FLAG_LANE_SHIFT(axis))
#define NADMM_FLAG_LANE_MASK 0xFCu
#define NADMM_FLAG_PIPELINED_PLANE 0x200u /* run the k >= 2 plane pass of a
                                     fixed schedule as a persistent kernel (two
                                     CTAs per SM, double-buffered copies)
                                     instead of one CTA per tile; same results */
#define NADMM_FLAG_FUSED_PENCIL 0x100u /* run the y/z FFT pass as one kernel (a
                                     2-CTA cluster per (component, kx) plane that
                                     swaps column halves through distributed
                                     shared memory) where it applies, instead of
                                     three kernels; nadmm_autotune tries both  */

#define NADMM_FLAG_FOUR_PASS 0x400u /* run every ADMM iteration as four kernels
                                     (plane pass, y-, z- and inverse y-pass) even
                                     where the two-kernel slab path applies (one
                                     cluster of three CTAs per z-plane doing the
                                     x- and y-DFTs, then one z-pass); same
                                     arithmetic, different rounding order       */

#define NADMM_FLAG_SLAB_PATH 0x800u /* run the slab path wherever the grid
                                     supports it.  Without this flag or
                                     NADMM_FLAG_FOUR_PASS a single grid takes
                                     the slab path only when its 3 nz CTAs fill
                                     at least 80 % of the waves the device
                                     holds (one wave of three-CTA clusters per
                                     z-plane each; decided when the workspace
                                     is attached); flat batches always take it,
                                     pairs on concurrent lanes do not      */

#define NADMM_FLAG_SLAB_PAIRS 0x4000u /* slab path with every cluster taking two
                                     z-planes in turn: a slab pass needs half the
                                     GPU's clusters, so the passes of
                                     registrations running on several streams
                                     share the GPU (implies NADMM_FLAG_SLAB_PATH
                                     where the grid supports the slab path)    */

/* z-slices per thread of the re-warp, gradient and compose kernels (bits
 * 12-13): 0 one, NADMM_FLAG_OUTER_Z2 two, NADMM_FLAG_OUTER_Z4 four; the same
 * results either way, nadmm_autotune picks one. */
#define NADMM_FLAG_OUTER_Z2 0x1000u
#define NADMM_FLAG_OUTER_Z4 0x2000u
#define NADMM_FLAG_OUTER_MASK 0x3000u

typedef struct nadmm_config {
  int32_t nx, ny, nz;         /* grid (M, N, H); see NADMM_ERR_UNSUPPORTED_SIZE */
  int32_t order_n;            /* regulariser order n, 1..8 (Eq. 2)            */
  float lambda;               /* regularisation weight lambda >= 0 (Eq. 2)    */
  float theta;                /* ADMM penalty theta > 0 (Eq. 4)               */
  int32_t outer_iters;        /* compositions, >= 1 (Eq. 1 with N = 1)        */
  int32_t inner_iters;        /* ADMM iterations per composition, >= 1 (Eq. 5)*/
  int32_t data_term;          /* s: 2 (L2, Sherman-Morrison) or 1 (L1)        */
  float eps;                  /* s = 1 denominator guard, > 0 (after Eq. 6)   */
  float bound_kappa;          /* max ||D v||_inf per step, > 0 or INFINITY    */
  float bound_delta;          /* max |v|_inf per step (voxels), > 0 or INFINITY */
  uint32_t flags;             /* NADMM_FLAG_*                                 */
  float admm_tol;             /* 0 or the ADMM stop: after iteration k >= 1,
                                 stop when ||w^k - w^(k-1)||_2 <= admm_tol
                                 ||w^k||_2; inner_iters is then a cap
                                 (Sec. 4, second version; default 0)       */
  float warp_tol;             /* 0 or the outer stop: after a re-warp, stop
                                 when ||I1w_o - I1w_(o-1)||_2 <= warp_tol
                                 ||I1w_(o-1)||_2; outer_iters is then a cap
                                 (the paper's "2 %" is 0.02; default 0)    */
  float restart_eta;          /* < 0 (default -1): Eq. 5 as printed.  >= 0:
                                 adaptive restart of the Nesterov momentum
                                 (not in the paper; the restart of Goldstein
                                 et al.'s fast ADMM, whose O(1/k^2) rate the
                                 paper cites after Eq. 5): with c_k =
                                 ||w^k - w_hat^k||^2 + ||b^k - b_hat^k||^2 and
                                 cbar (+inf at k = 0), c_k < eta cbar sets
                                 cbar = c_k, otherwise cbar /= eta and the
                                 momentum restarts at iteration k + 2 (the
                                 factors forming w_hat^{k+2}, w_hat^{k+3}, ...
                                 become beta_0 = 0, beta_1, ...).  eta = 0
                                 restarts at every test, INFINITY never;
                                 0.999 is Goldstein et al.'s value.  Needs
                                 the slab path, fixed iteration counts and no
                                 NADMM_FLAG_SAVE_FOR_BACKWARD                 */
} nadmm_config;

typedef struct nadmm_context* nadmm_handle;

/* Fill `cfg` with defaults for an nx x ny x nz grid: n = 2, lambda = 10,
 * theta = 0.1, 10 outer x 10 inner iterations, s = 2, eps = 1e-6,
 * kappa = 0.5, delta = 1.0, flags = 0.  Host only. */
void nadmm_config_init(nadmm_config* cfg, int32_t nx, int32_t ny, int32_t nz);

/* Validate `cfg` and create a handle (host memory only; no CUDA call).
 * Errors: INVALID_ARG, UNSUPPORTED_SIZE.  *out is NULL on failure. */
nadmm_status nadmm_create(const nadmm_config* cfg, nadmm_handle* out);

/* Release the handle and any CUDA graph/stream it created.  NULL is a no-op.
 * The workspace is the caller's and is not freed. */
void nadmm_destroy(nadmm_handle h);

/* Bytes of device workspace the handle needs (host only). */
nadmm_status nadmm_workspace_size(nadmm_handle h, size_t* bytes);

/* Attach a caller-owned device workspace of at least nadmm_workspace_size
 * bytes, 256-byte aligned, on the current device.  Uploads the FFT twiddle
 * and symbol tables into it (synchronous copy).  The memory must stay valid
 * until the handle is destroyed or another workspace is attached.
 * Errors: INVALID_ARG, ALIGNMENT, NO_WORKSPACE, CUDA. */
nadmm_status nadmm_set_workspace(nadmm_handle h, void* dev_ptr, size_t bytes);

/* Change lambda and theta (Eq. 2, Eq. 4) for later calls.  Host only. */
nadmm_status nadmm_set_params(nadmm_handle h, float lambda, float theta);

/* Full registration (Sec. 2 outer loop around Eq. 5/6):
 *   fixed  = I0 (target), device [nz][ny][nx];
 *   moving = I1 (source), device [nz][ny][nx];
 *   u_out  = displacement u with I1 o (Id + u) ~ I0, device [3][nz][ny][nx].
 * Runs outer_iters x (inner_iters ADMM iterations + bound + compose +
 * re-warp) as one CUDA-graph replay on `stream` (or direct launches with
 * NADMM_FLAG_NO_GRAPH).  Inputs are read-only; u_out is overwritten.
 * Errors: INVALID_ARG, ALIGNMENT, NO_WORKSPACE, CUDA. */
nadmm_status nadmm_register(nadmm_handle h, const float* fixed, const float* moving,
                            float* u_out, void* stream);

/* Same as nadmm_register with HOST buffers: copies fixed/moving host->device
 * into the workspace, registers, and copies u back device->host, all
 * enqueued on `stream`; returns after the stream has completed the copy of
 * u_out (pinned host memory makes the copies asynchronous DMA). */
nadmm_status nadmm_register_host(nadmm_handle h, const float* fixed_host,
                                 const float* moving_host, float* u_out_host, void* stream);

/* Synchronise `stream`, read and clear the device status word.
 * Returns NADMM_OK, NADMM_ERR_TIMEOUT or NADMM_ERR_NONFINITE (or CUDA on a
 * runtime error). */
nadmm_status nadmm_get_status(nadmm_handle h, void* stream);

/* Iterations the last registration on a single handle ran (synchronises
 * `stream`): outer steps composed and ADMM iterations whose result was used,
 * summed over the outer steps.  Without thresholds these are outer_iters and
 * outer_iters x inner_iters.  With admm_tol / warp_tol (Sec. 4, second
 * version) the kernels of a stopped loop still launch from the graph but
 * return at once; these counters say how much work ran.
 * Errors: INVALID_ARG, NO_WORKSPACE, CUDA. */
nadmm_status nadmm_get_iterations(nadmm_handle h, void* stream, int32_t* outer_run,
                                  int32_t* admm_run);

/* Thread-local description of the last failure of this thread. */
const char* nadmm_last_error(void);

/* Static name of a status code. */
const char* nadmm_status_string(nadmm_status s);

/* ---------------------------------------------------------------------
 * Batched registration: many independent pairs of different grid sizes
 * (the paper registers each ED/ES pair on its own; Sec. 4 runs 220 pairs).
 * --------------------------------------------------------------------- */

/* Create a handle for npairs pairs: pair i has grid dims[3i], dims[3i+1],
 * dims[3i+2] (nx, ny, nz) and every other setting from `base` (its nx, ny,
 * nz are ignored).  Each grid is validated as by nadmm_create; the first
 * failure is returned with "pair i: ..." in nadmm_last_error.
 *
 * By default the pairs run on `lanes` concurrent graph branches (default
 * min(npairs, 2); nadmm_batch_set_lanes), spread longest first to balance
 * voxel counts; pairs of one lane run one after another and share that
 * lane's scratch, so the workspace is one state region per lane (its largest
 * pair's) plus every pair's own region (tables, tape).  With two or more
 * lanes every pair takes the four-kernel path unless its flags force the
 * slab path, it uses adaptive restart or the handle keeps the reverse-mode
 * tape (NADMM_FLAG_SAVE_FOR_BACKWARD): four-kernel passes overlap across
 * lanes, and the slab path's reverse sweep is the faster one.
 * Flat execution (lane count 0, when every pair can take the slab path and
 * NADMM_FLAG_SAVE_FOR_BACKWARD is not set): every pair keeps its own state
 * region, and each phase of an ADMM iteration is one launch over all pairs
 * -- the slab pass of every z-plane of every pair (per shared-memory class:
 * planes that fit two CTAs per SM, then the rest; a class of at most four
 * waves of clusters one wave per launch) and the z-pass of every pair
 * sharing a z plan (one launch per plan) -- while the outer-step kernels run
 * per pair.  Host only. */
nadmm_status nadmm_create_batched(const nadmm_config* base, int32_t npairs, const int32_t* dims,
                                  nadmm_handle* out);

/* nadmm_create_batched with a whole configuration per pair: pair i is
 * registered with cfgs[i] (its grid, order, lambda, theta, data term, bound
 * ...).  Every pair must have the same outer_iters, inner_iters and flags (one
 * schedule); errors as nadmm_create_batched, INVALID_ARG when they differ.
 * The paper has no counterpart; host only. */
nadmm_status nadmm_create_batched_configs(const nadmm_config* cfgs, int32_t npairs,
                                          nadmm_handle* out);

/* Change the lane count of a batched handle before its workspace is
 * attached: 0 = flat execution (needs every pair on the slab path and no
 * reverse-mode tape), 1 = all pairs in sequence, lanes > npairs is clamped to
 * npairs.  Errors: INVALID_ARG (not batched, lanes < 0, flat not possible,
 * workspace already attached). */
nadmm_status nadmm_batch_set_lanes(nadmm_handle h, int32_t lanes);

/* The lane count of a batched handle (after clamping; 0 = flat).  Host only.
 * Errors: INVALID_ARG (not batched, lanes NULL). */
nadmm_status nadmm_batch_get_lanes(nadmm_handle h, int32_t* lanes);

/* Replace the plan bits (NADMM_FLAG_LANE*, NADMM_FLAG_FUSED_PENCIL,
 * NADMM_FLAG_FOUR_PASS, NADMM_FLAG_SLAB_PATH, NADMM_FLAG_OUTER_*) of pair
 * `pair` (0-based) of a
 * batched handle before its workspace is attached (e.g. with the result of
 * nadmm_autotune for that pair's grid); the workspace size may change.
 * Errors: INVALID_ARG. */
nadmm_status nadmm_batch_set_pair_plan(nadmm_handle h, int32_t pair, uint32_t plan_flags);

/* Register every pair of a batched handle: fixed[i], moving[i] device
 * [nz_i][ny_i][nx_i], u_out[i] device [3][nz_i][ny_i][nx_i] (host arrays of
 * npairs device pointers each).  The same computation as nadmm_register on
 * each pair (bit for bit that of a single handle on the path the pair takes:
 * the slab path when flat, the four-kernel path on two or more lanes unless
 * forced, see nadmm_create_batched), as one CUDA-graph replay on `stream`
 * (re-captured when any pointer changes) or, with NADMM_FLAG_NO_GRAPH,
 * direct launches (flat: the phases in order; lanes: the pairs in order).
 * nadmm_get_status on the handle reports the first pair whose status word
 * is set.  Only nadmm_register_batched,
 * nadmm_backward_batched, nadmm_get_status, nadmm_workspace_size,
 * nadmm_set_workspace, nadmm_batch_set_lanes and nadmm_destroy accept a
 * batched handle.
 * Errors: INVALID_ARG, ALIGNMENT, NO_WORKSPACE, CUDA. */
nadmm_status nadmm_register_batched(nadmm_handle h, const float* const* fixed,
                                    const float* const* moving, float* const* u_out,
                                    void* stream);

/* ---------------------------------------------------------------------
 * Pyramid (Sec. 4, "Hyperparameter tuning"): the registration run on
 * `levels` grids, each half the size of the next, coarsest first.
 * --------------------------------------------------------------------- */

/* Create a pyramid handle.  `finest` gives the full-resolution grid and every
 * other setting; level l (0 = finest) has grid (nx, ny, nz) / 2^l, which must
 * pass nadmm_create's checks, so every dimension must be divisible by
 * 2^(levels - 1).  outer[i] and inner[i] are the warpings and ADMM iterations
 * of the i-th level run, COARSEST FIRST (the paper's first version: outer
 * {10, 10, 5}, inner {10, 5, 5} on three levels).  Readings where the paper
 * gives no detail: a coarser image is the 2 x 2 x 2 block average of the
 * finer one; a level starts from the coarser level's displacement resampled
 * at cell centres and doubled, u_fine(x) = 2 u_coarse((x - 1/2) / 2)
 * (trilinear, clamped); lambda, theta, n, s and the velocity bound (in voxels
 * of each level) are shared.  1 <= levels <= 5; NADMM_FLAG_SAVE_FOR_BACKWARD
 * is rejected.  The workspace holds one shared state region, every level's
 * tables and the coarse images and displacements.  Host only.
 * Errors: INVALID_ARG, UNSUPPORTED_SIZE ("level l: ..."). */
nadmm_status nadmm_create_pyramid(const nadmm_config* finest, int32_t levels,
                                  const int32_t* outer, const int32_t* inner,
                                  nadmm_handle* out);

/* Register with a pyramid handle: fixed, moving device [nz][ny][nx] and u_out
 * device [3][nz][ny][nx] on the finest grid, as one CUDA-graph replay (or
 * direct launches with NADMM_FLAG_NO_GRAPH).  Only nadmm_register_pyramid,
 * nadmm_get_status, nadmm_workspace_size, nadmm_set_workspace and
 * nadmm_destroy accept a pyramid handle.
 * Errors: INVALID_ARG, ALIGNMENT, NO_WORKSPACE, CUDA. */
nadmm_status nadmm_register_pyramid(nadmm_handle h, const float* fixed, const float* moving,
                                    float* u_out, void* stream);

/* ---------------------------------------------------------------------
 * Step-level entry points: one part of the path each, on device buffers of
 * the handle's grid, using the handle's workspace as scratch.  They run the
 * same kernels as nadmm_register.
 * --------------------------------------------------------------------- */

/* Regulariser step alone (Eq. 5 line 2 solved by Eq. 6 last line):
 *   w = F^-1[ F(y) / (1 + (lambda/theta) K^n) ] per component,
 * y, w device [3][nz][ny][nx]; w may alias y. */
nadmm_status nadmm_spectral_solve(nadmm_handle h, const float* y, float* w, void* stream);

/* ADMM iterations k .. k+steps-1 of Eq. 5 for the linearisation (J, c):
 *   J device [3][nz][ny][nx] (= grad I1w), c device [nz][ny][nx] (= I1w - I0);
 *   w_km1, w_km2, b_km1, b_km2: state after iteration k-1, device
 *   [3][nz][ny][nx] (w^{k-1}, w^{k-2}, b^{k-1}, b^{k-2}); ignored when k = 0
 *   (w_hat^0 = b_hat^0 = 0), and w_km2/b_km2 ignored when k = 1 (beta_0 = 0);
 *   w_out, b_out: device [3][nz][ny][nx], receive w^{k+steps-1}, b^{k+steps-1}.
 * Uses the Nesterov factors beta_{k-1} = (alpha^{k-1} - 1)/alpha^k.
 * Output buffers must not alias inputs.  k >= 0, steps >= 1. */
nadmm_status nadmm_admm_run(nadmm_handle h, const float* J, const float* c,
                            const float* w_km1, const float* w_km2,
                            const float* b_km1, const float* b_km2,
                            int32_t k, int32_t steps, float* w_out, float* b_out,
                            void* stream);

/* Re-warp and re-linearise (Sec. 2, text after Eq. 2; Eq. 2's rho):
 *   I1w = I1 o (Id + u) (trilinear), J = grad I1w, c = I1w - I0.
 * fixed, moving device [nz][ny][nx]; u device [3][nz][ny][nx];
 * J device [3][nz][ny][nx]; c device [nz][ny][nx]; I1w_out device
 * [nz][ny][nx] or NULL.  Outputs must not alias inputs. */
nadmm_status nadmm_linearise(nadmm_handle h, const float* fixed, const float* moving,
                             const float* u, float* J, float* c, float* I1w_out,
                             void* stream);

/* Bound and compose (Sec. 2, Eq. 1 with N = 1):
 *   s = min(1, kappa / max ||D w||_inf, delta / max |w|_inf),
 *   u_out(x) = s w(x) + u_in(x + s w(x)).
 * w, u_in, u_out device [3][nz][ny][nx] (u_out must not alias u_in or w);
 * scale_out: device float receiving s, or NULL. */
nadmm_status nadmm_bound_compose(nadmm_handle h, const float* w, const float* u_in,
                                 float* u_out, float* scale_out, void* stream);

/* Jacobian determinant det(I + D u) with central differences (Sec. 4,
 * "Quantitative results"): det device [nz][ny][nx] or NULL;
 * nonpositive device uint32 receiving the count of det <= 0, or NULL. */
nadmm_status nadmm_jacobian_det(nadmm_handle h, const float* u, float* det,
                                uint32_t* nonpositive, void* stream);

/* Regulariser solve that allocates nothing.  The paper has no counterpart:
 * this entry exists for callers that may not allocate device memory -- a
 * library running inside an application or framework that owns every device
 * allocation through its own pool, or a latency-critical caller that cannot
 * risk the device synchronisation cudaMalloc/cudaFree may cause.
 *
 * Computes the same result as nadmm_spectral_solve for an nx x ny x nz grid,
 * order n, lambda and theta, without a handle or workspace: y, w device
 * [3][nz][ny][nx] fp32, 16-byte aligned, w may alias y.  Its limits are
 * narrower than nadmm_create's: every dimension >= 4 with prime factors in
 * {2, 3, 5, 7} only (nadmm_create also takes primes up to 509), nx a
 * multiple of 4, ny even, nz <= 256, 1 <= order_n <= 8.  The scratch (half
 * spectrum + FFT tables) lives in one static device array of 24 MiB
 * (25165824 bytes) that every GPU loading the library holds until the
 * process exits; grids needing more, i.e. when 3 (nx/2+1) ny nz 8 bytes plus
 * a few KB of tables exceed it (128x128x96 fits, 160x160x112 does not), are
 * rejected.  Every size and argument check runs before any device work and
 * returns NADMM_ERR_UNSUPPORTED_SIZE, INVALID_ARG or ALIGNMENT.  No
 * cudaMalloc, cudaFree or other allocating call is made.
 *
 * The first call on a device performs a one-time set-up on that device (it
 * looks up the array's device address with cudaGetSymbolAddress and raises
 * the pass kernels' shared-memory limits); make that first call before any
 * stream capture.  The address is cached for the life of the process: after
 * cudaDeviceReset (or a primary-context reset) it is stale, so do not call
 * this entry point again in a process that has reset the device.  Every
 * call shares the one array and it keeps the last call's contents (nothing
 * in it needs clearing: each call writes every byte it later reads, FFT
 * tables included, with one small table-fill launch), so calls whose device
 * work overlaps -- on different streams or from different threads -- race
 * and must be serialised by the caller. */
nadmm_status nadmm_spectral_solve_noalloc(int32_t nx, int32_t ny, int32_t nz, int32_t order_n,
                                          float lambda, float theta, const float* y, float* w,
                                          void* stream);

/* ---------------------------------------------------------------------
 * Autotuning of the FFT plans (the paper has no counterpart).
 * --------------------------------------------------------------------- */

/* Device bytes nadmm_autotune needs for `cfg`'s grid (host only). */
nadmm_status nadmm_autotune_workspace_size(const nadmm_config* cfg, size_t* bytes);

/* Time every plan choice of `cfg`'s grid -- each axis with both an 8- and a
 * 16-lane split tried both ways, the two-kernel slab path where it applies,
 * and the four-kernel path with and without the fused y/z pass -- on one
 * ADMM iteration (the k >= 2 pass(es); 3 warm-up and 10 timed repetitions,
 * CUDA events on `stream`, minimum kept) in the caller's device workspace
 * (at least nadmm_autotune_workspace_size bytes, 256-byte aligned; its
 * contents are overwritten) and write the fastest choice as NADMM_FLAG_LANE*,
 * NADMM_FLAG_FUSED_PENCIL and NADMM_FLAG_FOUR_PASS / NADMM_FLAG_SLAB_PATH bits, then
 * for that plan the z-slices per thread of the outer-step kernels (re-warp,
 * gradient, bound, compose of one outer step timed with 1, 2 and 4) as
 * NADMM_FLAG_OUTER_* bits, to *best_flags
 * (cfg->flags with those bits replaced) and its time in ms to *best_ms (host
 * pointers; best_ms may be NULL).  Synchronises `stream`.
 * Errors: INVALID_ARG, UNSUPPORTED_SIZE, ALIGNMENT, NO_WORKSPACE, CUDA. */
nadmm_status nadmm_autotune(const nadmm_config* cfg, void* workspace, size_t bytes,
                            void* stream, uint32_t* best_flags, float* best_ms);

/* ---------------------------------------------------------------------
 * Reverse mode (gradients through the registration).  The paper has no
 * counterpart; it differentiates Sec. 2's outer loop around Eq. 5/6 with the
 * s = 2 data step, so that the registration can sit inside a learned
 * pipeline.  Conventions at the non-smooth points: a clamped sample
 * coordinate passes no gradient unless strictly inside [0, dim - 1];
 * sign(0) = 0; the maxima of the velocity bound share their gradient equally
 * among the entries attaining them; s = min(1, kappa/max||Dw||,
 * delta/max|w|) follows the first candidate, in that order, attaining it.
 * --------------------------------------------------------------------- */

/* Vector-Jacobian product of the last nadmm_register (or nadmm_register_host)
 * on this handle, which must have NADMM_FLAG_SAVE_FOR_BACKWARD, data_term 2
 * and lambda > 0:
 *   fixed, moving: device [nz][ny][nx], the SAME data the forward pass used;
 *   grad_u: device [3][nz][ny][nx], dL/du for the forward output u;
 *   grad_fixed, grad_moving: device [nz][ny][nx], overwritten with dL/dI0,
 *   dL/dI1 through the registration;
 *   grad_lambda, grad_theta: device float (16-byte aligned) receiving
 *   dL/dlambda, dL/dtheta, or NULL.
 * Recomputes each outer step's ADMM iterates from the saved displacements
 * (one forward sweep plus one reverse sweep of K spectral solves per outer
 * step).  Captured into a CUDA graph (re-captured when a pointer changes)
 * unless NADMM_FLAG_NO_GRAPH.  Scatter-adds use float atomics, so results
 * may differ in the last bits between runs.
 * Errors: INVALID_ARG, ALIGNMENT, NO_WORKSPACE, NO_SAVED_FORWARD, CUDA. */
nadmm_status nadmm_backward(nadmm_handle h, const float* fixed, const float* moving,
                            const float* grad_u, float* grad_fixed, float* grad_moving,
                            float* grad_lambda, float* grad_theta, void* stream);

/* nadmm_backward for every pair of a batched handle created with
 * NADMM_FLAG_SAVE_FOR_BACKWARD, after a nadmm_register_batched on it: host
 * arrays of npairs device pointers, each entry as in nadmm_backward for that
 * pair's grid; grad_lambda and grad_theta may be NULL arrays or hold NULL
 * entries.  Each pair keeps its own tape (outer_iters x 3V floats); the
 * reverse-sweep scratch is shared by the pairs of a lane.  One CUDA-graph
 * replay (re-captured when a pointer changes) on `stream`.
 * Errors: INVALID_ARG, ALIGNMENT, NO_WORKSPACE, NO_SAVED_FORWARD, CUDA. */
nadmm_status nadmm_backward_batched(nadmm_handle h, const float* const* fixed,
                                    const float* const* moving, const float* const* grad_u,
                                    float* const* grad_fixed, float* const* grad_moving,
                                    float* const* grad_lambda, float* const* grad_theta,
                                    void* stream);

/* Loss L = 1/2 sum_x (I1(x + u(x)) - I0(x))^2 (trilinear, clamped), the
 * quantity whose gradients the reverse mode is tested on:
 * fixed, moving device [nz][ny][nx]; u device [3][nz][ny][nx];
 * loss: device float (16-byte aligned), summed in double, stored as float. */
nadmm_status nadmm_ssd_after_warp(nadmm_handle h, const float* fixed, const float* moving,
                                  const float* u, float* loss, void* stream);

/* Gradient of the loss above scaled by the device scalar grad_loss:
 * grad_fixed (or NULL), grad_moving, grad_u (or NULL) overwritten, device,
 * shaped like fixed, moving and u. */
nadmm_status nadmm_ssd_after_warp_backward(nadmm_handle h, const float* fixed,
                                           const float* moving, const float* u,
                                           const float* grad_loss, float* grad_fixed,
                                           float* grad_moving, float* grad_u, void* stream);

/* Failure-detection self-test (the paper has no counterpart): one block
 * waits, with the same bounded mbarrier wait the passes use for their bulk
 * copies but `attempts` (1 .. 2^20) tries, on a barrier that nothing
 * arrives at and no copy targets.  The wait expires, the kernel records
 * NADMM_ERR_TIMEOUT in the handle's status word and returns normally, so
 * the next nadmm_get_status reports NADMM_ERR_TIMEOUT and the context stays
 * usable.  Errors: INVALID_ARG, NO_WORKSPACE, CUDA. */
nadmm_status nadmm_selftest_wait_timeout(nadmm_handle h, int32_t attempts, void* stream);

/* Momentum restarts that took effect (config restart_eta >= 0; a test of
 * iteration k restarts iteration k + 2, so tests of the last two iterations of
 * a loop have none) counted over all outer steps
 * of the last nadmm_register on `h` (host int32).  Synchronises `stream`.
 * Errors: INVALID_ARG (no restart on this handle), NO_WORKSPACE, CUDA. */
nadmm_status nadmm_get_restarts(nadmm_handle h, void* stream, int32_t* restarts);

/* ---------------------------------------------------------------------
 * Measurement
 * --------------------------------------------------------------------- */

/* Kernel classes reported by nadmm_register_profiled. */
#define NADMM_KC_PLANE_FIRST   0  /* plane pass, k = 0 (no state read)          */
#define NADMM_KC_PLANE_K1      1  /* plane pass, k = 1 (beta_0 = 0)             */
#define NADMM_KC_PLANE         2  /* plane pass, k >= 2 (full Nesterov step)    */
#define NADMM_KC_PLANE_FINAL   3  /* plane pass, final inverse x-DFT -> w^K     */
#define NADMM_KC_PENCIL        4  /* pencil pass (y/z DFTs, symbol, inverses)   */
#define NADMM_KC_WARP          5  /* trilinear re-warp of I1                    */
#define NADMM_KC_GRAD          6  /* gradient + residual                        */
#define NADMM_KC_BOUND         7  /* velocity bound reduction                   */
#define NADMM_KC_COMPOSE       8  /* composition u <- s w + u o (Id + s w)      */
#define NADMM_KC_SLAB_FIRST    9  /* slab pass, k = 0                            */
#define NADMM_KC_SLAB_K1      10  /* slab pass, k = 1                            */
#define NADMM_KC_SLAB         11  /* slab pass, k >= 2 (x/y DFTs + point-wise)   */
#define NADMM_KC_SLAB_FINAL   12  /* slab pass, final inverse x/y DFTs -> w^K    */
#define NADMM_KC_ZSLAB        13  /* z-pass of the slab path (z-DFT, symbol)     */
#define NADMM_KC_COUNT        14

/* nadmm_register with direct launches on `stream`, a CUDA event recorded on
 * that stream before and after every kernel, and a stream synchronisation
 * at the end.  kernel_ms[NADMM_KC_COUNT] (host) receives the summed device
 * time of each kernel class, launches[NADMM_KC_COUNT] (host) the number of
 * launches.  Output u_out is the same as nadmm_register's. */
nadmm_status nadmm_register_profiled(nadmm_handle h, const float* fixed, const float* moving,
                                     float* u_out, void* stream, float* kernel_ms,
                                     int32_t* launches);

#ifdef __cplusplus
}
#endif
#endif /* NADMM_H */
