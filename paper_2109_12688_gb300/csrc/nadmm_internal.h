// Internal interfaces between the host orchestration (nadmm.cu) and the
// kernel translation units.  Not part of the public ABI.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "fft_device.cuh"

namespace nadmm {

// ---------------------------------------------------------------- ADMM passes
// Where the "plane pass" takes w^{k-1}, b^{k-1} from.
enum InMode : int {
  IN_NONE = 0,   // k = 0: w_hat^0 = b_hat^0 = 0
  IN_SPEC = 1,   // inverse x-transform of the filtered spectrum; b = y - w
  IN_STATE = 2,  // explicit real-space state buffers (step-level entry point)
  IN_FIELD = 3,  // plain forward transform of a real field (spectral solve)
};

// Plane pass: one CTA owns R rows (y0..y0+R-1) of one z-plane, all three
// components.  It finishes iteration k-1 (inverse x-DFT, dual update) and
// starts iteration k (Nesterov extrapolation, closed-form v-step, forward
// x-DFT), so the 3D transform needs only this pass and the pencil pass.
struct PlaneArgs {
  CUtensorMap smap;        // 3D view {ny, nz, 3 nkx} of the spectrum, box {R, 1, <= 256}
  float2* spec;            // [3][nkx][nz][ny] half spectrum (in/out)
  float* y;                // [3][V] y = v + b_hat of the current iteration (in/out) or null
  float* wp;               // [3][V] w state slot (in: w^{k-2}, out: w^{k-1})
  float* bp;               // [3][V] b state slot
  const float* J;          // [3][V]
  const float* c;          // [V]
  const float* w_in;       // IN_STATE: w^{k-1};  IN_FIELD: the field
  const float* b_in;       // IN_STATE: b^{k-1}
  const float* wprev_in;   // IN_STATE: w^{k-2}
  const float* bprev_in;   // IN_STATE: b^{k-2}
  float* w_out;            // no-step variant: receives w^{k-1}
  float* b_out;            // no-step variant: receives b^{k-1} (or null)
  const float2* twx;       // x-axis stage twiddles
  const int* posx;         // position of frequency kx after the forward x-DFT
  unsigned* status;        // device status word (bit 1: a bounded wait expired) or null
  float* u_hist;           // reverse-mode recompute: receives u^k = w_hat^k - b_hat^k, or null
  float* w_tile_out;       // reverse-mode recompute: where w^{k-1} goes instead of wp, or null
  unsigned* conv;          // threshold words (kConv*) or null when no threshold is set
  double* conv_acc;        // [0] sum (w^{k-1} - w^{k-2})^2, [1] sum (w^{k-1})^2
  float admm_tol;
  AxisPlan px;
  FastDiv nx_div;          // division by nx
  FastDiv lines_div;       // division by the line count 3 R / 2
  FastDiv half_div;        // division by R / 2
  FastDiv nkx_div;         // division by nkx
  FastDiv tiles_div;       // division by ny / R
  int nx, ny, nz, nkx;     // nkx = nx/2 + 1
  int R;                   // rows per CTA (even, divides ny)
  int pitch;               // shared-memory line pitch (>= nx)
  int xr1, xr2;            // lane-FFT plan of the x axis (xr2 = 0: shared-memory stages)
  int xlog2r2;             // log2(xr2), or -1 (line positions not swizzled)
  int pipe;                // 1: the k >= 2 pass runs as the pipelined persistent kernel
                           //    (needs spec_tma; opt-in)
  int spec_tma;            // 1: the CTA's spectrum block moves by tensor copies through
                           // the line buffer (needs smap); 0: per-thread loads/stores
  float beta;              // beta_{k-1}
  float theta, eps;
  int data_term;           // 1 or 2
};

// Pencil work on the half spectrum: forward y-DFTs (y-pass), z-DFT with the
// inverse-symbol multiply of Eq. 6 and inverse z-DFT (z-pass), inverse
// y-DFTs (y-pass).
struct PencilArgs {
  CUtensorMap zmap;        // 2D view [3 nkx nz rows][ny] of the spectrum, box [nz][zcols]
  float2* spec;            // [3][nkx][nz][ny] (in/out)
  const float2* twy;
  const float2* twz;
  const float* Kx;         // [nkx] 4 sin^2(pi kx / nx)
  const float* Ky;         // [ny] 4 sin^2(pi ky / ny) by position
  const float* Kz;         // [nz] 4 sin^2(pi kz / nz) by position
  unsigned* status;        // device status word (bit 1: a bounded wait expired) or null
  const unsigned* conv;    // threshold words (kConv*) or null
  AxisPlan py, pz;
  FastDiv yrows_div, zcols_div, ztiles_div, nkx_div;
  int ny, nz, nkx;
  int yrows;               // (component, kx, z) rows per y-pass CTA (divides nz)
  int ypitch;              // y-pass shared-memory row pitch (even: 16-byte aligned rows)
  int zcols;               // y positions per z-pass CTA (divides ny, even)
  int order_n;
  float gamma;             // lambda / theta
  float scale;             // 1 / (nx ny nz)
  int fused;               // 1: one fused y/z/y kernel (pencil_fused.cu) runs the pass
};

// ---------------------------------------------------------------- slab path
// Two kernels per ADMM iteration on the spectrum layout [z][3][ny][nkx]:
//   slab pass: one cluster of three CTAs per z-plane, CTA c holding the whole
//       half-spectrum plane of component c in shared memory: inverse y- and
//       x-DFTs, the point-wise part of the iteration (every CTA takes a third
//       of the plane's voxels for all three components, reading and writing
//       the other CTAs' planes through distributed shared memory), forward x-
//       and y-DFTs;
//   z-pass: z-DFT, multiply by 1/(1 + gamma K^n)/(nx ny nz), inverse z-DFT.
enum SlabMode : int {
  SLAB_FIRST = 0,       // k = 0: w_hat^0 = b_hat^0 = 0, no spectrum read
  SLAB_SPEC = 1,        // k = 1: spectrum of y^0 in, beta_0 = 0
  SLAB_SPEC_PREV = 2,   // k >= 2: spectrum in, w^{k-2}, b^{k-2} from the state slots
  SLAB_FINAL = 3,       // inverse transforms only: w^{K-1} (and b^{K-1}) out
  SLAB_FIELD = 4,       // forward transforms of a given field (spectral solve)
  SLAB_STATE = 5,       // k = 1 from explicit buffers w^{k-1}, b^{k-1}
  SLAB_STATE_PREV = 6,  // k >= 2 from explicit buffers w^{k-1}, b^{k-1}, w^{k-2}, b^{k-2}
  SLAB_ADJ = 7,         // reverse step k >= 1: S g in, adjoint point-wise step, F(g') out
  SLAB_ADJ_LAST = 8,    // reverse step k = 0: S g in, adjoint point-wise step, no transform out
};

// Reverse step k of Eq. 5 (s = 2) inside a slab pass (modes SLAB_ADJ*): the
// plane holds S g^k after the inverse transforms, g^k = wbar^k - bbar^k; the
// point-wise step adds the contributions to J, c, theta, gamma and to the
// adjoint slots of iterations k - 1 (added) and k - 2 (stored), and leaves
// g^{k-1} = wbar^{k-1} - bbar^{k-1} in the plane (and in g) for the forward
// transforms.
struct SlabAdj {
  const float *wk, *uk;    // [3][V] w^k, u^k = w_hat^k - b_hat^k of the recomputed forward
  const float* Bk;         // [3][V] bbar^k
  float *W1bar, *B1bar;    // [3][V] wbar^{k-1}, bbar^{k-1} (+=), null for k = 0
  float *W2bar, *B2bar;    // [3][V] wbar^{k-2}, bbar^{k-2} (stored), null for k <= 1
  const float* g_in;       // [3][V] g^k
  float* g_out;            // [3][V] g^{k-1} (k >= 1; may be g_in: each quad is read first)
  float *gJ, *gc;          // [3][V], [V] (+=)
  double* acc;             // [1] += dL/dtheta part, [2] += dL/dgamma part
  float inv_gamma;         // theta / lambda
};

struct SlabArgs {
  float2* spec;            // [nz][3][ny][nkx] half spectrum (in/out)
  float* y;                // [3][V] y = v + b_hat (in/out); FINAL: null unless b_out is wanted
  float* wp;               // [3][V] w state slot (in: w^{k-2}, out: w^{k-1})
  float* wp_out;           // where w^{k-1} goes when not back to wp (reverse-mode history), or null
  float* u_hist;           // [3][V] u^k = w_hat^k - b_hat^k recorded (reverse-mode history), or null
  float* bp;               // [3][V] b state slot
  const float* J;          // [3][V]
  const float* c;          // [V]
  const float* w_in;       // FIELD: the field; STATE*: w^{k-1}
  const float* b_in;       // STATE*: b^{k-1}
  const float* wprev_in;   // STATE2: w^{k-2}
  const float* bprev_in;   // STATE2: b^{k-2}
  float* w_out;            // FINAL: w^{K-1}
  float* b_out;            // FINAL: b^{K-1} = y - w^{K-1}, or null
  const float2* twx;       // stage twiddles of the nx/2-point lane plan [xr1, xr2]
  const float2* rtx;       // e^{-2 pi i k / nx}, k = 0..nx/2
  const int* posx;         // position holding frequency k (k < nx/2) after the forward DFT
  const int* fqx;          // frequency held at position p (inverse of posx)
  const float2* twy;       // stage twiddles of the y lane plan [yr1, yr2]
  unsigned* status;        // device status word (bit 1: a bounded wait expired) or null
  // adaptive restart (restart != 0): the factor forming w_hat^k is
  // beta_dev[k] (k = the iteration this pass starts); the pass that starts
  // iteration k >= 1 sums c_{k-1} = ||w^{k-1} - w_hat^{k-1}||^2 +
  // ||b^{k-1} - b_hat^{k-1}||^2, and its last CTA applies the rule to
  // beta_dev[k+1 ..]; u^k = w_hat^k - b_hat^k is kept in u_prev for that sum
  int restart;
  int k, kmax;             // iteration started by this pass; last iteration of the loop
  float eta;
  float* beta_dev;         // [kmax + 1] factors in use (reset by the k = 0 pass)
  const float* beta_seq;   // [kmax + 1] beta_0 = 0, beta_1, ... (Eq. 5)
  float* u_prev;           // [3][V] u^{k-1} in, u^k out
  double* racc;            // [0] running sum of the pass, [1] cbar
  unsigned* rwords;        // [0] CTAs of the pass that have reported, [1] restarts counted
  int zper;                // z-planes per cluster in one launch (1, or 2 for half the clusters)
  FastDiv qdiv;            // division by nx / 4 (voxel quads per row)
  int nx, ny, nz, nkx, mx;  // mx = nx / 2
  int xr1, xr2, yr1, yr2;
  float beta, theta, eps;
  int data_term;
  SlabAdj adj;             // modes SLAB_ADJ, SLAB_ADJ_LAST
};

// Whether the slab path has kernels for this grid and plans (x: nx/2 split
// [xr1, 8]; y, z: lane plans), and its shared memory per CTA.
bool slab_supported(int nx, int ny, int nz, const AxisPlan& pxh, const AxisPlan& py,
                    const AxisPlan& pz);
size_t slab_smem_bytes(const SlabArgs& a);
cudaError_t launch_slab(int mode, const SlabArgs& a, cudaStream_t s);
// Clusters of the slab pass that the current device holds at once for grid a.
cudaError_t slab_max_clusters(const SlabArgs& a, int* clusters);
// z-pass of the slab layout (uses spec, twz, Kx, Ky, Kz, pz, ny, nz, nkx,
// order_n, gamma, scale of the pencil arguments)
cudaError_t launch_zslab(const PencilArgs& a, cudaStream_t s);
cudaError_t configure_slab_kernels();
// Many grids in one launch (batched handles): pairs[p] for the CTAs / blocks
// [start[p], start[p+1]); the slab pass's CTAs per pair are 3 nz_p, the z-pass
// blocks per pair zslab_blocks(); every pair of one z-pass launch shares the
// z plan [r1, r2].  smem: the largest pair's slab_smem_bytes.
cudaError_t launch_slab_multi(int mode, const SlabArgs* pairs, const int* start, int npairs,
                              int total_ctas, size_t smem, float beta, int k, cudaStream_t s);
int zslab_blocks(const PencilArgs& a);
cudaError_t launch_zslab_multi(int r1, int r2, const PencilArgs* pairs, const int* start, int npairs,
                               int total_blocks, cudaStream_t s);

constexpr unsigned kStatusNonfinite = 1u;
constexpr unsigned kStatusTimeout = 2u;

// Threshold stopping (Sec. 4, second version): words of a handle's `conv`
// array.  A kernel of the inner loop returns at once when kConvInner or
// kConvOuter is set; a kernel of the outer step when kConvOuter is set.
enum ConvWord : int {
  kConvInner = 0,      // the ADMM residual met admm_tol in this outer step
  kConvOuter = 1,      // the warped-image change met warp_tol
  kConvPlaneDone = 2,  // CTAs of the measuring plane pass that have reported
  kConvWarpDone = 3,   // blocks of the measuring re-warp that have reported
  kConvAdmmRun = 4,    // ADMM iterations run (all outer steps)
  kConvOuterRun = 5,   // outer steps run
  kConvWords = 8
};

// One block waits (bounded, `attempts` tries) on a barrier nothing arrives at.
cudaError_t launch_wait_selftest(unsigned* status, int attempts, cudaStream_t s);

// Fill the FastDiv fields and pitches of the pass arguments from the sizes.
void finish_plane_args(PlaneArgs& a);
void finish_pencil_args(PencilArgs& a);
// Encode a.zmap for a.spec (host only; needs finish_pencil_args first).
cudaError_t encode_pencil_map(PencilArgs& a);
// Encode a.smap for a.spec (host only; needs finish_plane_args first).
cudaError_t encode_plane_map(PlaneArgs& a);

// Fused y/z/y pass (pencil_fused.cu): one cluster of two CTAs per (comp, kx).
bool fused_pencil_supported(const PencilArgs& a);
size_t fused_pencil_smem(const PencilArgs& a);
cudaError_t configure_fused_pencil();
cudaError_t launch_fused_pencil(const PencilArgs& a, cudaStream_t s);

// Lane-FFT y/z passes (lane_passes.cu) for two-stage plans [R1, R2 in {8, 16}].
bool lane_y_supported(const PencilArgs& a);
bool lane_z_supported(const PencilArgs& a);
cudaError_t launch_lane_y(const PencilArgs& a, bool inv, cudaStream_t s);
cudaError_t launch_lane_z(const PencilArgs& a, cudaStream_t s);

// mode = InMode * 4 + prev * 2 + step
cudaError_t launch_plane(int in_mode, bool prev, bool step, const PlaneArgs& a, cudaStream_t s);
cudaError_t launch_pencil(const PencilArgs& a, cudaStream_t s);
size_t plane_smem_bytes(const PlaneArgs& a, int in_mode, bool prev, bool step);
size_t plane_smem_max(const PlaneArgs& a);
size_t pencil_smem_bytes(const PencilArgs& a);
int rows_per_tile(int ny);
cudaError_t configure_admm_kernels(size_t plane_smem, size_t pencil_smem);
// configure_admm_kernels(227 KB, 227 KB) on the current device, once per device.
cudaError_t configure_admm_kernels_on_current_device();

// ---------------------------------------------------------------- launch helpers
// Programmatic dependent launch: every kernel is launched with programmatic
// stream serialisation, waits on the previous kernel with pdl_wait() before
// touching its outputs, and lets the next kernel start (pdl_trigger) only
// after that wait -- so a kernel's prologue never overlaps the kernel that
// produced its inputs, only the one after it.
#if defined(__CUDACC__)
__device__ __forceinline__ void pdl_wait() {
#if defined(__CUDA_ARCH__)
  asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}
__device__ __forceinline__ void pdl_trigger() {
#if defined(__CUDA_ARCH__)
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// A launch that starts only once the previous kernel on the stream has
// completed (no programmatic overlap): for cluster kernels that need the
// whole GPU free to place every cluster in one wave.
template <typename... KArgs, typename... Args>
cudaError_t launch_whole(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                         cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = nullptr;
  cfg.numAttrs = 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}
#endif

// ---------------------------------------------------------------- grid ops
// zv: z-slices per thread of the re-warp, gradient and compose kernels (1, 2
// or 4; a tuned plan choice, same results)
struct Dims {
  int nx, ny, nz;
  int zv = 1;
};

// red_reset (or null): two words zeroed for the next bound reduction
cudaError_t launch_warp(Dims d, const float* I1, const float* u, float* I1w, unsigned* red_reset,
                        cudaStream_t s);
cudaError_t launch_grad_residual(Dims d, const float* I1w, const float* I0, float* J, float* c,
                                 cudaStream_t s);
// red[0] = bits of max |w|_inf, red[1] = bits of max ||Dw||_inf (must start at 0)
cudaError_t launch_bound_reduce(Dims d, const float* w, unsigned* red, cudaStream_t s,
                                const unsigned* conv = nullptr);
// s from red; u_out = s w + u_in(x + s w); status |= 1 on non-finite maxima;
// with conv[kConvOuter] set: u_out = u_in
cudaError_t launch_compose(Dims d, const float* w, const float* u_in, float* u_out,
                           const unsigned* red, float kappa, float delta, unsigned* status,
                           float* scale_out, cudaStream_t s, unsigned* conv = nullptr);
// Re-warp that also measures the change of I1w against its previous content
// (conv_acc[2..3]) and sets conv[kConvOuter] when it is <= warp_tol; skipped
// when conv[kConvOuter] is already set.
cudaError_t launch_warp_measured(Dims d, const float* I1, const float* u, float* I1w,
                                 unsigned* red_reset, unsigned* conv, double* conv_acc,
                                 float warp_tol, bool measure, cudaStream_t s);
cudaError_t launch_grad_residual_conv(Dims d, const float* I1w, const float* I0, float* J, float* c,
                                      const unsigned* conv, cudaStream_t s);
cudaError_t launch_jacobian(Dims d, const float* u, float* det, unsigned* count, cudaStream_t s);
// pyramid: 2 x 2 x 2 block average onto `coarse`; cell-centred doubling upsample of u
cudaError_t launch_downsample2(Dims coarse, const float* fine, float* out, cudaStream_t s);
cudaError_t launch_upsample_u(Dims coarse, Dims fine, const float* uc, float* uf, cudaStream_t s);

// ---------------------------------------------------------------- reverse mode
// One reverse ADMM step k (grad_kernels.cu).  From the forward sweep: wk =
// w^k, uk = w_hat^k - b_hat^k.  g_in = wbar^k - bbar^k, Sg = S g_in, Bk =
// bbar^k.  Adds into W1bar/B1bar (k-1, null for k = 0), stores the first
// contribution to W2bar/B2bar (k-2, null for k < 2), writes g_out =
// wbar^{k-1} - bbar^{k-1}, accumulates gJ, gc and acc[1] (theta, data
// step), acc[2] (gamma).
struct AdjArgs {
  Dims d;
  const float *wk, *uk;
  const float *J, *c, *Sg, *g_in, *Bk;
  float *W1bar, *B1bar, *W2bar, *B2bar, *g_out;
  float *gJ, *gc;
  double* acc;
  float beta;       // beta'_k (0 for k = 0)
  float theta;
  float inv_gamma;  // theta / lambda
};

// acc[0] += <vbar, w> (gradient of the bound scale)
cudaError_t launch_compose_vjp(Dims d, const float* u_o, const float* w, const unsigned* red,
                               float kappa, float delta, const float* ubar, float* ubar_prev,
                               float* wbar, double* acc, cudaStream_t s);
// count must start at 0
cudaError_t launch_bound_vjp(Dims d, const float* w, const unsigned* red, float kappa,
                             float delta, const double* acc, unsigned* count, float* wbar,
                             cudaStream_t s);
cudaError_t launch_adj_step(const AdjArgs& a, cudaStream_t s);
cudaError_t launch_linearise_vjp(Dims d, const float* I1, const float* u_o, const float* gJ,
                                 const float* gc, float* grad_fixed, float* grad_moving,
                                 const float* ubar_prev, float* ubar_out, cudaStream_t s);
cudaError_t launch_param_grads(const double* acc, float lambda, float theta, float* glam,
                               float* gtheta, cudaStream_t s);
// *loss = acc[0] after acc[0] += 1/2 sum r^2 (acc[0] must start at 0)
cudaError_t launch_ssd(Dims d, const float* I0, const float* I1, const float* u, double* acc,
                       float* loss, cudaStream_t s);
cudaError_t launch_ssd_vjp(Dims d, const float* I0, const float* I1, const float* u,
                           const float* gL, float* grad_fixed, float* grad_moving, float* grad_u,
                           cudaStream_t s);

}  // namespace nadmm
