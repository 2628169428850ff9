// C ABI (include/nadmm.h): validation, workspace layout, FFT tables, the
// outer/inner loop schedule and its CUDA-graph capture.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/nadmm.h"
#include "nadmm_internal.h"
#include "plan.h"

using namespace nadmm;

namespace {

thread_local std::string g_err;

nadmm_status fail(nadmm_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

nadmm_status cuda_fail(cudaError_t e, const char* where) {
  return fail(NADMM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

constexpr size_t kAlign = 256;
constexpr size_t kMaxSmem = 227 * 1024;  // opt-in dynamic shared memory per CTA
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

struct nadmm_context {
  nadmm_config cfg;
  AxisPlan px, py, pz;
  std::vector<float2> twx, twy, twz;
  std::vector<int> posx;
  std::vector<float> Kx, Ky, Kz;
  std::vector<float> beta;   // beta_0 .. beta_{K-1}
  // slab path (two kernels per ADMM iteration): nx/2-point x plan, its
  // twiddles, positions and their inverse, and e^{-2 pi i k / nx}
  bool slab = false;      // the grid supports the slab path (its tables exist)
  bool use_slab = false;  // ... and runs it (decided when the workspace is attached)
  AxisPlan pxh;
  std::vector<float2> twxh, rtx;
  std::vector<int> posxh, fqxh;
  size_t o_twxh = 0, o_rtx = 0, o_posxh = 0, o_fqxh = 0;
  // adaptive restart (cfg.restart_eta >= 0, slab path only): u^k (state
  // region), the factors in use, beta_0.., the sums and the counters (tables)
  bool restart = false;
  size_t o_uprev = 0, o_bdev = 0, o_bseq = 0, o_racc = 0, o_rwords = 0;
  int R = 0;
  size_t V = 0, nkx = 0;
  size_t plane_smem = 0, pencil_smem = 0;
  // Workspace: a state region (fields and spectrum, offsets o_spec..o_io_u
  // from ws) and a table region (status/reduction words and FFT tables,
  // offsets o_red..o_Kz from wt).  A single handle places the tables right
  // after the state; the pairs of a batched handle that run one after
  // another on the same lane share one state region and own their tables.
  size_t o_spec, o_y, o_wp, o_bp, o_J, o_c, o_I1w, o_ut, o_io_f, o_io_m, o_io_u, state_total;
  // reverse mode (NADMM_FLAG_SAVE_FOR_BACKWARD): u at the start of every
  // outer step, the ADMM history w^k, b^k of one outer step, the rotating
  // adjoint slots wbar/bbar (3 each) and the adjoint work fields
  size_t o_tape = 0, o_hist = 0, o_adj = 0, o_g = 0, o_Sg = 0, o_gJ = 0, o_gc = 0, o_ub0 = 0,
         o_ub1 = 0;
  bool saved_forward = false;
  bool has_tape = false;  // o_tape (table region) is allocated
  size_t o_red, o_acc, o_conv, o_convacc, o_twx, o_twy, o_twz, o_posx, o_Kx, o_Ky, o_Kz, table_total;
  size_t total;  // single handle: align(state_total) + table_total
  char* ws = nullptr;
  char* wt = nullptr;
  CUtensorMap zmap;  // z-pass tensor map of the workspace spectrum
  CUtensorMap smap;  // plane-pass tensor map of the workspace spectrum
  bool smap_ok = false;
  // graph cache: slot 0 the forward registration, slot 1 the backward
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  std::vector<const void*> gkey[2];
  cudaStream_t cap = nullptr;
  // batched handle: the pairs, their lane (concurrent graph branch) and
  // the byte offsets of each lane's state and each pair's tables
  bool batched = false;
  // pyramid handle (Sec. 4): pairs[l] is level l (0 = finest), all levels
  // share one state region; lvl_off[l] holds I0_l, I1_l, u_l, u_up_l
  bool pyramid = false;
  std::vector<size_t> lvl_off;
  std::vector<nadmm_context*> pairs;
  int lanes = 0;
  std::vector<int> lane_of;
  std::vector<size_t> lane_off, tab_off;
  std::vector<cudaStream_t> lane_cap;
  std::vector<cudaEvent_t> lane_ev;  // [0] fork, [1 + l] join of lane l
  // flat batched execution: every pair has its own state region and each
  // phase of the iteration is one launch over all pairs (the slab pass) or
  // one launch per z plan (the z-pass); device tables at o_flat
  bool flat = false;
  struct ZGroup {
    int r1, r2, first, count, blocks;  // pairs zorder[first .. first+count)
  };
  std::vector<ZGroup> zgroups;
  std::vector<int> zorder;
  // slab-pass launches: pairs grouped by shared-memory class (two CTAs per
  // SM or one), so small planes keep their occupancy, and a class of a few
  // waves into launches of one wave each (upload_flat); blocks = CTAs
  struct SGroup {
    int first, count, blocks;
    size_t smem;
  };
  std::vector<SGroup> sgroups;
  std::vector<int> sorder;
  size_t o_flat = 0, o_flat_args = 0, o_flat_final = 0, o_flat_start = 0, o_flat_pencil = 0,
         o_flat_zstart = 0;

  template <class T>
  T* at(size_t off) const { return reinterpret_cast<T*>(ws + off); }
  template <class T>
  T* tab(size_t off) const { return reinterpret_cast<T*>(wt + off); }
};

namespace {

// NVTX range over one public call (host side: the enqueue or graph launch,
// and the waits of the host-buffer path); free when no tool is attached.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

// Prime factors above 7 get generic FFT stages: at most kMaxStages of them,
// each at most kMaxPrime.
bool good_factors(int n) {
  int big[kMaxStages], smooth = 1;
  const int cnt = generic_primes(n, big, kMaxStages, smooth);
  return cnt == 0 || (cnt <= kMaxStages && big[cnt - 1] <= kMaxPrime);
}

void invalidate_graph(nadmm_context* h) {
  for (int k = 0; k < 2; ++k) {
    if (h->gexec[k]) cudaGraphExecDestroy(h->gexec[k]);
    h->gexec[k] = nullptr;
    h->gkey[k].clear();
  }
}

nadmm_status validate(const nadmm_config* c) {
  if (!c) return fail(NADMM_ERR_INVALID_ARG, "config is NULL");
  if (c->nx < 4 || c->ny < 4 || c->nz < 4)
    return fail(NADMM_ERR_UNSUPPORTED_SIZE, "every dimension must be >= 4");
  if (c->nx % 4 != 0) return fail(NADMM_ERR_UNSUPPORTED_SIZE, "nx must be a multiple of 4");
  if (c->ny % 2 != 0) return fail(NADMM_ERR_UNSUPPORTED_SIZE, "ny must be even");
  if (!good_factors(c->nx) || !good_factors(c->ny) || !good_factors(c->nz))
    return fail(NADMM_ERR_UNSUPPORTED_SIZE, "every prime factor of a dimension must be <= 509");
  if (c->order_n < 1 || c->order_n > 8) return fail(NADMM_ERR_INVALID_ARG, "order_n must be in 1..8");
  if (!(c->lambda >= 0.0f) || !std::isfinite(c->lambda))
    return fail(NADMM_ERR_INVALID_ARG, "lambda must be finite and >= 0");
  if (!(c->theta > 0.0f) || !std::isfinite(c->theta))
    return fail(NADMM_ERR_INVALID_ARG, "theta must be finite and > 0");
  if (c->outer_iters < 1 || c->inner_iters < 1)
    return fail(NADMM_ERR_INVALID_ARG, "iteration counts must be >= 1");
  if (c->data_term != 1 && c->data_term != 2)
    return fail(NADMM_ERR_INVALID_ARG, "data_term must be 1 or 2");
  if (!(c->eps > 0.0f) || !std::isfinite(c->eps)) return fail(NADMM_ERR_INVALID_ARG, "eps must be > 0");
  if (!(c->admm_tol >= 0.0f) || !std::isfinite(c->admm_tol) || !(c->warp_tol >= 0.0f) ||
      !std::isfinite(c->warp_tol))
    return fail(NADMM_ERR_INVALID_ARG, "admm_tol and warp_tol must be finite and >= 0");
  if ((c->admm_tol > 0.0f || c->warp_tol > 0.0f) && (c->flags & NADMM_FLAG_SAVE_FOR_BACKWARD))
    return fail(NADMM_ERR_INVALID_ARG, "the reverse mode needs fixed iteration counts (no thresholds)");
  if (std::isnan(c->restart_eta))
    return fail(NADMM_ERR_INVALID_ARG, "restart_eta must not be NaN (< 0 turns restart off)");
  if (c->restart_eta >= 0.0f && ((c->flags & NADMM_FLAG_SAVE_FOR_BACKWARD) ||
                                 c->admm_tol > 0.0f || c->warp_tol > 0.0f))
    return fail(NADMM_ERR_INVALID_ARG,
                "adaptive restart needs fixed iteration counts and no reverse mode");
  if (!(c->bound_kappa > 0.0f) || !(c->bound_delta > 0.0f))
    return fail(NADMM_ERR_INVALID_ARG, "bound_kappa and bound_delta must be > 0 (INFINITY disables)");
  if (c->flags & ~(NADMM_FLAG_NO_GRAPH | NADMM_FLAG_SAVE_FOR_BACKWARD | NADMM_FLAG_LANE_MASK |
                   NADMM_FLAG_FUSED_PENCIL | NADMM_FLAG_PIPELINED_PLANE | NADMM_FLAG_FOUR_PASS |
                   NADMM_FLAG_SLAB_PATH | NADMM_FLAG_OUTER_MASK | NADMM_FLAG_SLAB_PAIRS))
    return fail(NADMM_ERR_INVALID_ARG, "unknown flag bits");
  if ((c->flags & NADMM_FLAG_OUTER_MASK) == NADMM_FLAG_OUTER_MASK)
    return fail(NADMM_ERR_INVALID_ARG, "NADMM_FLAG_OUTER_Z2 and NADMM_FLAG_OUTER_Z4 exclude each other");
  if ((c->flags & NADMM_FLAG_FOUR_PASS) && (c->flags & NADMM_FLAG_SLAB_PATH))
    return fail(NADMM_ERR_INVALID_ARG, "NADMM_FLAG_FOUR_PASS and NADMM_FLAG_SLAB_PATH exclude each other");
  for (int ax = 0; ax < 3; ++ax)
    if (((c->flags >> NADMM_FLAG_LANE_SHIFT(ax)) & 3u) == 3u)
      return fail(NADMM_ERR_INVALID_ARG, "plan bits of an axis ask for both 8 and 16 lanes");
  return NADMM_OK;
}

void compute_beta(nadmm_context* h) {
  // Eq. 5: alpha^0 = 1, alpha^{k+1} = (1 + sqrt(1 + 4 alpha_k^2)) / 2,
  // beta_k = (alpha^k - 1) / alpha^{k+1}; evaluated in double on the host.
  int K = h->cfg.inner_iters + 1;
  h->beta.assign(K, 0.0f);
  double a = 1.0;
  for (int k = 0; k < K; ++k) {
    double an = (1.0 + std::sqrt(1.0 + 4.0 * a * a)) / 2.0;
    h->beta[k] = (float)((a - 1.0) / an);
    a = an;
  }
}

float beta_for(const nadmm_context* h, int k) {  // factor used to form w_hat^k
  if (k <= 0) return 0.0f;
  if (k - 1 < (int)h->beta.size()) return h->beta[k - 1];
  double a = 1.0, b = 0.0;
  for (int i = 0; i < k; ++i) {
    double an = (1.0 + std::sqrt(1.0 + 4.0 * a * a)) / 2.0;
    b = (a - 1.0) / an;
    a = an;
  }
  return (float)b;
}

bool thresholds(const nadmm_context* h) { return h->cfg.admm_tol > 0.0f || h->cfg.warp_tol > 0.0f; }

PlaneArgs plane_args(const nadmm_context* h) {
  PlaneArgs a;
  std::memset(&a, 0, sizeof(a));
  a.spec = h->at<float2>(h->o_spec);
  a.y = h->at<float>(h->o_y);
  a.wp = h->at<float>(h->o_wp);
  a.bp = h->at<float>(h->o_bp);
  a.J = h->at<float>(h->o_J);
  a.c = h->at<float>(h->o_c);
  a.twx = h->tab<float2>(h->o_twx);
  a.posx = h->tab<int>(h->o_posx);
  a.px = h->px;
  a.nx = h->cfg.nx;
  a.ny = h->cfg.ny;
  a.nz = h->cfg.nz;
  a.nkx = (int)h->nkx;
  a.status = h->tab<unsigned>(h->o_red) + 2;
  a.theta = h->cfg.theta;
  a.eps = h->cfg.eps;
  a.data_term = h->cfg.data_term;
  finish_plane_args(a);
  a.smap = h->smap;
  if (!h->smap_ok) a.spec_tma = 0;
  a.pipe = (h->cfg.flags & NADMM_FLAG_PIPELINED_PLANE) ? 1 : 0;
  if (thresholds(h)) {
    a.conv = h->tab<unsigned>(h->o_conv);
    a.conv_acc = h->tab<double>(h->o_convacc);
    a.admm_tol = h->cfg.admm_tol;
  }
  return a;
}

PencilArgs pencil_args(const nadmm_context* h) {
  PencilArgs a;
  std::memset(&a, 0, sizeof(a));
  a.spec = h->at<float2>(h->o_spec);
  a.twy = h->tab<float2>(h->o_twy);
  a.twz = h->tab<float2>(h->o_twz);
  a.Kx = h->tab<float>(h->o_Kx);
  a.Ky = h->tab<float>(h->o_Ky);
  a.Kz = h->tab<float>(h->o_Kz);
  a.py = h->py;
  a.pz = h->pz;
  a.ny = h->cfg.ny;
  a.nz = h->cfg.nz;
  a.nkx = (int)h->nkx;
  a.status = h->tab<unsigned>(h->o_red) + 2;
  a.order_n = h->cfg.order_n;
  a.gamma = h->cfg.lambda / h->cfg.theta;
  a.scale = (float)(1.0 / ((double)h->cfg.nx * h->cfg.ny * h->cfg.nz));
  finish_pencil_args(a);
  if (h->cfg.flags & NADMM_FLAG_FUSED_PENCIL) a.fused = fused_pencil_supported(a) ? 1 : 0;
  a.zmap = h->zmap;
  if (thresholds(h)) a.conv = h->tab<unsigned>(h->o_conv);
  return a;
}

SlabArgs slab_args(const nadmm_context* h) {
  SlabArgs a;
  std::memset(&a, 0, sizeof(a));
  a.spec = h->at<float2>(h->o_spec);
  a.y = h->at<float>(h->o_y);
  a.wp = h->at<float>(h->o_wp);
  a.bp = h->at<float>(h->o_bp);
  a.J = h->at<float>(h->o_J);
  a.c = h->at<float>(h->o_c);
  a.twx = h->tab<float2>(h->o_twxh);
  a.rtx = h->tab<float2>(h->o_rtx);
  a.posx = h->tab<int>(h->o_posxh);
  a.fqx = h->tab<int>(h->o_fqxh);
  a.twy = h->tab<float2>(h->o_twy);
  a.status = h->tab<unsigned>(h->o_red) + 2;
  a.nx = h->cfg.nx;
  a.ny = h->cfg.ny;
  a.nz = h->cfg.nz;
  a.nkx = (int)h->nkx;
  a.mx = h->cfg.nx / 2;
  a.qdiv = make_fastdiv((uint32_t)(h->cfg.nx / 4));
  a.zper = (h->cfg.flags & NADMM_FLAG_SLAB_PAIRS) ? 2 : 1;
  a.xr1 = h->pxh.radix[0];
  a.xr2 = h->pxh.radix[1];
  a.yr1 = h->py.radix[0];
  a.yr2 = h->py.radix[1];
  a.theta = h->cfg.theta;
  a.eps = h->cfg.eps;
  a.data_term = h->cfg.data_term;
  if (h->restart) {
    a.restart = 1;
    a.eta = h->cfg.restart_eta;
    a.kmax = h->cfg.inner_iters - 1;
    a.beta_dev = h->tab<float>(h->o_bdev);
    a.beta_seq = h->tab<float>(h->o_bseq);
    a.u_prev = h->at<float>(h->o_uprev);
    a.racc = h->tab<double>(h->o_racc);
    a.rwords = h->tab<unsigned>(h->o_rwords);
  }
  return a;
}

Dims dims_of(const nadmm_context* h) {
  Dims d{h->cfg.nx, h->cfg.ny, h->cfg.nz};
  const uint32_t z = h->cfg.flags & NADMM_FLAG_OUTER_MASK;
  d.zv = z == NADMM_FLAG_OUTER_Z4 ? 4 : z == NADMM_FLAG_OUTER_Z2 ? 2 : 1;
  return d;
}

#define TRY(expr)                                  \
  do {                                             \
    cudaError_t e_ = (expr);                       \
    if (e_ != cudaSuccess) return e_;              \
  } while (0)

// Optional per-kernel timing: events recorded on the launch stream around
// every kernel of a direct-launch run (never active during graph capture).
struct Profiler {
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> marks;
  cudaError_t begin(int kc, cudaStream_t s, cudaEvent_t& start) {
    TRY(cudaEventCreate(&start));
    cudaError_t e = cudaEventRecord(start, s);
    if (e != cudaSuccess) cudaEventDestroy(start);
    return e;
  }
  cudaError_t end(int kc, cudaStream_t s, cudaEvent_t start) {
    cudaEvent_t stop;
    TRY(cudaEventCreate(&stop));
    cudaError_t e = cudaEventRecord(stop, s);
    marks.push_back({kc, {start, stop}});
    return e;
  }
  void release() {
    for (auto& m : marks) {
      cudaEventDestroy(m.second.first);
      cudaEventDestroy(m.second.second);
    }
    marks.clear();
  }
};
thread_local Profiler* g_prof = nullptr;

// Launch `expr` as kernel class kc, bracketed by events when profiling.
#define KLAUNCH(kc, s, expr)                          \
  do {                                                \
    cudaEvent_t st_ = nullptr;                        \
    if (g_prof) TRY(g_prof->begin((kc), (s), st_));   \
    TRY(expr);                                        \
    if (g_prof) TRY(g_prof->end((kc), (s), st_));     \
  } while (0)

// ADMM iterations k0 .. k0+steps-1 starting from `first` (plane pass that
// starts iteration k0), then the final inverse transform into w_out/b_out.
// With hist_w/hist_u (k0 = 0 only, the reverse-mode recompute), w^k and
// u^k = w_hat^k - b_hat^k of every iteration go to hist_w + k 3V and
// hist_u + k 3V: the plane passes write them directly (w^{k-1} by the tile
// stores, u^k by the point-wise step), w^{K-1} comes from the final pass.
// The same iterations on the slab path (two kernels per iteration); with
// hist_w/hist_u the slab passes write w^{k-1} to the history instead of the
// w state slot, read w^{k-2} from it, and record u^k.
cudaError_t enqueue_inner_slab(nadmm_context* h, const PlaneArgs& first, int in_first, bool prev_first,
                               int k0, int steps, const float* J, const float* c, float* w_out,
                               float* b_out, cudaStream_t s, float* hist_w = nullptr,
                               float* hist_u = nullptr) {
  const size_t F3 = 3 * h->V;
  SlabArgs a = slab_args(h);
  a.J = J;
  a.c = c;
  // restart runs over whole inner loops (k0 = 0); a loop resumed from given
  // state buffers (nadmm_admm_run) runs Eq. 5 as printed
  if (in_first != IN_NONE || k0 != 0) a.restart = 0;
  a.kmax = k0 + steps - 1;
  SlabArgs f = a;
  f.k = k0;
  int mode = SLAB_FIRST;
  if (in_first == IN_STATE) {
    mode = prev_first ? SLAB_STATE_PREV : SLAB_STATE;
    f.w_in = first.w_in;
    f.b_in = first.b_in;
    f.wprev_in = first.wprev_in;
    f.bprev_in = first.bprev_in;
  }
  f.beta = beta_for(h, k0);
  if (hist_w != nullptr) f.u_hist = hist_u + (size_t)k0 * F3;
  KLAUNCH(in_first == IN_NONE ? NADMM_KC_SLAB_FIRST : (prev_first ? NADMM_KC_SLAB : NADMM_KC_SLAB_K1),
          s, launch_slab(mode, f, s));
  const PencilArgs pa = pencil_args(h);
  for (int k = k0 + 1; k < k0 + steps; ++k) {
    KLAUNCH(NADMM_KC_ZSLAB, s, launch_zslab(pa, s));
    a.beta = beta_for(h, k);
    a.k = k;
    if (hist_w != nullptr) {  // w^{k-2} from the history, w^{k-1} into it, u^k recorded
      a.u_hist = hist_u + (size_t)k * F3;
      a.wp = hist_w + (size_t)(k >= 2 ? k - 2 : 0) * F3;  // k = 1 reads no w state
      a.wp_out = hist_w + (size_t)(k - 1) * F3;
    }
    KLAUNCH(k >= 2 ? NADMM_KC_SLAB : NADMM_KC_SLAB_K1, s,
            launch_slab(k >= 2 ? SLAB_SPEC_PREV : SLAB_SPEC, a, s));
  }
  KLAUNCH(NADMM_KC_ZSLAB, s, launch_zslab(pa, s));
  SlabArgs fin = a;
  fin.w_out = w_out;
  fin.b_out = b_out;
  fin.u_hist = nullptr;
  fin.wp_out = nullptr;
  if (b_out == nullptr) fin.y = nullptr;
  KLAUNCH(NADMM_KC_SLAB_FINAL, s, launch_slab(SLAB_FINAL, fin, s));
  return cudaSuccess;
}

cudaError_t enqueue_inner(nadmm_context* h, PlaneArgs first, int in_first, bool prev_first, int k0,
                          int steps, const float* J, const float* c, float* w_out, float* b_out,
                          cudaStream_t s, float* hist_w = nullptr, float* hist_u = nullptr) {
  if (h->use_slab && !thresholds(h) && (in_first == IN_NONE || in_first == IN_STATE) &&
      (hist_w == nullptr || (k0 == 0 && in_first == IN_NONE)))
    return enqueue_inner_slab(h, first, in_first, prev_first, k0, steps, J, c, w_out, b_out, s,
                              hist_w, hist_u);
  const size_t F3 = 3 * h->V;
  auto hw = [&](int k) { return hist_w + (size_t)k * F3; };
  first.J = J;
  first.c = c;
  first.beta = beta_for(h, k0);
  if (hist_w) first.u_hist = hist_u;
  KLAUNCH(in_first == IN_NONE ? NADMM_KC_PLANE_FIRST : (prev_first ? NADMM_KC_PLANE : NADMM_KC_PLANE_K1),
          s, launch_plane(in_first, prev_first, true, first, s));
  PencilArgs pa = pencil_args(h);
  PlaneArgs a = plane_args(h);
  a.J = J;
  a.c = c;
  for (int k = k0 + 1; k < k0 + steps; ++k) {
    KLAUNCH(NADMM_KC_PENCIL, s, launch_pencil(pa, s));
    a.beta = beta_for(h, k);
    if (hist_w) {  // w^{k-2} from the history, w^{k-1} into it, u^k recorded
      a.u_hist = hist_u + (size_t)k * F3;
      if (k == 1) {
        a.wp = hw(0);  // the k = 1 pass writes w^0 with per-thread stores
      } else {
        a.wp = hw(k - 2);
        a.w_tile_out = hw(k - 1);
      }
    }
    KLAUNCH(k >= 2 ? NADMM_KC_PLANE : NADMM_KC_PLANE_K1, s, launch_plane(IN_SPEC, k >= 2, true, a, s));
  }
  KLAUNCH(NADMM_KC_PENCIL, s, launch_pencil(pa, s));
  PlaneArgs fin = plane_args(h);
  fin.w_out = w_out;
  fin.b_out = b_out;
  if (b_out == nullptr) fin.y = nullptr;  // b^{K-1} not wanted: skip reading y
  KLAUNCH(NADMM_KC_PLANE_FINAL, s, launch_plane(IN_SPEC, false, false, fin, s));
  return cudaSuccess;
}

cudaError_t enqueue_register(nadmm_context* h, const float* I0, const float* I1, float* u_out,
                             cudaStream_t s, const float* u_init = nullptr) {
  const Dims d = dims_of(h);
  const size_t V = h->V;
  const int O = h->cfg.outer_iters, K = h->cfg.inner_iters;
  float* ut = h->at<float>(h->o_ut);
  float* I1w = h->at<float>(h->o_I1w);
  float* J = h->at<float>(h->o_J);
  float* c = h->at<float>(h->o_c);
  float* vbuf = h->at<float>(h->o_wp);  // velocity w^K reuses the w state slot
  unsigned* red = h->tab<unsigned>(h->o_red);
  // u ping-pongs between u_out and ut so that the last compose lands in u_out
  auto dst_of = [&](int o) { return ((O - 1 - o) % 2 == 0) ? u_out : ut; };
  float* u_cur = (dst_of(0) == u_out) ? ut : u_out;
  TRY(cudaMemsetAsync(red, 0, 4 * sizeof(unsigned), s));  // red[0..1], status red[2]
  if (h->restart) TRY(cudaMemsetAsync(h->tab<unsigned>(h->o_rwords), 0, 2 * sizeof(unsigned), s));
  unsigned* conv = thresholds(h) ? h->tab<unsigned>(h->o_conv) : nullptr;
  double* conv_acc = h->tab<double>(h->o_convacc);
  if (conv) {
    TRY(cudaMemsetAsync(conv, 0, kConvWords * sizeof(unsigned), s));
    TRY(cudaMemsetAsync(conv_acc, 0, 4 * sizeof(double), s));
  }
  if (u_init)  // start from a given displacement (a coarser pyramid level's)
    TRY(cudaMemcpyAsync(u_cur, u_init, 3 * V * sizeof(float), cudaMemcpyDeviceToDevice, s));
  else
    TRY(cudaMemsetAsync(u_cur, 0, 3 * V * sizeof(float), s));
  KLAUNCH(NADMM_KC_WARP, s, launch_warp(d, I1, u_cur, I1w, nullptr, s));
  KLAUNCH(NADMM_KC_GRAD, s, launch_grad_residual(d, I1w, I0, J, c, s));
  for (int o = 0; o < O; ++o) {
    if (h->has_tape)  // u at the start of outer step o, for the reverse sweep
      TRY(cudaMemcpyAsync(h->tab<float>(h->o_tape) + (size_t)o * 3 * V, u_cur, 3 * V * sizeof(float),
                          cudaMemcpyDeviceToDevice, s));
    PlaneArgs first = plane_args(h);
    TRY(enqueue_inner(h, first, IN_NONE, false, 0, K, J, c, vbuf, nullptr, s));
    // red[0..1] are zero here: cleared at the start, then by each re-warp
    KLAUNCH(NADMM_KC_BOUND, s, launch_bound_reduce(d, vbuf, red, s, conv));
    float* u_new = dst_of(o);
    KLAUNCH(NADMM_KC_COMPOSE, s,
            launch_compose(d, vbuf, u_cur, u_new, red, h->cfg.bound_kappa, h->cfg.bound_delta,
                           red + 2, nullptr, s, conv));
    u_cur = u_new;
    if (o + 1 < O) {
      KLAUNCH(NADMM_KC_WARP, s,
              launch_warp_measured(d, I1, u_cur, I1w, red, conv, conv_acc, h->cfg.warp_tol,
                                   conv != nullptr && h->cfg.warp_tol > 0.0f, s));
      KLAUNCH(NADMM_KC_GRAD, s, launch_grad_residual_conv(d, I1w, I0, J, c, conv, s));
    }
  }
  return cudaSuccess;
}

enum HandleKind { kSingle = 0, kBatched = 1, kPyramid = 2 };

int kind_of(const nadmm_context* h) { return h->batched ? kBatched : h->pyramid ? kPyramid : kSingle; }

nadmm_status need_ws(const nadmm_context* h, int want = kSingle) {
  if (!h) return fail(NADMM_ERR_INVALID_ARG, "handle is NULL");
  if (kind_of(h) != want) {
    static const char* const names[3] = {"a single-pair handle (nadmm_create)",
                                         "a batched handle (nadmm_create_batched)",
                                         "a pyramid handle (nadmm_create_pyramid)"};
    return fail(NADMM_ERR_INVALID_ARG, std::string("this call needs ") + names[want] + ", got " +
                                           names[kind_of(h)]);
  }
  if (!h->wt) return fail(NADMM_ERR_NO_WORKSPACE, "no workspace attached (nadmm_set_workspace)");
  return NADMM_OK;
}

nadmm_status check_dev_ptrs(std::initializer_list<const void*> ptrs) {
  for (const void* p : ptrs) {
    if (!p) return fail(NADMM_ERR_INVALID_ARG, "device pointer is NULL");
    if (!aligned16(p)) return fail(NADMM_ERR_ALIGNMENT, "device pointer not 16-byte aligned");
  }
  return NADMM_OK;
}

constexpr int kDefaultLanes = 2;
// Largest slab-pass shared memory that still leaves room for two CTAs per SM
// (228 KB per SM, 1 KB reserved per CTA).
constexpr size_t kSlabTwoPerSm = 113 * 1024;

// R2 tried first for an axis's lane plan: the flag bits, else the defaults
// measured on 128x128x96 (x 8, y 16, z 8).
int lane_first(uint32_t flags, int axis) {
  const uint32_t b = (flags >> NADMM_FLAG_LANE_SHIFT(axis)) & 3u;
  if (b == 1u) return 8;
  if (b == 2u) return 16;
  return axis == 1 ? 16 : 8;
}

// Plans, tables and the workspace layout of one grid (host memory only).
nadmm_status create_single(const nadmm_config* cfg, nadmm_context** out) {
  nadmm_status st = validate(cfg);
  if (st != NADMM_OK) return st;
  nadmm_context* h = new nadmm_context();
  h->cfg = *cfg;
  if (!factor_axis(cfg->nx, h->px, true, lane_first(cfg->flags, 0)) ||
      !factor_axis(cfg->ny, h->py, true, lane_first(cfg->flags, 1)) ||
      !factor_axis(cfg->nz, h->pz, true, lane_first(cfg->flags, 2))) {
    delete h;
    return fail(NADMM_ERR_UNSUPPORTED_SIZE, "no radix plan for these dimensions");
  }
  h->V = (size_t)cfg->nx * cfg->ny * cfg->nz;
  h->nkx = (size_t)cfg->nx / 2 + 1;
  {
    PlaneArgs pa;
    std::memset(&pa, 0, sizeof(pa));
    pa.nx = cfg->nx;
    pa.ny = cfg->ny;
    pa.nz = cfg->nz;
    pa.px = h->px;
    finish_plane_args(pa);
    PencilArgs qa;
    std::memset(&qa, 0, sizeof(qa));
    qa.ny = cfg->ny;
    qa.nz = cfg->nz;
    qa.nkx = (int)h->nkx;
    qa.py = h->py;
    qa.pz = h->pz;
    finish_pencil_args(qa);
    h->R = pa.R;
    h->plane_smem = plane_smem_max(pa);
    h->pencil_smem = pencil_smem_bytes(qa);
  }
  if (h->pencil_smem > kMaxSmem || h->plane_smem > kMaxSmem) {
    delete h;
    return fail(NADMM_ERR_UNSUPPORTED_SIZE,
                "a pass's shared-memory tile exceeds the 227 KB per CTA (nx too large)");
  }
  if (cfg->nz > 256) {
    delete h;
    return fail(NADMM_ERR_UNSUPPORTED_SIZE, "nz must be <= 256 (one TMA box spans the z axis)");
  }
  h->twx = axis_twiddles(h->px);
  h->twy = axis_twiddles(h->py);
  h->twz = axis_twiddles(h->pz);
  h->posx = pos_table(h->px);
  h->Kx = symbol_natural(cfg->nx, (int)h->nkx);
  h->Ky = symbol_by_position(h->py);
  h->Kz = symbol_by_position(h->pz);
  compute_beta(h);
  {
    const int mx = cfg->nx / 2;
    // the pipelined plane pass and the fused y/z pass are four-kernel variants
    const uint32_t four = NADMM_FLAG_FOUR_PASS | NADMM_FLAG_PIPELINED_PLANE | NADMM_FLAG_FUSED_PENCIL;
    if (!(cfg->flags & four) && mx % 8 == 0) {
      two_stage_plan(mx, mx / 8, 8, h->pxh);
      h->slab = slab_supported(cfg->nx, cfg->ny, cfg->nz, h->pxh, h->py, h->pz);
    }
    if (h->slab) {
      h->twxh = axis_twiddles(h->pxh);
      h->posxh = pos_table(h->pxh);
      h->fqxh.assign(mx, 0);
      for (int k = 0; k < mx; ++k) h->fqxh[h->posxh[k]] = k;
      const double two_pi = 6.283185307179586476925286766559;
      for (int k = 0; k <= mx; ++k) {
        const double a = -two_pi * (double)k / (double)cfg->nx;
        h->rtx.push_back(make_float2((float)std::cos(a), (float)std::sin(a)));
      }
    }
  }
  if (cfg->restart_eta >= 0.0f) {
    if (!h->slab) {
      delete h;
      return fail(NADMM_ERR_UNSUPPORTED_SIZE,
                  "adaptive restart runs on the slab path only (nx/2 a multiple of 8, lane "
                  "plans for y and z, a z-plane within one CTA, no NADMM_FLAG_FOUR_PASS)");
    }
    h->restart = true;
  }
  const size_t V = h->V;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t r = o;
    o = align_up(o + bytes);
    return r;
  };
  h->o_spec = take(3 * h->nkx * cfg->ny * cfg->nz * sizeof(float2));
  if (h->restart) h->o_uprev = take(3 * V * sizeof(float));
  h->o_y = take(3 * V * sizeof(float));
  h->o_wp = take(3 * V * sizeof(float));
  h->o_bp = take(3 * V * sizeof(float));
  h->o_J = take(3 * V * sizeof(float));
  h->o_c = take(V * sizeof(float));
  h->o_I1w = take(V * sizeof(float));
  h->o_ut = take(3 * V * sizeof(float));
  h->o_io_f = take(V * sizeof(float));
  h->o_io_m = take(V * sizeof(float));
  h->o_io_u = take(3 * V * sizeof(float));
  if (cfg->flags & NADMM_FLAG_SAVE_FOR_BACKWARD) {
    const size_t F3 = 3 * V * sizeof(float);
    h->o_hist = take(2 * (size_t)cfg->inner_iters * F3);
    h->o_adj = take(6 * F3);
    h->o_g = take(F3);
    h->o_Sg = take(F3);
    h->o_gJ = take(F3);
    h->o_gc = take(V * sizeof(float));
    h->o_ub0 = take(F3);
    h->o_ub1 = take(F3);
  }
  h->state_total = o;
  o = 0;
  h->o_red = take(4 * sizeof(unsigned));
  h->o_acc = take(4 * sizeof(double));
  h->o_conv = take(kConvWords * sizeof(unsigned));
  h->o_convacc = take(4 * sizeof(double));
  h->o_twx = take(h->twx.size() * sizeof(float2));
  h->o_twy = take(h->twy.size() * sizeof(float2));
  h->o_twz = take(h->twz.size() * sizeof(float2));
  h->o_posx = take(h->posx.size() * sizeof(int));
  h->o_Kx = take(h->Kx.size() * sizeof(float));
  h->o_Ky = take(h->Ky.size() * sizeof(float));
  h->o_Kz = take(h->Kz.size() * sizeof(float));
  if (h->slab) {
    h->o_twxh = take(h->twxh.size() * sizeof(float2));
    h->o_rtx = take(h->rtx.size() * sizeof(float2));
    h->o_posxh = take(h->posxh.size() * sizeof(int));
    h->o_fqxh = take(h->fqxh.size() * sizeof(int));
  }
  if (h->restart) {
    h->o_bdev = take((size_t)cfg->inner_iters * sizeof(float));
    h->o_bseq = take((size_t)cfg->inner_iters * sizeof(float));
    h->o_racc = take(2 * sizeof(double));
    h->o_rwords = take(2 * sizeof(unsigned));
  }
  // the tape belongs to the pair (it must outlive other pairs' use of a
  // shared state region), so it sits with the tables
  if (cfg->flags & NADMM_FLAG_SAVE_FOR_BACKWARD) {
    h->has_tape = true;
    h->o_tape = take((size_t)cfg->outer_iters * 3 * V * sizeof(float));
  }
  h->table_total = o;
  *out = h;
  return NADMM_OK;
}

void destroy_context(nadmm_context* h) {
  if (!h) return;
  invalidate_graph(h);
  if (h->cap) cudaStreamDestroy(h->cap);
  for (cudaStream_t s : h->lane_cap) cudaStreamDestroy(s);
  for (cudaEvent_t e : h->lane_ev) cudaEventDestroy(e);
  for (nadmm_context* p : h->pairs) destroy_context(p);
  delete h;
}

// Longest-first greedy split of the pairs over `lanes` graph branches
// (balanced by voxel count), then the batched workspace layout: one state
// region per lane, sized for its largest pair, followed by every pair's
// tables.
void assign_lanes(nadmm_context* b, int lanes) {
  const int n = (int)b->pairs.size();
  b->lanes = lanes;
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return b->pairs[x]->V > b->pairs[y]->V; });
  std::vector<size_t> load(lanes, 0), state(lanes, 0);
  b->lane_of.assign(n, 0);
  for (int i : order) {
    int best = 0;
    for (int l = 1; l < lanes; ++l)
      if (load[l] < load[best]) best = l;
    b->lane_of[i] = best;
    load[best] += b->pairs[i]->V;
    state[best] = std::max(state[best], b->pairs[i]->state_total);
  }
  size_t o = 0;
  b->lane_off.assign(lanes, 0);
  for (int l = 0; l < lanes; ++l) {
    b->lane_off[l] = o;
    o = align_up(o + state[l]);
  }
  b->tab_off.assign(n, 0);
  for (int i = 0; i < n; ++i) {
    b->tab_off[i] = o;
    o = align_up(o + b->pairs[i]->table_total);
  }
  b->total = o;
}

// Whether every pair of a batched handle can run flat: all on the slab path,
// no reverse-mode tape (the reverse sweep runs per pair on lanes).
bool flat_possible(const nadmm_context* b) {
  if (b->cfg.flags & NADMM_FLAG_SAVE_FOR_BACKWARD) return false;
  for (const nadmm_context* p : b->pairs)
    if (!p->slab) return false;
  return true;
}

// Flat layout: one state region per pair, every pair's tables, then the
// launch tables (per-pair slab arguments for the passes and for the final
// pass, CTA starts, per-pair z-pass arguments grouped by z plan, block starts).
void assign_flat(nadmm_context* b) {
  const int n = (int)b->pairs.size();
  assign_lanes(b, n);  // n lanes of one pair each: every pair its own state region
  b->flat = true;
  b->zorder.clear();
  b->zgroups.clear();
  for (int i = 0; i < n; ++i) {
    const AxisPlan& pz = b->pairs[i]->pz;
    bool found = false;
    for (auto& g : b->zgroups)
      if (g.r1 == pz.radix[0] && g.r2 == pz.radix[1]) found = true;
    if (found) continue;
    nadmm_context::ZGroup g{pz.radix[0], pz.radix[1], (int)b->zorder.size(), 0, 0};
    for (int j = i; j < n; ++j) {
      const AxisPlan& qz = b->pairs[j]->pz;
      if (qz.radix[0] == g.r1 && qz.radix[1] == g.r2) {
        b->zorder.push_back(j);
        ++g.count;
      }
    }
    b->zgroups.push_back(g);
  }
  // slab groups: planes that leave room for two CTAs per SM, then the rest
  b->sorder.clear();
  b->sgroups.clear();
  for (int cls = 0; cls < 2; ++cls) {
    nadmm_context::SGroup g{(int)b->sorder.size(), 0, 0, 0};
    for (int i = 0; i < n; ++i) {
      const size_t sm = slab_smem_bytes(slab_args(b->pairs[i]));
      if ((sm <= kSlabTwoPerSm) == (cls == 0)) {
        b->sorder.push_back(i);
        ++g.count;
      }
    }
    if (g.count) b->sgroups.push_back(g);
  }
  size_t o = b->total;
  b->o_flat = o;
  auto take = [&](size_t bytes) {
    size_t r = o;
    o = align_up(o + bytes);
    return r;
  };
  b->o_flat_args = take((size_t)n * sizeof(SlabArgs));
  b->o_flat_final = take((size_t)n * sizeof(SlabArgs));
  b->o_flat_start = take((size_t)(2 * n) * sizeof(int));  // at most one launch per pair
  b->o_flat_pencil = take((size_t)n * sizeof(PencilArgs));
  b->o_flat_zstart = take((size_t)(n + b->zgroups.size()) * sizeof(int));
  b->total = o;
}

// Lane count 0 means flat execution.
void relayout(nadmm_context* b, int lanes) {
  b->flat = false;
  if (lanes == 0)
    assign_flat(b);
  else
    assign_lanes(b, lanes);
}

// Every pass kernel may take up to the opt-in shared-memory limit; the
// attribute belongs to the device that is current when it is set, so it is
// raised to the maximum once per device and each launch asks for what its
// grid needs.
cudaError_t configure_kernels_once() { return configure_admm_kernels_on_current_device(); }

// Attach the state region ws and the table region wt to a single-grid
// context: upload the tables, clear the status words, encode the z-pass
// tensor map.
nadmm_status attach(nadmm_context* h, char* ws, char* wt) {
  invalidate_graph(h);
  h->saved_forward = false;
  h->ws = ws;
  h->wt = wt;
  struct Up { size_t off; const void* src; size_t n; } ups[] = {
      {h->o_twx, h->twx.data(), h->twx.size() * sizeof(float2)},
      {h->o_twy, h->twy.data(), h->twy.size() * sizeof(float2)},
      {h->o_twz, h->twz.data(), h->twz.size() * sizeof(float2)},
      {h->o_posx, h->posx.data(), h->posx.size() * sizeof(int)},
      {h->o_Kx, h->Kx.data(), h->Kx.size() * sizeof(float)},
      {h->o_Ky, h->Ky.data(), h->Ky.size() * sizeof(float)},
      {h->o_Kz, h->Kz.data(), h->Kz.size() * sizeof(float)},
      {h->o_twxh, h->twxh.data(), h->twxh.size() * sizeof(float2)},
      {h->o_rtx, h->rtx.data(), h->rtx.size() * sizeof(float2)},
      {h->o_posxh, h->posxh.data(), h->posxh.size() * sizeof(int)},
      {h->o_fqxh, h->fqxh.data(), h->fqxh.size() * sizeof(int)},
      {h->o_bseq, h->beta.data(), h->restart ? (size_t)h->cfg.inner_iters * sizeof(float) : 0},
  };
  cudaError_t e = cudaSuccess;
  for (const Up& u : ups) {
    if (u.n == 0) continue;
    e = cudaMemcpy(wt + u.off, u.src, u.n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) break;
  }
  if (e == cudaSuccess) e = cudaMemset(wt + h->o_red, 0, 4 * sizeof(unsigned));
  if (e != cudaSuccess) {
    h->ws = h->wt = nullptr;
    return cuda_fail(e, "upload of FFT tables");
  }
  PencilArgs pa = pencil_args(h);
  e = encode_pencil_map(pa);
  if (e != cudaSuccess) {
    h->ws = h->wt = nullptr;
    return cuda_fail(e, "cuTensorMapEncodeTiled");
  }
  h->zmap = pa.zmap;
  h->smap_ok = false;
  PlaneArgs sa = plane_args(h);
  if (sa.spec_tma) {
    e = encode_plane_map(sa);
    if (e != cudaSuccess) {
      h->ws = h->wt = nullptr;
      return cuda_fail(e, "cuTensorMapEncodeTiled (plane)");
    }
    h->smap = sa.smap;
    h->smap_ok = true;
  }
  // the slab path for this grid on its own: forced by the flag or by restart
  // (which only the slab path implements), else when its clusters fill the
  // device's waves well
  h->use_slab = false;
  if (h->slab) {
    if ((h->cfg.flags & (NADMM_FLAG_SLAB_PATH | NADMM_FLAG_SLAB_PAIRS)) || h->restart) {
      h->use_slab = true;
    } else {
      int clusters = 0;
      e = slab_max_clusters(slab_args(h), &clusters);
      if (e != cudaSuccess) {
        h->ws = h->wt = nullptr;
        return cuda_fail(e, "cudaOccupancyMaxActiveClusters");
      }
      const int ctas = 3 * h->cfg.nz, cap = 3 * std::max(clusters, 1);
      const int waves = (ctas + cap - 1) / cap;
      h->use_slab = (double)ctas >= 0.8 * (double)waves * (double)cap;
    }
  }
  return NADMM_OK;
}

// Read and clear one context's device status word (stream already synced).
nadmm_status read_status(nadmm_context* h) {
  unsigned word = 0;
  unsigned* dev = h->tab<unsigned>(h->o_red) + 2;
  cudaError_t e = cudaMemcpy(&word, dev, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(dev, 0, sizeof(unsigned));
  if (e != cudaSuccess) return cuda_fail(e, "status read");
  if (word & kStatusTimeout)
    return fail(NADMM_ERR_TIMEOUT, "a kernel's bounded wait for its bulk copies expired");
  if (word & kStatusNonfinite)
    return fail(NADMM_ERR_NONFINITE, "non-finite velocity met in the bound step");
  return NADMM_OK;
}

// Capture fn(stream) into h's graph (re-captured when key changes), then replay.
template <class F>
nadmm_status replay(nadmm_context* h, int slot, const std::vector<const void*>& key,
                    cudaStream_t stream, const char* what, F&& fn) {
  cudaGraphExec_t& gexec = h->gexec[slot];
  if (!gexec || h->gkey[slot] != key) {
    if (gexec) cudaGraphExecDestroy(gexec);
    gexec = nullptr;
    h->gkey[slot].clear();
    cudaError_t e;
    if (!h->cap) {
      e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreateWithFlags");
    }
    e = cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    cudaError_t le = fn(h->cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(h->cap, &g);
    if (le != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(le, what);
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      gexec = nullptr;
      return cuda_fail(e, "cudaGraphInstantiate");
    }
    h->gkey[slot] = key;
  }
  cudaError_t e = cudaGraphLaunch(gexec, stream);
  return e == cudaSuccess ? NADMM_OK : cuda_fail(e, "cudaGraphLaunch");
}

// The flat launch tables of a batched handle (after its pairs are attached).
// A class whose clusters fill at most four waves is split into launches of
// one wave each (a pair larger than that is a launch of its own): measured
// at three 128x128x96 pairs (three waves), one launch per pair took 7.4 ms
// per registration against 8.0 for one launch of all three.  Larger classes
// stay one launch, whose many waves pack uneven pairs densely (64 uneven
// pairs: 489 ms as one launch per phase, 657 ms split into waves).
cudaError_t upload_flat(nadmm_context* b) {
  const int n = (int)b->pairs.size();
  {
    std::vector<nadmm_context::SGroup> waves;
    for (const auto& g : b->sgroups) {
      int cap = 0;
      size_t smem = 0;
      const nadmm_context* widest = nullptr;
      for (int j = 0; j < g.count; ++j) {
        const nadmm_context* p = b->pairs[b->sorder[g.first + j]];
        const size_t sm = slab_smem_bytes(slab_args(p));
        if (widest == nullptr || sm > smem) {
          smem = sm;
          widest = p;
        }
      }
      TRY(slab_max_clusters(slab_args(widest), &cap));
      cap = std::max(cap, 1);
      int total = 0;
      for (int j = 0; j < g.count; ++j) total += b->pairs[b->sorder[g.first + j]]->cfg.nz;
      if (total > 4 * cap) {
        waves.push_back(nadmm_context::SGroup{g.first, g.count, 0, 0});
        continue;
      }
      nadmm_context::SGroup w{g.first, 0, 0, 0};
      int clusters = 0;
      for (int j = 0; j < g.count; ++j) {
        const int nz = b->pairs[b->sorder[g.first + j]]->cfg.nz;
        if (w.count > 0 && clusters + nz > cap) {
          waves.push_back(w);
          w = nadmm_context::SGroup{g.first + j, 0, 0, 0};
          clusters = 0;
        }
        ++w.count;
        clusters += nz;
      }
      if (w.count) waves.push_back(w);
    }
    b->sgroups = waves;
  }
  std::vector<SlabArgs> base(n), fin(n);
  std::vector<int> start(n + b->sgroups.size(), 0);
  for (size_t gi = 0; gi < b->sgroups.size(); ++gi) {
    auto& g = b->sgroups[gi];
    int ctas = 0;
    g.smem = 0;
    for (int j = 0; j < g.count; ++j) {
      nadmm_context* p = b->pairs[b->sorder[g.first + j]];
      SlabArgs& a = base[g.first + j];
      a = slab_args(p);
      fin[g.first + j] = a;
      fin[g.first + j].w_out = p->at<float>(p->o_wp);  // the velocity w^K, as in enqueue_register
      fin[g.first + j].b_out = nullptr;
      fin[g.first + j].y = nullptr;
      start[g.first + gi + j] = ctas;
      ctas += 3 * p->cfg.nz;
      g.smem = std::max(g.smem, slab_smem_bytes(a));
    }
    start[g.first + gi + g.count] = ctas;
    g.blocks = ctas;
  }
  std::vector<PencilArgs> pen(n);
  std::vector<int> zstart(n + b->zgroups.size(), 0);
  for (size_t gi = 0; gi < b->zgroups.size(); ++gi) {
    auto& g = b->zgroups[gi];
    int blocks = 0;
    for (int j = 0; j < g.count; ++j) {
      nadmm_context* p = b->pairs[b->zorder[g.first + j]];
      pen[g.first + j] = pencil_args(p);
      zstart[g.first + gi + j] = blocks;
      blocks += zslab_blocks(pen[g.first + j]);
    }
    zstart[g.first + gi + g.count] = blocks;
    g.blocks = blocks;
  }
  char* t = b->ws;
  TRY(cudaMemcpy(t + b->o_flat_args, base.data(), n * sizeof(SlabArgs), cudaMemcpyHostToDevice));
  TRY(cudaMemcpy(t + b->o_flat_final, fin.data(), n * sizeof(SlabArgs), cudaMemcpyHostToDevice));
  TRY(cudaMemcpy(t + b->o_flat_start, start.data(), start.size() * sizeof(int),
                 cudaMemcpyHostToDevice));
  TRY(cudaMemcpy(t + b->o_flat_pencil, pen.data(), n * sizeof(PencilArgs), cudaMemcpyHostToDevice));
  TRY(cudaMemcpy(t + b->o_flat_zstart, zstart.data(), zstart.size() * sizeof(int),
                 cudaMemcpyHostToDevice));
  return cudaSuccess;
}

// All pairs of a flat batched handle: per-pair outer-step kernels, one slab
// pass over all pairs and one z-pass per z plan for every ADMM iteration.
cudaError_t enqueue_batched_flat(nadmm_context* b, const float* const* I0, const float* const* I1,
                                 float* const* u_out, cudaStream_t s) {
  const int n = (int)b->pairs.size();
  const int O = b->cfg.outer_iters, K = b->cfg.inner_iters;
  nadmm_context* p0 = b->pairs[0];
  const SlabArgs* args = reinterpret_cast<const SlabArgs*>(b->ws + b->o_flat_args);
  const SlabArgs* fin = reinterpret_cast<const SlabArgs*>(b->ws + b->o_flat_final);
  const int* start = reinterpret_cast<const int*>(b->ws + b->o_flat_start);
  const PencilArgs* pen = reinterpret_cast<const PencilArgs*>(b->ws + b->o_flat_pencil);
  const int* zstart = reinterpret_cast<const int*>(b->ws + b->o_flat_zstart);
  auto dst_of = [&](int i, int o) {
    return ((O - 1 - o) % 2 == 0) ? u_out[i] : b->pairs[i]->at<float>(b->pairs[i]->o_ut);
  };
  auto slabs = [&](int mode, const SlabArgs* a, float beta, int k) -> cudaError_t {
    for (size_t gi = 0; gi < b->sgroups.size(); ++gi) {
      const auto& g = b->sgroups[gi];
      TRY(launch_slab_multi(mode, a + g.first, start + g.first + gi, g.count, g.blocks, g.smem, beta,
                            k, s));
    }
    return cudaSuccess;
  };
  auto zpasses = [&]() -> cudaError_t {
    for (size_t gi = 0; gi < b->zgroups.size(); ++gi) {
      const auto& g = b->zgroups[gi];
      TRY(launch_zslab_multi(g.r1, g.r2, pen + g.first, zstart + g.first + gi, g.count, g.blocks, s));
    }
    return cudaSuccess;
  };
  std::vector<float*> u_cur(n);
  for (int i = 0; i < n; ++i) {
    nadmm_context* p = b->pairs[i];
    unsigned* red = p->tab<unsigned>(p->o_red);
    TRY(cudaMemsetAsync(red, 0, 4 * sizeof(unsigned), s));
    if (p->restart) TRY(cudaMemsetAsync(p->tab<unsigned>(p->o_rwords), 0, 2 * sizeof(unsigned), s));
    u_cur[i] = (dst_of(i, 0) == u_out[i]) ? p->at<float>(p->o_ut) : u_out[i];
    TRY(cudaMemsetAsync(u_cur[i], 0, 3 * p->V * sizeof(float), s));
  }
  for (int i = 0; i < n; ++i) {
    nadmm_context* p = b->pairs[i];
    TRY(launch_warp(dims_of(p), I1[i], u_cur[i], p->at<float>(p->o_I1w), nullptr, s));
    TRY(launch_grad_residual(dims_of(p), p->at<float>(p->o_I1w), I0[i], p->at<float>(p->o_J),
                             p->at<float>(p->o_c), s));
  }
  for (int o = 0; o < O; ++o) {
    TRY(slabs(SLAB_FIRST, args, 0.0f, 0));
    for (int k = 1; k < K; ++k) {
      TRY(zpasses());
      TRY(slabs(k >= 2 ? SLAB_SPEC_PREV : SLAB_SPEC, args, beta_for(p0, k), k));
    }
    TRY(zpasses());
    TRY(slabs(SLAB_FINAL, fin, 0.0f, K));
    for (int i = 0; i < n; ++i) {
      nadmm_context* p = b->pairs[i];
      const Dims d = dims_of(p);
      unsigned* red = p->tab<unsigned>(p->o_red);
      float* vbuf = p->at<float>(p->o_wp);
      TRY(launch_bound_reduce(d, vbuf, red, s));
      float* u_new = dst_of(i, o);
      TRY(launch_compose(d, vbuf, u_cur[i], u_new, red, p->cfg.bound_kappa, p->cfg.bound_delta,
                         red + 2, nullptr, s));
      u_cur[i] = u_new;
    }
    if (o + 1 < O) {
      for (int i = 0; i < n; ++i) {
        nadmm_context* p = b->pairs[i];
        TRY(launch_warp(dims_of(p), I1[i], u_cur[i], p->at<float>(p->o_I1w),
                        p->tab<unsigned>(p->o_red), s));
        TRY(launch_grad_residual(dims_of(p), p->at<float>(p->o_I1w), I0[i], p->at<float>(p->o_J),
                                 p->at<float>(p->o_c), s));
      }
    }
  }
  return cudaSuccess;
}

// Streams and events of the lanes (created outside any stream capture).
cudaError_t ensure_lanes(nadmm_context* b) {
  if ((int)b->lane_cap.size() == b->lanes) return cudaSuccess;
  for (cudaStream_t q : b->lane_cap) cudaStreamDestroy(q);
  for (cudaEvent_t ev : b->lane_ev) cudaEventDestroy(ev);
  b->lane_cap.clear();
  b->lane_ev.clear();
  for (int l = 0; l < b->lanes; ++l) {
    cudaStream_t q;
    TRY(cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking));
    b->lane_cap.push_back(q);
  }
  for (int l = 0; l <= b->lanes; ++l) {
    cudaEvent_t ev;
    TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    b->lane_ev.push_back(ev);
  }
  return cudaSuccess;
}

// All pairs of a batched handle: lane l's pairs in order on its own stream,
// the lanes forked from and joined back into `s`.
cudaError_t enqueue_batched(nadmm_context* b, const float* const* I0, const float* const* I1,
                            float* const* u_out, cudaStream_t s) {
  const int n = (int)b->pairs.size();
  TRY(cudaEventRecord(b->lane_ev[0], s));
  for (int l = 0; l < b->lanes; ++l) {
    cudaStream_t q = b->lane_cap[l];
    TRY(cudaStreamWaitEvent(q, b->lane_ev[0], 0));
    for (int i = 0; i < n; ++i)
      if (b->lane_of[i] == l) TRY(enqueue_register(b->pairs[i], I0[i], I1[i], u_out[i], q));
    TRY(cudaEventRecord(b->lane_ev[1 + l], q));
    TRY(cudaStreamWaitEvent(s, b->lane_ev[1 + l], 0));
  }
  return cudaSuccess;
}

cudaError_t enqueue_backward(nadmm_context* h, const float* I0, const float* I1, const float* gu,
                             float* gI0, float* gI1, float* glam, float* gtheta, cudaStream_t s);

// Reverse sweeps of all pairs of a batched handle, lanes as in enqueue_batched.
cudaError_t enqueue_batched_backward(nadmm_context* b, const float* const* I0,
                                     const float* const* I1, const float* const* gu,
                                     float* const* gI0, float* const* gI1, float* const* glam,
                                     float* const* gtheta, cudaStream_t s) {
  const int n = (int)b->pairs.size();
  TRY(cudaEventRecord(b->lane_ev[0], s));
  for (int l = 0; l < b->lanes; ++l) {
    cudaStream_t q = b->lane_cap[l];
    TRY(cudaStreamWaitEvent(q, b->lane_ev[0], 0));
    for (int i = 0; i < n; ++i)
      if (b->lane_of[i] == l)
        TRY(enqueue_backward(b->pairs[i], I0[i], I1[i], gu[i], gI0[i], gI1[i],
                             glam ? glam[i] : nullptr, gtheta ? gtheta[i] : nullptr, q));
    TRY(cudaEventRecord(b->lane_ev[1 + l], q));
    TRY(cudaStreamWaitEvent(s, b->lane_ev[1 + l], 0));
  }
  return cudaSuccess;
}

// The levels of a pyramid handle, coarsest first: block-average the images
// down, register each level from the upsampled result of the coarser one.
cudaError_t enqueue_pyramid(nadmm_context* p, const float* I0, const float* I1, float* u_out,
                            cudaStream_t s) {
  const int L = (int)p->pairs.size();
  auto lvl = [&](int l, int part) -> float* {  // part: 0 I0, 1 I1, 2 u, 3 u_up
    const nadmm_context* c = p->pairs[l];
    const size_t V = c->V;
    const size_t off[4] = {0, align_up(V * 4), 2 * align_up(V * 4),
                           2 * align_up(V * 4) + align_up(3 * V * 4)};
    return reinterpret_cast<float*>(p->ws + p->lvl_off[l] + off[part]);
  };
  for (int l = 1; l < L; ++l) {
    const Dims dc = dims_of(p->pairs[l]);
    TRY(launch_downsample2(dc, l == 1 ? I0 : lvl(l - 1, 0), lvl(l, 0), s));
    TRY(launch_downsample2(dc, l == 1 ? I1 : lvl(l - 1, 1), lvl(l, 1), s));
  }
  for (int l = L - 1; l >= 0; --l) {
    const float* f = l == 0 ? I0 : lvl(l, 0);
    const float* m = l == 0 ? I1 : lvl(l, 1);
    float* dst = l == 0 ? u_out : lvl(l, 2);
    TRY(enqueue_register(p->pairs[l], f, m, dst, s, l == L - 1 ? nullptr : lvl(l, 3)));
    if (l > 0) TRY(launch_upsample_u(dims_of(p->pairs[l]), dims_of(p->pairs[l - 1]), dst, lvl(l - 1, 3), s));
  }
  return cudaSuccess;
}

nadmm_status run_register(nadmm_context* h, const float* I0, const float* I1, float* u_out,
                          cudaStream_t stream) {
  if (h->cfg.flags & NADMM_FLAG_NO_GRAPH) {
    cudaError_t e = enqueue_register(h, I0, I1, u_out, stream);
    return e == cudaSuccess ? NADMM_OK : cuda_fail(e, "nadmm_register");
  }
  return replay(h, 0, {I0, I1, u_out}, stream, "capture of nadmm_register",
                [&](cudaStream_t cs) { return enqueue_register(h, I0, I1, u_out, cs); });
}


// Reverse sweep of nadmm_register (s = 2): for the gradient gu of the final
// displacement, grad_fixed, grad_moving (overwritten) and, if not null,
// grad_lambda, grad_theta (device floats).  Outer steps are taken backwards;
// each recomputes its linearisation and its ADMM iterates from the saved u
// at its start, then runs the adjoints of compose, bound, the K ADMM steps
// and the linearisation.
// w = S y (the w-step's spectral solve, Eq. 6 last line) on the handle's
// path: forward x/y DFTs, z-pass with the filter, inverse x/y DFTs (three
// kernels) on the slab path; plane pass, y/z/y passes, final plane pass on
// the four-kernel path.
cudaError_t enqueue_solve(nadmm_context* h, const float* y, float* w, cudaStream_t s) {
  if (h->use_slab) {
    SlabArgs f = slab_args(h);
    f.w_in = y;
    TRY(launch_slab(SLAB_FIELD, f, s));
    TRY(launch_zslab(pencil_args(h), s));
    SlabArgs fin = slab_args(h);
    fin.y = nullptr;
    fin.w_out = w;
    fin.b_out = nullptr;
    return launch_slab(SLAB_FINAL, fin, s);
  }
  PlaneArgs a = plane_args(h);
  a.y = nullptr;
  a.w_in = y;
  TRY(launch_plane(IN_FIELD, false, true, a, s));
  TRY(launch_pencil(pencil_args(h), s));
  PlaneArgs f = plane_args(h);
  f.y = nullptr;
  f.w_out = w;
  f.b_out = nullptr;
  return launch_plane(IN_SPEC, false, false, f, s);
}

cudaError_t enqueue_backward(nadmm_context* h, const float* I0, const float* I1, const float* gu,
                             float* gI0, float* gI1, float* glam, float* gtheta, cudaStream_t s) {
  const Dims d = dims_of(h);
  const size_t V = h->V, F3 = 3 * V * sizeof(float);
  const int O = h->cfg.outer_iters, K = h->cfg.inner_iters;
  const float kappa = h->cfg.bound_kappa, delta = h->cfg.bound_delta;
  float* I1w = h->at<float>(h->o_I1w);
  float* J = h->at<float>(h->o_J);
  float* c = h->at<float>(h->o_c);
  float* tape = h->tab<float>(h->o_tape);
  float* hw = h->at<float>(h->o_hist);
  float* hu = hw + (size_t)K * 3 * V;
  float* adj = h->at<float>(h->o_adj);
  auto Wbar = [&](int k) { return adj + (size_t)(((k % 3) + 3) % 3) * 3 * V; };
  auto Bbar = [&](int k) { return adj + (size_t)(3 + ((k % 3) + 3) % 3) * 3 * V; };
  auto hist = [&](float* base, int k) { return base + (size_t)k * 3 * V; };
  float* g = h->at<float>(h->o_g);
  float* Sg = h->at<float>(h->o_Sg);
  float* gJ = h->at<float>(h->o_gJ);
  float* gc = h->at<float>(h->o_gc);
  float* ub0 = h->at<float>(h->o_ub0);
  float* ub1 = h->at<float>(h->o_ub1);
  unsigned* red = h->tab<unsigned>(h->o_red);
  double* acc = h->tab<double>(h->o_acc);

  TRY(cudaMemsetAsync(gI0, 0, V * sizeof(float), s));
  TRY(cudaMemsetAsync(gI1, 0, V * sizeof(float), s));
  TRY(cudaMemsetAsync(acc, 0, 3 * sizeof(double), s));
  TRY(cudaMemcpyAsync(ub0, gu, F3, cudaMemcpyDeviceToDevice, s));
  for (int o = O - 1; o >= 0; --o) {
    const float* u_o = tape + (size_t)o * 3 * V;
    // forward recomputation of outer step o
    TRY(launch_warp(d, I1, u_o, I1w, red, s));  // also clears red[0..1]
    TRY(launch_grad_residual(d, I1w, I0, J, c, s));
    TRY(enqueue_inner(h, plane_args(h), IN_NONE, false, 0, K, J, c, hist(hw, K - 1), nullptr, s,
                      hw, hu));
    const float* w = hist(hw, K - 1);
    TRY(launch_bound_reduce(d, w, red, s));
    // compose and bound
    TRY(cudaMemsetAsync(ub1, 0, F3, s));
    TRY(cudaMemsetAsync(acc, 0, sizeof(double), s));
    TRY(cudaMemsetAsync(red + 3, 0, sizeof(unsigned), s));
    TRY(cudaMemsetAsync(adj, 0, 6 * F3, s));
    TRY(launch_compose_vjp(d, u_o, w, red, kappa, delta, ub0, ub1, Wbar(K - 1), acc, s));
    TRY(launch_bound_vjp(d, w, red, kappa, delta, acc, red + 3, Wbar(K - 1), s));
    // ADMM iterations K-1 .. 0
    TRY(cudaMemsetAsync(gJ, 0, F3, s));
    TRY(cudaMemsetAsync(gc, 0, V * sizeof(float), s));
    const float* g_in = Wbar(K - 1);  // bbar^{K-1} = 0
    if (h->use_slab) {
      // slab path: the spectrum of g^{K-1}, then per reverse step one slab
      // pass (S g^k in, the adjoint point-wise step, the spectrum of g^{k-1}
      // out) and one z-pass
      SlabArgs f = slab_args(h);
      f.w_in = g_in;
      TRY(launch_slab(SLAB_FIELD, f, s));
      TRY(launch_zslab(pencil_args(h), s));
      for (int k = K - 1; k >= 0; --k) {
        SlabArgs a = slab_args(h);
        a.beta = beta_for(h, k);
        a.J = J;
        a.c = c;
        SlabAdj& r = a.adj;
        r.wk = hist(hw, k);
        r.uk = hist(hu, k);
        r.Bk = Bbar(k);
        if (k >= 1) {
          r.W1bar = Wbar(k - 1);
          r.B1bar = Bbar(k - 1);
        }
        if (k >= 2) {
          r.W2bar = Wbar(k - 2);
          r.B2bar = Bbar(k - 2);
        }
        r.g_in = g_in;
        r.g_out = g;
        r.gJ = gJ;
        r.gc = gc;
        r.acc = acc;
        r.inv_gamma = h->cfg.theta / h->cfg.lambda;
        TRY(launch_slab(k >= 1 ? SLAB_ADJ : SLAB_ADJ_LAST, a, s));
        if (k >= 1) TRY(launch_zslab(pencil_args(h), s));
        g_in = g;
      }
      TRY(launch_linearise_vjp(d, I1, u_o, gJ, gc, gI0, gI1, ub1, ub0, s));
      continue;
    }
    for (int k = K - 1; k >= 0; --k) {
      TRY(enqueue_solve(h, g_in, Sg, s));
      AdjArgs a;
      std::memset(&a, 0, sizeof(a));
      a.d = d;
      a.wk = hist(hw, k);
      a.uk = hist(hu, k);
      if (k >= 1) {
        a.W1bar = Wbar(k - 1);
        a.B1bar = Bbar(k - 1);
      }
      if (k >= 2) {
        a.W2bar = Wbar(k - 2);
        a.B2bar = Bbar(k - 2);
      }
      a.J = J;
      a.c = c;
      a.Sg = Sg;
      a.g_in = g_in;
      a.Bk = Bbar(k);
      a.g_out = g;
      a.gJ = gJ;
      a.gc = gc;
      a.acc = acc;
      a.beta = beta_for(h, k);
      a.theta = h->cfg.theta;
      a.inv_gamma = h->cfg.theta / h->cfg.lambda;
      TRY(launch_adj_step(a, s));
      g_in = g;
    }
    TRY(launch_linearise_vjp(d, I1, u_o, gJ, gc, gI0, gI1, ub1, ub0, s));
  }
  return launch_param_grads(acc, h->cfg.lambda, h->cfg.theta, glam, gtheta, s);
}

}  // namespace

// ====================================================================== ABI
extern "C" {

void nadmm_config_init(nadmm_config* c, int32_t nx, int32_t ny, int32_t nz) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->nx = nx;
  c->ny = ny;
  c->nz = nz;
  c->order_n = 2;
  c->lambda = 10.0f;
  c->theta = 0.1f;
  c->outer_iters = 10;
  c->inner_iters = 10;
  c->data_term = 2;
  c->eps = 1e-6f;
  c->bound_kappa = 0.5f;
  c->bound_delta = 1.0f;
  c->flags = 0;
  c->admm_tol = 0.0f;
  c->warp_tol = 0.0f;
  c->restart_eta = -1.0f;
}

const char* nadmm_last_error(void) { return g_err.c_str(); }

const char* nadmm_status_string(nadmm_status s) {
  switch (s) {
    case NADMM_OK: return "NADMM_OK";
    case NADMM_ERR_INVALID_ARG: return "NADMM_ERR_INVALID_ARG";
    case NADMM_ERR_UNSUPPORTED_SIZE: return "NADMM_ERR_UNSUPPORTED_SIZE";
    case NADMM_ERR_ALIGNMENT: return "NADMM_ERR_ALIGNMENT";
    case NADMM_ERR_NO_WORKSPACE: return "NADMM_ERR_NO_WORKSPACE";
    case NADMM_ERR_CUDA: return "NADMM_ERR_CUDA";
    case NADMM_ERR_NONFINITE: return "NADMM_ERR_NONFINITE";
    case NADMM_ERR_TIMEOUT: return "NADMM_ERR_TIMEOUT";
    case NADMM_ERR_NO_SAVED_FORWARD: return "NADMM_ERR_NO_SAVED_FORWARD";
  }
  return "unknown nadmm_status";
}

nadmm_status nadmm_create(const nadmm_config* cfg, nadmm_handle* out) {
  if (!out) return fail(NADMM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  nadmm_context* h = nullptr;
  nadmm_status st = create_single(cfg, &h);
  if (st != NADMM_OK) return st;
  h->total = align_up(h->state_total) + h->table_total;
  *out = h;
  return NADMM_OK;
}

// A batched handle from one configuration per pair (cfgs[i].nx/ny/nz are
// pair i's grid); shared by nadmm_create_batched and
// nadmm_create_batched_configs.
nadmm_status create_batched_from(const nadmm_config* cfgs, int32_t npairs, nadmm_handle* out) {
  nadmm_context* b = new nadmm_context();
  b->cfg = cfgs[0];
  b->batched = true;
  for (int i = 0; i < npairs; ++i) {
    const nadmm_config& c = cfgs[i];
    if (c.outer_iters != cfgs[0].outer_iters || c.inner_iters != cfgs[0].inner_iters ||
        c.flags != cfgs[0].flags) {
      destroy_context(b);
      return fail(NADMM_ERR_INVALID_ARG,
                  "pair " + std::to_string(i) +
                      ": every pair of a batch needs the same outer_iters, inner_iters and flags");
    }
    nadmm_context* p = nullptr;
    nadmm_status st = create_single(&c, &p);
    if (st != NADMM_OK) {
      g_err = "pair " + std::to_string(i) + ": " + g_err;
      destroy_context(b);
      return st;
    }
    b->pairs.push_back(p);
  }
  // concurrent lanes by default (flat execution on request, lane count 0):
  // measured at 128x128x96 and on 64 uneven pairs, two or three lanes of
  // four-kernel registrations beat flat slab passes (457 vs 489 ms for the
  // 64 pairs; 6.5 vs 7.4 ms per registration for three pairs)
  relayout(b, std::min(npairs, kDefaultLanes));
  *out = b;
  return NADMM_OK;
}

nadmm_status nadmm_create_batched(const nadmm_config* base, int32_t npairs, const int32_t* dims,
                                  nadmm_handle* out) {
  if (!out) return fail(NADMM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!base || !dims) return fail(NADMM_ERR_INVALID_ARG, "NULL argument");
  if (npairs < 1) return fail(NADMM_ERR_INVALID_ARG, "npairs must be >= 1");
  std::vector<nadmm_config> cfgs(npairs, *base);
  for (int i = 0; i < npairs; ++i) {
    cfgs[i].nx = dims[3 * i];
    cfgs[i].ny = dims[3 * i + 1];
    cfgs[i].nz = dims[3 * i + 2];
  }
  return create_batched_from(cfgs.data(), npairs, out);
}

nadmm_status nadmm_create_batched_configs(const nadmm_config* cfgs, int32_t npairs,
                                          nadmm_handle* out) {
  if (!out) return fail(NADMM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!cfgs) return fail(NADMM_ERR_INVALID_ARG, "NULL argument");
  if (npairs < 1) return fail(NADMM_ERR_INVALID_ARG, "npairs must be >= 1");
  return create_batched_from(cfgs, npairs, out);
}

nadmm_status nadmm_create_pyramid(const nadmm_config* finest, int32_t levels, const int32_t* outer,
                                  const int32_t* inner, nadmm_handle* out) {
  if (!out) return fail(NADMM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!finest || !outer || !inner) return fail(NADMM_ERR_INVALID_ARG, "NULL argument");
  if (levels < 1 || levels > 5) return fail(NADMM_ERR_INVALID_ARG, "levels must be in 1..5");
  if (finest->flags & NADMM_FLAG_SAVE_FOR_BACKWARD)
    return fail(NADMM_ERR_INVALID_ARG, "pyramid handles have no reverse mode");
  const int f = 1 << (levels - 1);
  if (finest->nx % f || finest->ny % f || finest->nz % f)
    return fail(NADMM_ERR_UNSUPPORTED_SIZE, "every dimension must be divisible by 2^(levels-1)");
  nadmm_context* p = new nadmm_context();
  p->cfg = *finest;
  p->pyramid = true;
  for (int l = 0; l < levels; ++l) {
    nadmm_config c = *finest;
    c.nx >>= l;
    c.ny >>= l;
    c.nz >>= l;
    c.outer_iters = outer[levels - 1 - l];  // arrays run coarsest first
    c.inner_iters = inner[levels - 1 - l];
    nadmm_context* q = nullptr;
    nadmm_status st = create_single(&c, &q);
    if (st != NADMM_OK) {
      g_err = "level " + std::to_string(l) + ": " + g_err;
      destroy_context(p);
      return st;
    }
    p->pairs.push_back(q);
  }
  size_t state = 0;
  for (nadmm_context* q : p->pairs) state = std::max(state, q->state_total);
  size_t o = align_up(state);
  p->tab_off.assign(levels, 0);
  p->lvl_off.assign(levels, 0);
  for (int l = 0; l < levels; ++l) {
    p->tab_off[l] = o;
    o = align_up(o + p->pairs[l]->table_total);
  }
  for (int l = 0; l < levels; ++l) {  // I0_l, I1_l, u_l, u_up_l (level 0 uses u_up only)
    const size_t V = p->pairs[l]->V;
    p->lvl_off[l] = o;
    o += 2 * align_up(V * 4) + 2 * align_up(3 * V * 4);
  }
  p->total = o;
  *out = p;
  return NADMM_OK;
}

nadmm_status nadmm_register_pyramid(nadmm_handle h, const float* fixed, const float* moving,
                                    float* u_out, void* stream) {
  const TraceRange trace("nadmm_register_pyramid");
  nadmm_status st = need_ws(h, kPyramid);
  if (st != NADMM_OK) return st;
  if ((st = check_dev_ptrs({fixed, moving, u_out})) != NADMM_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if (h->cfg.flags & NADMM_FLAG_NO_GRAPH) {
    cudaError_t e = enqueue_pyramid(h, fixed, moving, u_out, s);
    return e == cudaSuccess ? NADMM_OK : cuda_fail(e, "nadmm_register_pyramid");
  }
  return replay(h, 0, {fixed, moving, u_out}, s, "capture of nadmm_register_pyramid",
                [&](cudaStream_t cs) { return enqueue_pyramid(h, fixed, moving, u_out, cs); });
}

nadmm_status nadmm_batch_set_pair_plan(nadmm_handle h, int32_t pair, uint32_t plan_flags) {
  if (!h || !h->batched) return fail(NADMM_ERR_INVALID_ARG, "not a batched handle");
  if (h->wt) return fail(NADMM_ERR_INVALID_ARG, "set plans before nadmm_set_workspace");
  if (pair < 0 || pair >= (int32_t)h->pairs.size()) return fail(NADMM_ERR_INVALID_ARG, "pair out of range");
  const uint32_t tuned = NADMM_FLAG_LANE_MASK | NADMM_FLAG_FUSED_PENCIL | NADMM_FLAG_FOUR_PASS |
                         NADMM_FLAG_SLAB_PATH | NADMM_FLAG_OUTER_MASK;
  if (plan_flags & ~tuned)
    return fail(NADMM_ERR_INVALID_ARG,
                "only NADMM_FLAG_LANE*, NADMM_FLAG_FUSED_PENCIL, NADMM_FLAG_FOUR_PASS, "
                "NADMM_FLAG_SLAB_PATH and NADMM_FLAG_OUTER_* bits");
  nadmm_config c = h->pairs[pair]->cfg;
  c.flags = (c.flags & ~tuned) | plan_flags;
  nadmm_context* q = nullptr;
  nadmm_status st = create_single(&c, &q);
  if (st != NADMM_OK) return st;
  destroy_context(h->pairs[pair]);
  h->pairs[pair] = q;
  if (h->flat)
    relayout(h, flat_possible(h) ? 0 : std::min<int>((int)h->pairs.size(), kDefaultLanes));
  else
    relayout(h, h->lanes);
  return NADMM_OK;
}

nadmm_status nadmm_batch_set_lanes(nadmm_handle h, int32_t lanes) {
  if (!h || !h->batched) return fail(NADMM_ERR_INVALID_ARG, "not a batched handle");
  if (lanes < 0) return fail(NADMM_ERR_INVALID_ARG, "lanes must be >= 0 (0: flat)");
  if (h->wt) return fail(NADMM_ERR_INVALID_ARG, "set the lane count before nadmm_set_workspace");
  if (lanes == 0 && !flat_possible(h))
    return fail(NADMM_ERR_INVALID_ARG,
                "flat execution needs every pair on the slab path and no reverse-mode tape");
  relayout(h, lanes == 0 ? 0 : std::min<int>(lanes, (int)h->pairs.size()));
  return NADMM_OK;
}

nadmm_status nadmm_batch_get_lanes(nadmm_handle h, int32_t* lanes) {
  if (!h || !h->batched || !lanes) return fail(NADMM_ERR_INVALID_ARG, "not a batched handle");
  *lanes = h->flat ? 0 : h->lanes;
  return NADMM_OK;
}

void nadmm_destroy(nadmm_handle h) { destroy_context(h); }

nadmm_status nadmm_workspace_size(nadmm_handle h, size_t* bytes) {
  if (!h || !bytes) return fail(NADMM_ERR_INVALID_ARG, "NULL argument");
  *bytes = h->total;
  return NADMM_OK;
}

nadmm_status nadmm_set_workspace(nadmm_handle h, void* dev_ptr, size_t bytes) {
  if (!h || !dev_ptr) return fail(NADMM_ERR_INVALID_ARG, "NULL argument");
  if (((uintptr_t)dev_ptr % kAlign) != 0)
    return fail(NADMM_ERR_ALIGNMENT, "workspace must be 256-byte aligned");
  if (bytes < h->total) return fail(NADMM_ERR_NO_WORKSPACE, "workspace smaller than nadmm_workspace_size");
  invalidate_graph(h);
  h->ws = h->wt = nullptr;
  char* base = static_cast<char*>(dev_ptr);
  cudaError_t e = configure_kernels_once();
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
  if (h->pyramid) {
    for (size_t l = 0; l < h->pairs.size(); ++l) {
      nadmm_status st = attach(h->pairs[l], base, base + h->tab_off[l]);
      if (st != NADMM_OK) {
        for (nadmm_context* q : h->pairs) q->ws = q->wt = nullptr;
        return st;
      }
    }
    h->ws = base;
    h->wt = base;
  } else if (!h->batched) {
    nadmm_status st = attach(h, base, base + align_up(h->state_total));
    if (st != NADMM_OK) return st;
  } else {
    for (size_t i = 0; i < h->pairs.size(); ++i) {
      nadmm_context* p = h->pairs[i];
      nadmm_status st = attach(p, base + h->lane_off[h->lane_of[i]], base + h->tab_off[i]);
      if (st != NADMM_OK) {
        for (nadmm_context* q : h->pairs) q->ws = q->wt = nullptr;
        return st;
      }
    }
    h->ws = base;
    h->wt = base;
    if (h->flat) {
      for (nadmm_context* q : h->pairs) q->use_slab = true;
    } else if (h->lanes >= 2 && !(h->cfg.flags & NADMM_FLAG_SAVE_FOR_BACKWARD)) {
      // pairs running concurrently take the four-kernel path, whose passes
      // overlap across lanes (a slab pass needs every SM's registers), unless
      // the slab path is forced (flags, or adaptive restart).  With the
      // reverse-mode tape each pair keeps its own path: the slab path's
      // reverse sweep is the faster one (16 uneven pairs forward + backward:
      // 502 ms against 519 ms on the four-kernel path)
      for (nadmm_context* q : h->pairs)
        if (!(q->cfg.flags & (NADMM_FLAG_SLAB_PATH | NADMM_FLAG_SLAB_PAIRS)) && !q->restart)
          q->use_slab = false;
    }
    e = h->flat ? upload_flat(h) : ensure_lanes(h);
    if (e != cudaSuccess) {
      for (nadmm_context* q : h->pairs) q->ws = q->wt = nullptr;
      h->ws = h->wt = nullptr;
      return cuda_fail(e, h->flat ? "flat launch tables" : "lane streams");
    }
  }
  return NADMM_OK;
}

nadmm_status nadmm_set_params(nadmm_handle h, float lambda, float theta) {
  if (!h) return fail(NADMM_ERR_INVALID_ARG, "handle is NULL");
  nadmm_config c = h->cfg;
  c.lambda = lambda;
  c.theta = theta;
  nadmm_status st = validate(&c);
  if (st != NADMM_OK) return st;
  h->cfg = c;
  invalidate_graph(h);
  return NADMM_OK;
}

nadmm_status nadmm_register(nadmm_handle h, const float* fixed, const float* moving, float* u_out,
                            void* stream) {
  const TraceRange trace("nadmm_register");
  nadmm_status st = need_ws(h);
  if (st != NADMM_OK) return st;
  if ((st = check_dev_ptrs({fixed, moving, u_out})) != NADMM_OK) return st;
  st = run_register(h, fixed, moving, u_out, (cudaStream_t)stream);
  if (st == NADMM_OK && h->has_tape) h->saved_forward = true;
  return st;
}

nadmm_status nadmm_register_host(nadmm_handle h, const float* fixed_host, const float* moving_host,
                                 float* u_out_host, void* stream) {
  const TraceRange trace("nadmm_register_host");
  nadmm_status st = need_ws(h);
  if (st != NADMM_OK) return st;
  if (!fixed_host || !moving_host || !u_out_host) return fail(NADMM_ERR_INVALID_ARG, "NULL host buffer");
  cudaStream_t s = (cudaStream_t)stream;
  float* f = h->at<float>(h->o_io_f);
  float* m = h->at<float>(h->o_io_m);
  float* u = h->at<float>(h->o_io_u);
  const size_t V = h->V;
  cudaError_t e = cudaMemcpyAsync(f, fixed_host, V * sizeof(float), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m, moving_host, V * sizeof(float), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
  if ((st = run_register(h, f, m, u, s)) != NADMM_OK) return st;
  if (h->has_tape) h->saved_forward = true;
  e = cudaMemcpyAsync(u_out_host, u, 3 * V * sizeof(float), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? NADMM_OK : cuda_fail(e, "device-to-host copy");
}

nadmm_status nadmm_register_profiled(nadmm_handle h, const float* fixed, const float* moving,
                                     float* u_out, void* stream, float* kernel_ms,
                                     int32_t* launches) {
  const TraceRange trace("nadmm_register_profiled");
  nadmm_status st = need_ws(h);
  if (st != NADMM_OK) return st;
  if ((st = check_dev_ptrs({fixed, moving, u_out})) != NADMM_OK) return st;
  if (!kernel_ms || !launches) return fail(NADMM_ERR_INVALID_ARG, "NULL output array");
  cudaStream_t s = (cudaStream_t)stream;
  Profiler prof;
  g_prof = &prof;
  cudaError_t e = enqueue_register(h, fixed, moving, u_out, s);
  g_prof = nullptr;
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  for (int i = 0; i < NADMM_KC_COUNT; ++i) {
    kernel_ms[i] = 0.0f;
    launches[i] = 0;
  }
  if (e == cudaSuccess) {
    for (auto& m : prof.marks) {
      float ms = 0.0f;
      e = cudaEventElapsedTime(&ms, m.second.first, m.second.second);
      if (e != cudaSuccess) break;
      kernel_ms[m.first] += ms;
      launches[m.first] += 1;
    }
  }
  prof.release();
  return e == cudaSuccess ? NADMM_OK : cuda_fail(e, "nadmm_register_profiled");
}

nadmm_status nadmm_get_status(nadmm_handle h, void* stream) {
  if (!h) return fail(NADMM_ERR_INVALID_ARG, "handle is NULL");
  if (!h->wt) return fail(NADMM_ERR_NO_WORKSPACE, "no workspace attached (nadmm_set_workspace)");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  if (!h->batched && !h->pyramid) return read_status(h);
  nadmm_status worst = NADMM_OK;
  std::string msg;
  for (size_t i = 0; i < h->pairs.size(); ++i) {
    nadmm_status st = read_status(h->pairs[i]);
    if (st != NADMM_OK && worst == NADMM_OK) {
      worst = st;
      msg = "pair " + std::to_string(i) + ": " + g_err;
    }
  }
  if (worst != NADMM_OK) g_err = msg;
  return worst;
}

nadmm_status nadmm_register_batched(nadmm_handle h, const float* const* fixed,
                                    const float* const* moving, float* const* u_out, void* stream) {
  const TraceRange trace("nadmm_register_batched");
  nadmm_status st = need_ws(h, kBatched);
  if (st != NADMM_OK) return st;
  if (!fixed || !moving || !u_out) return fail(NADMM_ERR_INVALID_ARG, "NULL pointer array");
  const int n = (int)h->pairs.size();
  std::vector<const void*> key;
  key.reserve(3 * n);
  for (int i = 0; i < n; ++i) {
    if ((st = check_dev_ptrs({fixed[i], moving[i], u_out[i]})) != NADMM_OK) {
      g_err = "pair " + std::to_string(i) + ": " + g_err;
      return st;
    }
    key.push_back(fixed[i]);
    key.push_back(moving[i]);
    key.push_back(u_out[i]);
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (h->flat && (h->cfg.flags & NADMM_FLAG_NO_GRAPH)) {
    cudaError_t e = enqueue_batched_flat(h, fixed, moving, u_out, s);
    if (e != cudaSuccess) return cuda_fail(e, "nadmm_register_batched");
  } else if (h->flat) {
    st = replay(h, 0, key, s, "capture of nadmm_register_batched",
                [&](cudaStream_t cs) { return enqueue_batched_flat(h, fixed, moving, u_out, cs); });
  } else if (h->cfg.flags & NADMM_FLAG_NO_GRAPH) {
    for (int i = 0; i < n; ++i) {
      cudaError_t e = enqueue_register(h->pairs[i], fixed[i], moving[i], u_out[i], s);
      if (e != cudaSuccess) return cuda_fail(e, "nadmm_register_batched");
    }
  } else {
    st = replay(h, 0, key, s, "capture of nadmm_register_batched",
                [&](cudaStream_t cs) { return enqueue_batched(h, fixed, moving, u_out, cs); });
  }
  if (st == NADMM_OK)
    for (nadmm_context* p : h->pairs)
      if (p->has_tape) p->saved_forward = true;
  return st;
}

nadmm_status nadmm_backward_batched(nadmm_handle h, const float* const* fixed,
                                    const float* const* moving, const float* const* grad_u,
                                    float* const* grad_fixed, float* const* grad_moving,
                                    float* const* grad_lambda, float* const* grad_theta,
                                    void* stream) {
  const TraceRange trace("nadmm_backward_batched");
  nadmm_status st = need_ws(h, kBatched);
  if (st != NADMM_OK) return st;
  if (!(h->cfg.flags & NADMM_FLAG_SAVE_FOR_BACKWARD))
    return fail(NADMM_ERR_NO_SAVED_FORWARD, "handle created without NADMM_FLAG_SAVE_FOR_BACKWARD");
  if (h->cfg.data_term != 2)
    return fail(NADMM_ERR_INVALID_ARG, "the reverse mode supports the s = 2 data term only");
  if (!(h->cfg.lambda > 0.0f)) return fail(NADMM_ERR_INVALID_ARG, "the reverse mode needs lambda > 0");
  if (!fixed || !moving || !grad_u || !grad_fixed || !grad_moving)
    return fail(NADMM_ERR_INVALID_ARG, "NULL pointer array");
  const int n = (int)h->pairs.size();
  std::vector<const void*> key;
  for (int i = 0; i < n; ++i) {
    if (!h->pairs[i]->saved_forward)
      return fail(NADMM_ERR_NO_SAVED_FORWARD, "no nadmm_register_batched call since the workspace was attached");
    if ((st = check_dev_ptrs({fixed[i], moving[i], grad_u[i], grad_fixed[i], grad_moving[i]})) != NADMM_OK) {
      g_err = "pair " + std::to_string(i) + ": " + g_err;
      return st;
    }
    const void* gl = grad_lambda ? grad_lambda[i] : nullptr;
    const void* gt = grad_theta ? grad_theta[i] : nullptr;
    if ((gl && !aligned16(gl)) || (gt && !aligned16(gt)))
      return fail(NADMM_ERR_ALIGNMENT, "pair " + std::to_string(i) + ": grad_lambda/theta not aligned");
    for (const void* p : {(const void*)fixed[i], (const void*)moving[i], (const void*)grad_u[i],
                          (const void*)grad_fixed[i], (const void*)grad_moving[i], gl, gt})
      key.push_back(p);
  }
  cudaStream_t s = (cudaStream_t)stream;
  auto fn = [&](cudaStream_t cs) {
    return enqueue_batched_backward(h, fixed, moving, grad_u, grad_fixed, grad_moving, grad_lambda,
                                    grad_theta, cs);
  };
  if (h->cfg.flags & NADMM_FLAG_NO_GRAPH) {
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < n && e == cudaSuccess; ++i)
      e = enqueue_backward(h->pairs[i], fixed[i], moving[i], grad_u[i], grad_fixed[i],
                           grad_moving[i], grad_lambda ? grad_lambda[i] : nullptr,
                           grad_theta ? grad_theta[i] : nullptr, s);
    return e == cudaSuccess ? NADMM_OK : cuda_fail(e, "nadmm_backward_batched");
  }
  return replay(h, 1, key, s, "capture of nadmm_backward_batched", fn);
}

nadmm_status nadmm_spectral_solve(nadmm_handle h, const float* y, float* w, void* stream) {
  nadmm_status st = need_ws(h);
  if (st != NADMM_OK) return st;
  if ((st = check_dev_ptrs({y, w})) != NADMM_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if (h->use_slab) {
    SlabArgs f = slab_args(h);
    f.w_in = y;
    cudaError_t e = launch_slab(SLAB_FIELD, f, s);
    if (e == cudaSuccess) e = launch_zslab(pencil_args(h), s);
    if (e == cudaSuccess) {
      SlabArgs fin = slab_args(h);
      fin.y = nullptr;
      fin.w_out = w;
      fin.b_out = nullptr;
      e = launch_slab(SLAB_FINAL, fin, s);
    }
    return e == cudaSuccess ? NADMM_OK : cuda_fail(e, "nadmm_spectral_solve");
  }
  PlaneArgs a = plane_args(h);
  a.y = nullptr;
  a.w_in = y;
  cudaError_t e = launch_plane(IN_FIELD, false, true, a, s);
  if (e == cudaSuccess) e = launch_pencil(pencil_args(h), s);
  if (e == cudaSuccess) {
    PlaneArgs f = plane_args(h);
    f.y = nullptr;
    f.w_out = w;
    f.b_out = nullptr;
    e = launch_plane(IN_SPEC, false, false, f, s);
  }
  return e == cudaSuccess ? NADMM_OK : cuda_fail(e, "nadmm_spectral_solve");
}

nadmm_status nadmm_admm_run(nadmm_handle h, const float* J, const float* c, const float* w_km1,
                            const float* w_km2, const float* b_km1, const float* b_km2, int32_t k,
                            int32_t steps, float* w_out, float* b_out, void* stream) {
  nadmm_status st = need_ws(h);
  if (st != NADMM_OK) return st;
  if (k < 0 || steps < 1) return fail(NADMM_ERR_INVALID_ARG, "need k >= 0 and steps >= 1");
  if ((st = check_dev_ptrs({J, c, w_out, b_out})) != NADMM_OK) return st;
  if (k >= 1 && (st = check_dev_ptrs({w_km1, b_km1})) != NADMM_OK) return st;
  if (k >= 2 && (st = check_dev_ptrs({w_km2, b_km2})) != NADMM_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  PlaneArgs first = plane_args(h);
  int in_mode = IN_NONE;
  bool prev = false;
  if (k >= 1) {
    in_mode = IN_STATE;
    first.w_in = w_km1;
    first.b_in = b_km1;
    if (k >= 2) {
      prev = true;
      first.wprev_in = w_km2;
      first.bprev_in = b_km2;
    }
  }
  cudaError_t e = enqueue_inner(h, first, in_mode, prev, k, steps, J, c, w_out, b_out, s);
  return e == cudaSuccess ? NADMM_OK : cuda_fail(e, "nadmm_admm_run");
}

nadmm_status nadmm_linearise(nadmm_handle h, const float* fixed, const float* moving, const float* u,
                             float* J, float* c, float* I1w_out, void* stream) {
  nadmm_status st = need_ws(h);
  if (st != NADMM_OK) return st;
  if ((st = check_dev_ptrs({fixed, moving, u, J, c})) != NADMM_OK) return st;
  if (I1w_out && !aligned16(I1w_out)) return fail(NADMM_ERR_ALIGNMENT, "I1w_out not 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  float* I1w = I1w_out ? I1w_out : h->at<float>(h->o_I1w);
  cudaError_t e = launch_warp(dims_of(h), moving, u, I1w, nullptr, s);
  if (e == cudaSuccess) e = launch_grad_residual(dims_of(h), I1w, fixed, J, c, s);
  return e == cudaSuccess ? NADMM_OK : cuda_fail(e, "nadmm_linearise");
}

nadmm_status nadmm_bound_compose(nadmm_handle h, const float* w, const float* u_in, float* u_out,
                                 float* scale_out, void* stream) {
  nadmm_status st = need_ws(h);
  if (st != NADMM_OK) return st;
  if ((st = check_dev_ptrs({w, u_in, u_out})) != NADMM_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned* red = h->tab<unsigned>(h->o_red);
  cudaError_t e = cudaMemsetAsync(red, 0, 2 * sizeof(unsigned), s);
  if (e == cudaSuccess) e = launch_bound_reduce(dims_of(h), w, red, s);
  if (e == cudaSuccess)
    e = launch_compose(dims_of(h), w, u_in, u_out, red, h->cfg.bound_kappa, h->cfg.bound_delta,
                       red + 2, scale_out, s);
  return e == cudaSuccess ? NADMM_OK : cuda_fail(e, "nadmm_bound_compose");
}

nadmm_status nadmm_jacobian_det(nadmm_handle h, const float* u, float* det, uint32_t* nonpositive,
                                void* stream) {
  if (!h) return fail(NADMM_ERR_INVALID_ARG, "handle is NULL");
  if (h->batched || h->pyramid)
    return fail(NADMM_ERR_INVALID_ARG, "this call needs a single-pair handle (nadmm_create)");
  if (nadmm_status st = check_dev_ptrs({u}); st != NADMM_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (nonpositive) e = cudaMemsetAsync(nonpositive, 0, sizeof(uint32_t), s);
  if (e == cudaSuccess) e = launch_jacobian(dims_of(h), u, det, nonpositive, s);
  return e == cudaSuccess ? NADMM_OK : cuda_fail(e, "nadmm_jacobian_det");
}

nadmm_status nadmm_backward(nadmm_handle h, const float* fixed, const float* moving,
                            const float* grad_u, float* grad_fixed, float* grad_moving,
                            float* grad_lambda, float* grad_theta, void* stream) {
  const TraceRange trace("nadmm_backward");
  nadmm_status st = need_ws(h);
  if (st != NADMM_OK) return st;
  if (!(h->cfg.flags & NADMM_FLAG_SAVE_FOR_BACKWARD))
    return fail(NADMM_ERR_NO_SAVED_FORWARD, "handle created without NADMM_FLAG_SAVE_FOR_BACKWARD");
  if (!h->saved_forward)
    return fail(NADMM_ERR_NO_SAVED_FORWARD, "no nadmm_register call since the workspace was attached");
  if (h->cfg.data_term != 2)
    return fail(NADMM_ERR_INVALID_ARG, "the reverse mode supports the s = 2 data term only");
  if (!(h->cfg.lambda > 0.0f)) return fail(NADMM_ERR_INVALID_ARG, "the reverse mode needs lambda > 0");
  if ((st = check_dev_ptrs({fixed, moving, grad_u, grad_fixed, grad_moving})) != NADMM_OK) return st;
  if (grad_lambda && !aligned16(grad_lambda)) return fail(NADMM_ERR_ALIGNMENT, "grad_lambda not aligned");
  if (grad_theta && !aligned16(grad_theta)) return fail(NADMM_ERR_ALIGNMENT, "grad_theta not aligned");
  cudaStream_t s = (cudaStream_t)stream;
  auto fn = [&](cudaStream_t cs) {
    return enqueue_backward(h, fixed, moving, grad_u, grad_fixed, grad_moving, grad_lambda,
                            grad_theta, cs);
  };
  if (h->cfg.flags & NADMM_FLAG_NO_GRAPH) {
    cudaError_t e = fn(s);
    return e == cudaSuccess ? NADMM_OK : cuda_fail(e, "nadmm_backward");
  }
  return replay(h, 1, {fixed, moving, grad_u, grad_fixed, grad_moving, grad_lambda, grad_theta}, s,
                "capture of nadmm_backward", fn);
}

nadmm_status nadmm_ssd_after_warp(nadmm_handle h, const float* fixed, const float* moving,
                                  const float* u, float* loss, void* stream) {
  nadmm_status st = need_ws(h);
  if (st != NADMM_OK) return st;
  if ((st = check_dev_ptrs({fixed, moving, u, loss})) != NADMM_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  double* acc = h->tab<double>(h->o_acc) + 3;
  cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double), s);
  if (e == cudaSuccess) e = launch_ssd(dims_of(h), fixed, moving, u, acc, loss, s);
  return e == cudaSuccess ? NADMM_OK : cuda_fail(e, "nadmm_ssd_after_warp");
}

nadmm_status nadmm_ssd_after_warp_backward(nadmm_handle h, const float* fixed, const float* moving,
                                           const float* u, const float* grad_loss,
                                           float* grad_fixed, float* grad_moving, float* grad_u,
                                           void* stream) {
  nadmm_status st = need_ws(h);
  if (st != NADMM_OK) return st;
  if ((st = check_dev_ptrs({fixed, moving, u, grad_loss, grad_moving})) != NADMM_OK) return st;
  if (grad_fixed && !aligned16(grad_fixed)) return fail(NADMM_ERR_ALIGNMENT, "grad_fixed not aligned");
  if (grad_u && !aligned16(grad_u)) return fail(NADMM_ERR_ALIGNMENT, "grad_u not aligned");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(grad_moving, 0, h->V * sizeof(float), s);
  if (e == cudaSuccess)
    e = launch_ssd_vjp(dims_of(h), fixed, moving, u, grad_loss, grad_fixed, grad_moving, grad_u, s);
  return e == cudaSuccess ? NADMM_OK : cuda_fail(e, "nadmm_ssd_after_warp_backward");
}

nadmm_status nadmm_selftest_wait_timeout(nadmm_handle h, int32_t attempts, void* stream) {
  nadmm_status st = need_ws(h);
  if (st != NADMM_OK) return st;
  if (attempts < 1 || attempts > (1 << 20))
    return fail(NADMM_ERR_INVALID_ARG, "attempts must be in 1 .. 2^20");
  cudaError_t e = launch_wait_selftest(h->tab<unsigned>(h->o_red) + 2, attempts,
                                       (cudaStream_t)stream);
  return e == cudaSuccess ? NADMM_OK : cuda_fail(e, "nadmm_selftest_wait_timeout");
}

nadmm_status nadmm_autotune_workspace_size(const nadmm_config* cfg, size_t* bytes) {
  if (!bytes) return fail(NADMM_ERR_INVALID_ARG, "bytes is NULL");
  nadmm_config c = *cfg;
  c.flags &= ~(NADMM_FLAG_SAVE_FOR_BACKWARD | NADMM_FLAG_LANE_MASK | NADMM_FLAG_FOUR_PASS |
               NADMM_FLAG_FUSED_PENCIL | NADMM_FLAG_PIPELINED_PLANE);
  c.restart_eta = -1.0f;
  c.admm_tol = c.warp_tol = 0.0f;
  size_t most = 0;
  for (uint32_t combo = 0; combo < 8; ++combo) {
    nadmm_config t = c;
    for (int ax = 0; ax < 3; ++ax)
      t.flags |= (((combo >> ax) & 1u) ? 2u : 1u) << NADMM_FLAG_LANE_SHIFT(ax);
    nadmm_context* h = nullptr;
    nadmm_status st = create_single(&t, &h);
    if (st != NADMM_OK) return st;
    most = std::max(most, align_up(h->state_total) + h->table_total);
    destroy_context(h);
  }
  *bytes = most;
  return NADMM_OK;
}

nadmm_status nadmm_autotune(const nadmm_config* cfg, void* workspace, size_t bytes, void* stream,
                            uint32_t* best_flags, float* best_ms) {
  const TraceRange trace("nadmm_autotune");
  if (!cfg || !workspace || !best_flags) return fail(NADMM_ERR_INVALID_ARG, "NULL argument");
  if (((uintptr_t)workspace % kAlign) != 0)
    return fail(NADMM_ERR_ALIGNMENT, "workspace must be 256-byte aligned");
  size_t need = 0;
  nadmm_status st = nadmm_autotune_workspace_size(cfg, &need);
  if (st != NADMM_OK) return st;
  if (bytes < need) return fail(NADMM_ERR_NO_WORKSPACE, "workspace smaller than nadmm_autotune_workspace_size");
  cudaError_t e = configure_kernels_once();
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
  cudaStream_t s = (cudaStream_t)stream;
  char* base = static_cast<char*>(workspace);
  e = cudaMemsetAsync(base, 0, need, s);  // defined (zero) inputs for every trial
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return cuda_fail(e, "cudaEventCreate");
  }
  nadmm_config c = *cfg;
  c.flags &= ~(NADMM_FLAG_SAVE_FOR_BACKWARD | NADMM_FLAG_LANE_MASK | NADMM_FLAG_FUSED_PENCIL |
               NADMM_FLAG_FOUR_PASS | NADMM_FLAG_PIPELINED_PLANE | NADMM_FLAG_SLAB_PATH |
               NADMM_FLAG_OUTER_MASK);
  c.restart_eta = -1.0f;
  c.admm_tol = c.warp_tol = 0.0f;
  std::vector<std::vector<int>> seen;
  float best = -1.0f;
  uint32_t best_f = c.flags;
  // bits 0-2: 16 lanes on x / y / z; bit 3: fused y/z pass; bit 4: four-kernel path
  for (uint32_t combo = 0; combo < 32 && st == NADMM_OK; ++combo) {
    nadmm_config t = c;
    for (int ax = 0; ax < 3; ++ax)
      t.flags |= (((combo >> ax) & 1u) ? 2u : 1u) << NADMM_FLAG_LANE_SHIFT(ax);
    if (combo & 8u) t.flags |= NADMM_FLAG_FUSED_PENCIL;
    t.flags |= (combo & 16u) ? NADMM_FLAG_FOUR_PASS : NADMM_FLAG_SLAB_PATH;
    if ((combo & 8u) && !(combo & 16u)) continue;  // fusion is a four-kernel variant
    nadmm_context* h = nullptr;
    if ((st = create_single(&t, &h)) != NADMM_OK) break;
    // skip combinations whose kernels coincide with ones already timed (a
    // grid without the slab path runs its four-kernel plan either way)
    const int fused = (combo & 8u) ? (int)fused_pencil_supported(pencil_args(h)) : 0;
    const int slab = h->slab ? 1 : 0;
    std::vector<int> key = {slab ? h->pxh.radix[0] : h->px.radix[0],
                            slab ? 0 : h->px.radix[1], h->py.radix[0], h->py.radix[1],
                            h->pz.radix[0], h->pz.radix[1], fused, slab};
    bool dup = false;
    for (const auto& k : seen) dup = dup || k == key;
    if (!dup) {
      seen.push_back(key);
      st = attach(h, base, base + align_up(h->state_total));
      if (st == NADMM_OK) {
        PlaneArgs a = plane_args(h);
        a.J = h->at<float>(h->o_J);
        a.c = h->at<float>(h->o_c);
        a.beta = 0.5f;
        SlabArgs sa = slab_args(h);
        sa.beta = 0.5f;
        const PencilArgs pa = pencil_args(h);
        float ms = 0.0f, t_min = -1.0f;
        for (int rep = 0; rep < 13 && e == cudaSuccess; ++rep) {
          if (rep >= 3) e = cudaEventRecord(e0, s);
          if (slab) {
            if (e == cudaSuccess) e = launch_slab(SLAB_SPEC_PREV, sa, s);
            if (e == cudaSuccess) e = launch_zslab(pa, s);
          } else {
            if (e == cudaSuccess) e = launch_plane(IN_SPEC, true, true, a, s);
            if (e == cudaSuccess) e = launch_pencil(pa, s);
          }
          if (rep >= 3) {
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && (t_min < 0.0f || ms < t_min)) t_min = ms;
          }
        }
        if (e != cudaSuccess) st = cuda_fail(e, "autotune trial");
        else if (best < 0.0f || t_min < best) {
          best = t_min;
          best_f = t.flags;
        }
      }
    }
    destroy_context(h);
  }
  // the outer-step kernels of the chosen plan with 1, 2 and 4 z-slices per thread
  if (st == NADMM_OK) {
    nadmm_config t = c;
    t.flags = best_f;
    nadmm_context* h = nullptr;
    if ((st = create_single(&t, &h)) == NADMM_OK &&
        (st = attach(h, base, base + align_up(h->state_total))) == NADMM_OK) {
      float* u0 = h->at<float>(h->o_io_u);
      float* u1 = h->at<float>(h->o_ut);
      float* w = h->at<float>(h->o_wp);
      float* I = h->at<float>(h->o_io_f);
      unsigned* red = h->tab<unsigned>(h->o_red);
      float best_outer = -1.0f;
      uint32_t best_z = 0;
      const uint32_t zbits[3] = {0u, NADMM_FLAG_OUTER_Z2, NADMM_FLAG_OUTER_Z4};
      for (int zi = 0; zi < 3 && e == cudaSuccess; ++zi) {
        Dims d = dims_of(h);
        d.zv = 1 << zi;
        float ms = 0.0f, t_min = -1.0f;
        for (int rep = 0; rep < 13 && e == cudaSuccess; ++rep) {
          if (rep >= 3) e = cudaEventRecord(e0, s);
          if (e == cudaSuccess) e = launch_warp(d, I, u0, h->at<float>(h->o_I1w), red, s);
          if (e == cudaSuccess)
            e = launch_grad_residual(d, h->at<float>(h->o_I1w), I, h->at<float>(h->o_J),
                                     h->at<float>(h->o_c), s);
          if (e == cudaSuccess) e = launch_bound_reduce(d, w, red, s);
          if (e == cudaSuccess)
            e = launch_compose(d, w, u0, u1, red, t.bound_kappa, t.bound_delta, red + 2, nullptr, s);
          if (rep >= 3) {
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && (t_min < 0.0f || ms < t_min)) t_min = ms;
          }
        }
        if (e == cudaSuccess && (best_outer < 0.0f || t_min < best_outer)) {
          best_outer = t_min;
          best_z = zbits[zi];
        }
      }
      if (e != cudaSuccess) st = cuda_fail(e, "autotune trial (outer step)");
      else best_f |= best_z;
    }
    destroy_context(h);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != NADMM_OK) return st;
  const uint32_t tuned = NADMM_FLAG_LANE_MASK | NADMM_FLAG_FUSED_PENCIL | NADMM_FLAG_FOUR_PASS |
                         NADMM_FLAG_SLAB_PATH | NADMM_FLAG_OUTER_MASK;
  *best_flags = (cfg->flags & ~tuned) | (best_f & tuned);
  if (best_ms) *best_ms = best;
  return NADMM_OK;
}

nadmm_status nadmm_get_iterations(nadmm_handle h, void* stream, int32_t* outer_run,
                                  int32_t* admm_run) {
  if (!h || !outer_run || !admm_run) return fail(NADMM_ERR_INVALID_ARG, "NULL argument");
  if (h->batched || h->pyramid)
    return fail(NADMM_ERR_INVALID_ARG, "this call needs a single-pair handle (nadmm_create)");
  if (!h->wt) return fail(NADMM_ERR_NO_WORKSPACE, "no workspace attached (nadmm_set_workspace)");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  if (!thresholds(h)) {
    *outer_run = h->cfg.outer_iters;
    *admm_run = h->cfg.outer_iters * h->cfg.inner_iters;
    return NADMM_OK;
  }
  unsigned w[kConvWords];
  e = cudaMemcpy(w, h->tab<unsigned>(h->o_conv), sizeof(w), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "counter read");
  *outer_run = (int32_t)w[kConvOuterRun];
  *admm_run = (int32_t)w[kConvAdmmRun];
  return NADMM_OK;
}

}  // extern "C"

nadmm_status nadmm_get_restarts(nadmm_handle h, void* stream, int32_t* restarts) {
  nadmm_status st = need_ws(h);
  if (st != NADMM_OK) return st;
  if (!restarts) return fail(NADMM_ERR_INVALID_ARG, "NULL argument");
  if (!h->restart) return fail(NADMM_ERR_INVALID_ARG, "the handle has no adaptive restart");
  unsigned words[2] = {0, 0};
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e == cudaSuccess)
    e = cudaMemcpy(words, h->tab<unsigned>(h->o_rwords), sizeof(words), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "nadmm_get_restarts");
  *restarts = (int32_t)words[1];
  return NADMM_OK;
}

namespace nadmm {
// Lets other translation units of the library report through nadmm_last_error.
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace nadmm
