// y- and z-passes of the spectral w-step (Eq. 6, last line) for axes whose
// plan splits as n = R1 * R2 with R2 in {8, 16} ("lane FFTs").
//
// One line is held by R2 lanes of a warp; lane l keeps the R1 values at
// positions l + R2 j.  The first stage (R1-point DFTs and twiddles) runs on
// those registers straight after coalesced global loads; one exchange through
// a warp-private, XOR-swizzled shared buffer gives each lane whole blocks of
// R2 consecutive positions for the second stage.  Positions and the
// digit-reversed order are those of the generic plan [R1, R2], so these
// kernels are interchangeable with the shared-memory stage kernels.
//
//   y-pass: one line = one (component, kx, z) row of ny values (contiguous);
//   z-pass: one line = one (component, kx, y) column of nz values (stride
//           ny); its second stage is the last forward stage, the inverse
//           symbol multiply and the first inverse stage fused in registers.
// Every warp works alone: no block barriers and no waits on other warps.
#include <cuda_runtime.h>

#include "fft_device.cuh"
#include "lane_fft.cuh"
#include "nadmm_internal.h"
#include "plan.h"

namespace nadmm {

constexpr int kLaneThreads = 128;  // 4 independent warps

template <int R1, int R2, bool INV>
__global__ void __launch_bounds__(kLaneThreads) k_ylane(const __grid_constant__ PencilArgs a) {
  constexpr int N = R1 * R2, LPW = 32 / R2, P = N + 8;
  extern __shared__ float2 sm_all[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / R2, l = lane % R2;
  float2* sm = sm_all + (warp * LPW + g) * P;
  const int total = 3 * a.nkx * a.nz;
  const int row = (blockIdx.x * (kLaneThreads / 32) + warp) * LPW + g;
  const bool active = row < total;
  pdl_wait();  // the spectrum comes from the previous kernel
  if (a.conv != nullptr && (a.conv[kConvInner] | a.conv[kConvOuter])) return;  // threshold stop
  pdl_trigger();
  float2* line = a.spec + (size_t)(active ? row : 0) * N;
  float2 v[R1];
  if (!INV) {
#pragma unroll
    for (int j = 0; j < R1; ++j) v[j] = active ? __ldcg(line + l + R2 * j) : make_float2(0.f, 0.f);
    lane_stage1<R1, R2, false>(v, a.twy, l);
#pragma unroll
    for (int k = 0; k < R1; ++k) sm[swz<R2>(l + R2 * k)] = v[k];
    __syncwarp();
    for (int b = l; b < R1; b += R2) {
      float2 w[R2];
#pragma unroll
      for (int j = 0; j < R2; ++j) w[j] = sm[swz<R2>(b * R2 + j)];
      dft<R2, false>(w);
#pragma unroll
      for (int j = 0; j < R2; ++j) sm[swz<R2>(b * R2 + j)] = w[j];
    }
    __syncwarp();
    if (active) {
#pragma unroll
      for (int k = 0; k < R1; ++k) __stcg(line + l + R2 * k, sm[swz<R2>(l + R2 * k)]);
    }
  } else {
#pragma unroll
    for (int k = 0; k < R1; ++k) v[k] = active ? __ldcg(line + l + R2 * k) : make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < R1; ++k) sm[swz<R2>(l + R2 * k)] = v[k];
    __syncwarp();
    for (int b = l; b < R1; b += R2) {
      float2 w[R2];
#pragma unroll
      for (int j = 0; j < R2; ++j) w[j] = sm[swz<R2>(b * R2 + j)];
      dft<R2, true>(w);
#pragma unroll
      for (int j = 0; j < R2; ++j) sm[swz<R2>(b * R2 + j)] = w[j];
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < R1; ++k) v[k] = sm[swz<R2>(l + R2 * k)];
    lane_stage1<R1, R2, true>(v, a.twy, l);
    if (active) {
#pragma unroll
      for (int j = 0; j < R1; ++j) __stcg(line + l + R2 * j, v[j]);
    }
  }
}

// Resident blocks requested per SM: the small shapes fit 64 registers.
template <int R1, int R2>
constexpr int zlane_min_blocks() {
  return (R2 == 8 && R1 <= 12) ? 8 : 6;
}

template <int R1, int R2>
__global__ void __launch_bounds__(kLaneThreads, zlane_min_blocks<R1, R2>())
    k_zlane(const __grid_constant__ PencilArgs a) {
  constexpr int N = R1 * R2, CPW = 32 / R2;
  constexpr int P = N + (R2 == 8 ? 4 : 8);  // column pitch: a half-warp's columns on other banks
  extern __shared__ float2 sm_all[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int l = lane / CPW, col = lane % CPW;  // consecutive lanes on consecutive y
  float2* sm = sm_all + (warp * CPW + col) * P;
  const int groups = a.ny / CPW;                // column groups per (component, kx) plane
  const int tasks = 3 * a.nkx * groups;
  const int task = blockIdx.x * (kLaneThreads / 32) + warp;
  const bool active = task < tasks;
  const int plane = active ? task / groups : 0;
  const int y = (active ? task - plane * groups : 0) * CPW + col;
  const int kx = plane % a.nkx;
  pdl_wait();
  if (a.conv != nullptr && (a.conv[kConvInner] | a.conv[kConvOuter])) return;  // threshold stop
  pdl_trigger();
  float2* base = a.spec + (size_t)plane * a.ny * a.nz + y;
  const size_t zs = (size_t)a.ny;
  float2 v[R1];
#pragma unroll
  for (int j = 0; j < R1; ++j) v[j] = active ? __ldcg(base + (l + R2 * j) * zs) : make_float2(0.f, 0.f);
  lane_stage1<R1, R2, false>(v, a.twz, l);
#pragma unroll
  for (int k = 0; k < R1; ++k) sm[swz<R2>(l + R2 * k)] = v[k];
  __syncwarp();
  // last forward stage, 1/(1 + gamma K^n)/(nx ny nz) at (kx, y, z position),
  // first inverse stage
  const float kxy = __ldg(a.Kx + kx) + __ldg(a.Ky + y);
  for (int b = l; b < R1; b += R2) {
    float2 w[R2];
#pragma unroll
    for (int j = 0; j < R2; ++j) w[j] = sm[swz<R2>(b * R2 + j)];
    dft<R2, false>(w);
#pragma unroll
    for (int k = 0; k < R2; ++k) {
      const float K = kxy + __ldg(a.Kz + b * R2 + k);
      float Kn = K;
      for (int i = 1; i < a.order_n; ++i) Kn *= K;
      w[k] = cscale(w[k], __fdividef(a.scale, 1.0f + a.gamma * Kn));
    }
    dft<R2, true>(w);
#pragma unroll
    for (int j = 0; j < R2; ++j) sm[swz<R2>(b * R2 + j)] = w[j];
  }
  __syncwarp();
#pragma unroll
  for (int k = 0; k < R1; ++k) v[k] = sm[swz<R2>(l + R2 * k)];
  lane_stage1<R1, R2, true>(v, a.twz, l);
  if (active) {
#pragma unroll
    for (int j = 0; j < R1; ++j) __stcg(base + (l + R2 * j) * zs, v[j]);
  }
}

// ---------------------------------------------------------------- dispatch
namespace {

template <int R1, int R2>
cudaError_t launch_y(const PencilArgs& a, bool inv, cudaStream_t s) {
  constexpr int N = R1 * R2, LPW = 32 / R2;
  const int rows = 3 * a.nkx * a.nz;
  const int per_cta = (kLaneThreads / 32) * LPW;
  const dim3 grid((unsigned)((rows + per_cta - 1) / per_cta));
  const size_t smem = (size_t)per_cta * (N + 8) * sizeof(float2);
  return inv ? launch_pdl(k_ylane<R1, R2, true>, grid, dim3(kLaneThreads), smem, s, a)
             : launch_pdl(k_ylane<R1, R2, false>, grid, dim3(kLaneThreads), smem, s, a);
}

template <int R1, int R2>
cudaError_t launch_z(const PencilArgs& a, cudaStream_t s) {
  constexpr int N = R1 * R2, CPW = 32 / R2;
  const int tasks = 3 * a.nkx * (a.ny / CPW);
  const int per_cta = kLaneThreads / 32;
  const dim3 grid((unsigned)((tasks + per_cta - 1) / per_cta));
  const size_t smem = (size_t)per_cta * CPW * (N + (R2 == 8 ? 4 : 8)) * sizeof(float2);
  return launch_pdl(k_zlane<R1, R2>, grid, dim3(kLaneThreads), smem, s, a);
}

}  // namespace

static bool is_lane_plan(const AxisPlan& p) {
  return p.nst == 2 && p.m[1] == 1 && lane_pair_supported(p.radix[0], p.radix[1]);
}

bool lane_y_supported(const PencilArgs& a) { return is_lane_plan(a.py); }
bool lane_z_supported(const PencilArgs& a) {
  return is_lane_plan(a.pz) && a.ny % (32 / a.pz.radix[1]) == 0;
}

cudaError_t launch_lane_y(const PencilArgs& a, bool inv, cudaStream_t s) {
  const int r1 = a.py.radix[0], r2 = a.py.radix[1];
#define X(A, B) \
  if (r1 == A && r2 == B) return launch_y<A, B>(a, inv, s);
  NADMM_LANE_CASES(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t launch_lane_z(const PencilArgs& a, cudaStream_t s) {
  const int r1 = a.pz.radix[0], r2 = a.pz.radix[1];
#define X(A, B) \
  if (r1 == A && r2 == B) return launch_z<A, B>(a, s);
  NADMM_LANE_CASES(X)
#undef X
  return cudaErrorInvalidValue;
}

}  // namespace nadmm
