// Fused y/z/y pass of the spectral w-step (Eq. 6, last line): forward y-DFTs,
// forward z-DFT, the multiply by 1/(1 + gamma K^n)/(nx ny nz), inverse
// z-DFT and inverse y-DFTs of one (component, kx) plane of the half
// spectrum, in one kernel.
//
// A plane [nz][ny] is held by a cluster of two CTAs, each with half of the
// z rows in shared memory (rows padded to ny + 4 and permuted inside blocks
// of 8, so that the column accesses of the z-transform hit distinct banks).
// The y-transforms are lane FFTs on the CTA's own rows.  For the z-transform
// the two CTAs swap the column halves of their rows through distributed
// shared memory, so each CTA holds full z-columns for half of the y
// positions; after it they swap back and run the inverse y-transforms.  The
// spectrum is read and written once per ADMM iteration instead of three
// times, and the whole plane stays on chip between the passes.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "fft_device.cuh"
#include "lane_fft.cuh"
#include "nadmm_internal.h"
#include "plan.h"
#include "tma.cuh"

namespace cg = cooperative_groups;

namespace nadmm {

constexpr int kFusedThreads = 256;
constexpr int kFusedPadding = 4;  // row pitch ny + 4: consecutive rows 8 banks apart

// Shared-memory row of local z index zl (0 <= zl < nz/2): rows are permuted
// inside aligned blocks of 8 (an involution).
__device__ __forceinline__ int zrow(int zl) { return zl ^ ((zl >> 3) & 7); }

#if defined(__CUDA_ARCH__)
// Forward y-transform of one row in place: natural order in, swizzled
// digit-reversed order out (the lane FFT of lane_fft.cuh with a natural
// input).  R2 lanes of one warp, lane l, group mask `mask`.
template <int R1, int R2>
__device__ __forceinline__ void row_fft_fwd(float2* row, const float2* __restrict__ tw, int l,
                                            unsigned mask) {
  float2 v[R1];
#pragma unroll
  for (int j = 0; j < R1; ++j) v[j] = row[l + R2 * j];
  lane_stage1<R1, R2, false>(v, tw, l);
  __syncwarp(mask);  // the group has read the row before it is overwritten
#pragma unroll
  for (int k = 0; k < R1; ++k) row[swz<R2>(l + R2 * k)] = v[k];
  __syncwarp(mask);
  lane_stage2<R1, R2, false>(row, l);
  __syncwarp(mask);
}

// Inverse y-transform of one row in place: swizzled digit-reversed in,
// natural order out.
template <int R1, int R2>
__device__ __forceinline__ void row_fft_inv(float2* row, const float2* __restrict__ tw, int l,
                                            unsigned mask) {
  lane_stage2<R1, R2, true>(row, l);
  __syncwarp(mask);
  float2 v[R1];
#pragma unroll
  for (int k = 0; k < R1; ++k) v[k] = row[swz<R2>(l + R2 * k)];
  lane_stage1<R1, R2, true>(v, tw, l);
  __syncwarp(mask);
#pragma unroll
  for (int j = 0; j < R1; ++j) row[l + R2 * j] = v[j];
}

// Swap with the peer CTA: my rows at the peer's columns go to the peer's
// slab, at my columns; the peer's rows at my columns arrive in mine.
template <int S, int HALF, int P>
__device__ __forceinline__ void swap_halves(cg::cluster_group& cluster, float2* slab,
                                            float2* peer, int my_c0, int peer_c0, int tid) {
  constexpr int N = S * HALF;
  constexpr int PER = (N + kFusedThreads - 1) / kFusedThreads;
  float2 st[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int e = tid + i * kFusedThreads;
    if (e < N) {
      const int r = e / HALF, c = e - (e / HALF) * HALF;
      st[i] = slab[r * P + peer_c0 + c];
    }
  }
  cluster.sync();  // both CTAs hold their outgoing blocks
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int e = tid + i * kFusedThreads;
    if (e < N) {
      const int r = e / HALF, c = e - (e / HALF) * HALF;
      peer[r * P + my_c0 + c] = st[i];
    }
  }
  cluster.sync();  // every remote write has landed
}
#endif

template <int R1Y, int R2Y, int R1Z>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kFusedThreads, 3)
    k_pencil_fused(const __grid_constant__ PencilArgs a) {
#if defined(__CUDA_ARCH__)
  constexpr int NY = R1Y * R2Y, NZ = R1Z * 8, S = NZ / 2, HALF = NY / 2;
  constexpr int P = NY + kFusedPadding;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  float2* slab = reinterpret_cast<float2*>(smem_raw + 128);
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();  // 0: z in [0, S), 1: z in [S, NZ)
  const int plane = (int)(blockIdx.x >> 1);     // comp * nkx + kx
  const int kx = plane - (int)fdiv((uint32_t)plane, a.nkx_div) * a.nkx;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float2* gplane = a.spec + (size_t)plane * NZ * NY;
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  pdl_wait();  // the spectrum comes from the previous kernel
  pdl_trigger();
  // threshold stop: both CTAs of the cluster read the same words
  if (a.conv != nullptr && (a.conv[kConvInner] | a.conv[kConvOuter])) return;

  // own half of the plane, one bulk copy per row
  const uint32_t row_bytes = (uint32_t)(NY * sizeof(float2));
  if (warp == 0) {
    if (lane == 0) mbar_expect_tx(bar, row_bytes * S);
    __syncwarp();
    for (int zl = lane; zl < S; zl += 32)
      bulk_load(slab + zrow(zl) * P, gplane + (size_t)(rank * S + zl) * NY, row_bytes, bar);
  }
  if (!__syncthreads_and(mbar_wait_bounded(bar, 0))) {
    // record it and carry on: the peer waits at the cluster barriers below
    if (tid == 0 && a.status != nullptr) atomicOr(a.status, kStatusTimeout);
    mbar_wait_bounded(bar, 0);
  }

  // forward y-transforms of the CTA's rows
  {
    constexpr int LPW = 32 / R2Y;
    const int g = lane / R2Y, l = lane - g * R2Y;
    const unsigned gmask = ((R2Y == 32) ? 0xffffffffu : ((1u << R2Y) - 1u)) << (g * R2Y);
    for (int r = warp * LPW + g; r < S; r += (kFusedThreads / 32) * LPW)
      row_fft_fwd<R1Y, R2Y>(slab + r * P, a.twy, l, gmask);
  }
  __syncthreads();
  float2* peer = cluster.map_shared_rank(slab, rank ^ 1);
  const int my_c0 = rank * HALF, peer_c0 = (rank ^ 1) * HALF;
  swap_halves<S, HALF, P>(cluster, slab, peer, my_c0, peer_c0, tid);

  // z-transforms of my HALF columns: element z at row zrow(z mod S), column
  // my_c0 + c for my rows, peer_c0 + c for the peer's
  {
    constexpr int CPW = 4;
    const int l = lane / CPW, col = lane - (lane / CPW) * CPW;  // consecutive lanes, consecutive y
    const float kxv = __ldg(a.Kx + kx);
    for (int c = warp * CPW + col; c < HALF; c += (kFusedThreads / 32) * CPW) {
      auto at = [&](int z) -> float2* {
        const int h = z >= S ? 1 : 0;
        const int zl = z - h * S;
        return slab + zrow(zl) * P + ((h == rank) ? my_c0 : peer_c0) + c;
      };
      float2 v[R1Z];
#pragma unroll
      for (int j = 0; j < R1Z; ++j) v[j] = *at(l + 8 * j);
      lane_stage1<R1Z, 8, false>(v, a.twz, l);
      __syncwarp();
#pragma unroll
      for (int k = 0; k < R1Z; ++k) *at(l + 8 * k) = v[k];
      __syncwarp();
      // last forward stage, 1/(1 + gamma K^n)/(nx ny nz), first inverse stage;
      // the column's y position is swz(my_c0 + c) (the swizzle is an involution)
      const float kxy = kxv + __ldg(a.Ky + swz<R2Y>(my_c0 + c));
      for (int b = l; b < R1Z; b += 8) {
        float2 w[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) w[j] = *at(8 * b + j);
        dft<8, false>(w);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float K = kxy + __ldg(a.Kz + 8 * b + k);
          float Kn = K;
          for (int i = 1; i < a.order_n; ++i) Kn *= K;
          w[k] = cscale(w[k], __fdividef(a.scale, 1.0f + a.gamma * Kn));
        }
        dft<8, true>(w);
#pragma unroll
        for (int j = 0; j < 8; ++j) *at(8 * b + j) = w[j];
      }
      __syncwarp();
#pragma unroll
      for (int k = 0; k < R1Z; ++k) v[k] = *at(l + 8 * k);
      lane_stage1<R1Z, 8, true>(v, a.twz, l);
#pragma unroll
      for (int j = 0; j < R1Z; ++j) *at(l + 8 * j) = v[j];
      __syncwarp();
    }
  }
  __syncthreads();
  swap_halves<S, HALF, P>(cluster, slab, peer, my_c0, peer_c0, tid);

  // inverse y-transforms, back to natural order
  {
    constexpr int LPW = 32 / R2Y;
    const int g = lane / R2Y, l = lane - g * R2Y;
    const unsigned gmask = ((R2Y == 32) ? 0xffffffffu : ((1u << R2Y) - 1u)) << (g * R2Y);
    for (int r = warp * LPW + g; r < S; r += (kFusedThreads / 32) * LPW)
      row_fft_inv<R1Y, R2Y>(slab + r * P, a.twy, l, gmask);
  }
  fence_proxy_async();  // the rows are read by bulk copies next
  __syncthreads();
  if (warp == 0) {
    for (int zl = lane; zl < S; zl += 32)
      bulk_store(gplane + (size_t)(rank * S + zl) * NY, slab + zrow(zl) * P, row_bytes);
    bulk_commit();
    bulk_wait_read();
  }
#endif
}

// ---------------------------------------------------------------- dispatch
#define NADMM_FUSED_CASES(X) \
  X(6, 16, 8) X(6, 16, 10) X(6, 16, 12) X(6, 16, 14) \
  X(8, 16, 8) X(8, 16, 10) X(8, 16, 12) X(8, 16, 14) \
  X(10, 16, 8) X(10, 16, 10) X(10, 16, 12) X(10, 16, 14)

size_t fused_pencil_smem(const PencilArgs& a) {
  return 128 + (size_t)(a.nz / 2) * (a.ny + kFusedPadding) * sizeof(float2);
}

bool fused_pencil_supported(const PencilArgs& a) {
  if (a.py.nst != 2 || a.pz.nst != 2 || a.py.m[1] != 1 || a.pz.m[1] != 1) return false;
  if (a.pz.radix[1] != 8 || a.nz % 16 != 0 || (a.ny / 2) % 16 != 0) return false;
  if (fused_pencil_smem(a) > 100 * 1024) return false;  // at least two clusters' CTAs per SM
  const int r1y = a.py.radix[0], r2y = a.py.radix[1], r1z = a.pz.radix[0];
#define X(A, B, C) \
  if (r1y == A && r2y == B && r1z == C) return true;
  NADMM_FUSED_CASES(X)
#undef X
  return false;
}

cudaError_t configure_fused_pencil() {
  cudaError_t e = cudaSuccess;
#define X(A, B, C)                                                                          \
  if (e == cudaSuccess)                                                                     \
    e = cudaFuncSetAttribute(k_pencil_fused<A, B, C>,                                       \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024 + 128);
  NADMM_FUSED_CASES(X)
#undef X
  return e;
}

cudaError_t launch_fused_pencil(const PencilArgs& a, cudaStream_t s) {
  const int r1y = a.py.radix[0], r2y = a.py.radix[1], r1z = a.pz.radix[0];
  const dim3 grid((unsigned)(2 * 3 * a.nkx)), block(kFusedThreads);
  const size_t smem = fused_pencil_smem(a);
#define X(A, B, C) \
  if (r1y == A && r2y == B && r1z == C) return launch_pdl(k_pencil_fused<A, B, C>, grid, block, smem, s, a);
  NADMM_FUSED_CASES(X)
#undef X
  return cudaErrorInvalidValue;
}

}  // namespace nadmm
