// Warp-level two-stage line FFTs ("lane FFTs") for plans n = R1 * R2 with
// R2 in {8, 16}: R2 lanes hold one line, lane l the positions l + R2 j.
// Used by the y/z passes (lane_passes.cu) and by the plane pass's x-DFTs.
#pragma once
#include "fft_device.cuh"

namespace nadmm {

// Position p of a line stored at p ^ ((p / R2) mod R2): rows of R2-blocks
// are rotated so that both access patterns (lane l writing l + R2 k, a lane
// reading a whole block) spread over the banks.
template <int R2>
__device__ __forceinline__ int swz(int p) {
  return p ^ ((p / R2) & (R2 - 1));
}

// Same swizzle for a runtime R2 (log2r2 = log2 R2); identity when log2r2 < 0.
NADMM_HD int swz_rt(int p, int log2r2) {
  return log2r2 < 0 ? p : p ^ ((p >> log2r2) & ((1 << log2r2) - 1));
}

template <int R1, int R2, bool INV>
__device__ __forceinline__ void lane_stage1(float2 (&v)[R1], const float2* __restrict__ tw, int l) {
  if (!INV) {
    dft<R1, false>(v);
#pragma unroll
    for (int k = 1; k < R1; ++k) v[k] = cmul(v[k], __ldg(tw + (k - 1) * R2 + l));
  } else {
#pragma unroll
    for (int k = 1; k < R1; ++k) v[k] = cmulc(v[k], __ldg(tw + (k - 1) * R2 + l));
    dft<R1, true>(v);
  }
}

// lane_stage1 with the lane's twiddles already in registers: twr[k - 1] =
// tw[(k - 1) R2 + l], k = 1 .. R1 - 1.
template <int R1, int R2, bool INV>
__device__ __forceinline__ void lane_stage1_reg(float2 (&v)[R1], const float2 (&twr)[R1 - 1]) {
  if (!INV) {
    dft<R1, false>(v);
#pragma unroll
    for (int k = 1; k < R1; ++k) v[k] = cmul(v[k], twr[k - 1]);
  } else {
#pragma unroll
    for (int k = 1; k < R1; ++k) v[k] = cmulc(v[k], twr[k - 1]);
    dft<R1, true>(v);
  }
}

template <int R1, int R2>
__device__ __forceinline__ void lane_twiddles(const float2* __restrict__ tw, int l,
                                              float2 (&twr)[R1 - 1]) {
#pragma unroll
  for (int k = 1; k < R1; ++k) twr[k - 1] = __ldg(tw + (k - 1) * R2 + l);
}

// Second stage on whole blocks b = l, l + R2, ... < R1 of a swizzled line.
template <int R1, int R2, bool INV>
__device__ __forceinline__ void lane_stage2(float2* line, int l) {
  for (int b = l; b < R1; b += R2) {
    float2 w[R2];
#pragma unroll
    for (int j = 0; j < R2; ++j) w[j] = line[swz<R2>(b * R2 + j)];
    dft<R2, INV>(w);
#pragma unroll
    for (int j = 0; j < R2; ++j) line[swz<R2>(b * R2 + j)] = w[j];
  }
}

// In-place transform of one swizzled line in shared memory by its R2 lanes
// (lane l of the group).  Forward: natural order in, digit-reversed out;
// inverse: the reverse.  The group's lanes must be converged in one warp.
template <int R1, int R2, bool INV>
__device__ __forceinline__ void lane_line_fft(float2* line, const float2* __restrict__ tw, int l,
                                              unsigned mask) {
  float2 v[R1];
  if (!INV) {
#pragma unroll
    for (int j = 0; j < R1; ++j) v[j] = line[swz<R2>(l + R2 * j)];
    lane_stage1<R1, R2, false>(v, tw, l);
#pragma unroll
    for (int k = 0; k < R1; ++k) line[swz<R2>(l + R2 * k)] = v[k];
    __syncwarp(mask);
    lane_stage2<R1, R2, false>(line, l);
    __syncwarp(mask);
  } else {
    lane_stage2<R1, R2, true>(line, l);
    __syncwarp(mask);
#pragma unroll
    for (int k = 0; k < R1; ++k) v[k] = line[swz<R2>(l + R2 * k)];
    lane_stage1<R1, R2, true>(v, tw, l);
#pragma unroll
    for (int j = 0; j < R1; ++j) line[swz<R2>(l + R2 * j)] = v[j];
    __syncwarp(mask);
  }
}

#define NADMM_LANE_CASES(X) \
  X(3, 8) X(4, 8) X(6, 8) X(8, 8) X(9, 8) X(10, 8) X(12, 8) X(14, 8) X(16, 8) \
  X(3, 16) X(4, 16) X(6, 16) X(8, 16) X(9, 16) X(10, 16) X(12, 16) X(14, 16) X(16, 16)

// Runtime dispatch over the supported (R1, R2); returns false if unsupported.
template <bool INV>
__device__ __forceinline__ bool lane_line_fft_rt(int r1, int r2, float2* line,
                                                 const float2* __restrict__ tw, int l,
                                                 unsigned mask) {
#define X(A, B)                                     \
  if (r1 == A && r2 == B) {                         \
    lane_line_fft<A, B, INV>(line, tw, l, mask);    \
    return true;                                    \
  }
  NADMM_LANE_CASES(X)
#undef X
  return false;
}

}  // namespace nadmm
