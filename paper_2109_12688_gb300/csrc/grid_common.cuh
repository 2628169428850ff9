// Device helpers shared by the outer-step kernels and their adjoints, so
// that both sample, bound and difference with identical arithmetic.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include "nadmm_internal.h"

namespace nadmm {

// (1 - t) a + t b, exact at t = 0 and t = 1 (a sample on a grid point, or
// clamped to the last one, returns the grid value itself)
__device__ __forceinline__ float lerp(float a, float b, float t) {
  return fmaf(t, b, fmaf(-t, a, a));
}

__device__ __forceinline__ float trilerp(const float* __restrict__ f, Dims d, float px, float py,
                                         float pz) {
  px = fminf(fmaxf(px, 0.0f), (float)(d.nx - 1));
  py = fminf(fmaxf(py, 0.0f), (float)(d.ny - 1));
  pz = fminf(fmaxf(pz, 0.0f), (float)(d.nz - 1));
  int ix = min((int)floorf(px), d.nx - 2);
  int iy = min((int)floorf(py), d.ny - 2);
  int iz = min((int)floorf(pz), d.nz - 2);
  float fx = px - (float)ix, fy = py - (float)iy, fz = pz - (float)iz;
  const size_t sx = 1, sy = (size_t)d.nx, sz = (size_t)d.nx * d.ny;
  const float* p = f + (size_t)iz * sz + (size_t)iy * sy + ix;
  float c000 = __ldg(p), c001 = __ldg(p + sx);
  float c010 = __ldg(p + sy), c011 = __ldg(p + sy + sx);
  float c100 = __ldg(p + sz), c101 = __ldg(p + sz + sx);
  float c110 = __ldg(p + sz + sy), c111 = __ldg(p + sz + sy + sx);
  float c00 = lerp(c000, c001, fx);
  float c01 = lerp(c010, c011, fx);
  float c10 = lerp(c100, c101, fx);
  float c11 = lerp(c110, c111, fx);
  float c0 = lerp(c00, c01, fy);
  float c1 = lerp(c10, c11, fy);
  return lerp(c0, c1, fz);
}

// Block (32, 8) covers 32 x-consecutive voxels of 8 rows; grid (nx/32, ny/8,
// z-slices).  Coordinates come from the block indices (no division).
constexpr int kBX = 32, kBY = 8;

// Neighbour offsets of voxel i = (x, y, z) for clamped central differences.
struct Nbr {
  size_t xp, xm, yp, ym, zp, zm;
};

__device__ __forceinline__ Nbr neighbours(Dims d, int x, int y, int z, size_t i) {
  const size_t sy = (size_t)d.nx, sz = (size_t)d.nx * d.ny;
  Nbr n;
  n.xp = i + (x + 1 < d.nx ? 1 : 0);
  n.xm = i - (x > 0 ? 1 : 0);
  n.yp = i + (y + 1 < d.ny ? sy : 0);
  n.ym = i - (y > 0 ? sy : 0);
  n.zp = i + (z + 1 < d.nz ? sz : 0);
  n.zm = i - (z > 0 ? sz : 0);
  return n;
}

// Row sum |d f/dx| + |d f/dy| + |d f/dz| of one component of the velocity
// Jacobian (the bound's ||D w||_inf is the max over components and voxels).
__device__ __forceinline__ float jacobian_row(const float* __restrict__ f, const Nbr& n) {
  return fabsf(0.5f * (__ldg(f + n.xp) - __ldg(f + n.xm))) +
         fabsf(0.5f * (__ldg(f + n.yp) - __ldg(f + n.ym))) +
         fabsf(0.5f * (__ldg(f + n.zp) - __ldg(f + n.zm)));
}

__device__ __forceinline__ float bound_factor(const unsigned* red, float kappa, float delta,
                                              unsigned* status) {
  float mabs = __uint_as_float(red[0]);
  float mjac = __uint_as_float(red[1]);
  if (!isfinite(mabs) || !isfinite(mjac)) {
    if (status) atomicOr(status, 1u);
    return 0.0f;
  }
  float s = 1.0f;
  if (isfinite(kappa) && mjac > 0.0f) s = fminf(s, kappa / mjac);
  if (isfinite(delta) && mabs > 0.0f) s = fminf(s, delta / mabs);
  return s;
}

}  // namespace nadmm
