// Outer diffeomorphic step (Sec. 2, Eq. 1 with N = 1) and grid utilities:
//   bound the velocity, compose phi <- phi o (Id + v), re-warp the moving
//   image by trilinear interpolation and recompute its gradient and the
//   residual that linearise the data term of Eq. 2 for the next ADMM solve.
// Sampling clamps coordinates to [0, dim - 1]; gradients are central
// differences with clamped indices, (f[i+1] - f[i-1]) / 2.
#include <cuda_runtime.h>
#include <math.h>

#include "grid_common.cuh"
#include "nadmm_internal.h"

namespace nadmm {

// Sums (a, b) over the block, added to acc[0..1] (double) by one thread.
__device__ __forceinline__ void block_add2(float a, float b, double* acc) {
  for (int off = 16; off > 0; off >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, off);
    b += __shfl_xor_sync(0xffffffffu, b, off);
  }
  __shared__ float pa[kBY], pb[kBY];
  if (threadIdx.x == 0) {
    pa[threadIdx.y] = a;
    pb[threadIdx.y] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    double sa = 0.0, sb = 0.0;
    for (int k = 0; k < kBY; ++k) {
      sa += pa[k];
      sb += pb[k];
    }
    atomicAdd(acc, sa);
    atomicAdd(acc + 1, sb);
  }
}

// I1w(x) = I1(x + u(x)).  Also clears the bound reduction words of the next
// outer step (the compose that read them has completed).  With `measure`,
// the change against the previous I1w is summed, and the last block to
// finish decides the outer stop (sqrt(sum d^2) <= warp_tol sqrt(sum old^2)).
// ZV z-slices per thread (blockIdx.z covers slices ZV blockIdx.z ..): more
// independent gathers in flight per thread; the same result for every ZV.
template <int ZV>
__global__ void __launch_bounds__(kBX * kBY)
    k_warp(Dims d, const float* __restrict__ I1, const float* __restrict__ u,
           float* __restrict__ I1w, unsigned* red, unsigned* conv, double* conv_acc,
           float warp_tol, int measure) {
  const size_t V = (size_t)d.nx * d.ny * d.nz;
  pdl_wait();
  pdl_trigger();
  if (conv != nullptr && conv[kConvOuter]) return;
  const int x = blockIdx.x * kBX + threadIdx.x, y = blockIdx.y * kBY + threadIdx.y;
  if (red != nullptr && (blockIdx.x | blockIdx.y | blockIdx.z) == 0 && threadIdx.y == 0 &&
      threadIdx.x < 2)
    red[threadIdx.x] = 0u;
  float dd = 0.0f, oo = 0.0f;
  if (x < d.nx && y < d.ny) {
#pragma unroll
    for (int zz = 0; zz < ZV; ++zz) {
      const int z = blockIdx.z * ZV + zz;
      if (z < d.nz) {
        const size_t i = ((size_t)z * d.ny + y) * d.nx + x;
        const float v =
            trilerp(I1, d, (float)x + u[i], (float)y + u[V + i], (float)z + u[2 * V + i]);
        if (measure) {
          const float old = I1w[i];
          dd += (v - old) * (v - old);
          oo += old * old;
        }
        I1w[i] = v;
      }
    }
  }
  if (!measure) return;
  block_add2(dd, oo, conv_acc + 2);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    __threadfence();
    const unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
    if (atomicAdd(conv + kConvWarpDone, 1u) == nblk - 1) {  // last block: all sums are in
      __threadfence();
      const double d2 = atomicAdd(conv_acc + 2, 0.0), o2 = atomicAdd(conv_acc + 3, 0.0);
      conv[kConvOuter] = (sqrt(d2) <= (double)warp_tol * sqrt(o2)) ? 1u : 0u;
      conv_acc[2] = 0.0;
      conv_acc[3] = 0.0;
      conv[kConvWarpDone] = 0u;
    }
  }
}

// J = grad I1w (clamped central differences), c = I1w - I0
template <int ZV>
__global__ void __launch_bounds__(kBX * kBY) k_grad_residual(Dims d,
                                                             const float* __restrict__ I1w,
                                                             const float* __restrict__ I0,
                                                             float* __restrict__ J,
                                                             float* __restrict__ c,
                                                             const unsigned* conv) {
  pdl_wait();
  pdl_trigger();
  if (conv != nullptr && conv[kConvOuter]) return;
  const size_t V = (size_t)d.nx * d.ny * d.nz;
  const size_t sy = (size_t)d.nx, sz = (size_t)d.nx * d.ny;
  const int x = blockIdx.x * kBX + threadIdx.x, y = blockIdx.y * kBY + threadIdx.y;
  if (x >= d.nx || y >= d.ny) return;
#pragma unroll
  for (int zz = 0; zz < ZV; ++zz) {
    const int z = blockIdx.z * ZV + zz;
    if (z < d.nz) {
      const size_t i = ((size_t)z * d.ny + y) * d.nx + x;
      const size_t xp = i + (x + 1 < d.nx ? 1 : 0), xm = i - (x > 0 ? 1 : 0);
      const size_t yp = i + (y + 1 < d.ny ? sy : 0), ym = i - (y > 0 ? sy : 0);
      const size_t zp = i + (z + 1 < d.nz ? sz : 0), zm = i - (z > 0 ? sz : 0);
      J[i] = 0.5f * (__ldg(I1w + xp) - __ldg(I1w + xm));
      J[V + i] = 0.5f * (__ldg(I1w + yp) - __ldg(I1w + ym));
      J[2 * V + i] = 0.5f * (__ldg(I1w + zp) - __ldg(I1w + zm));
      c[i] = __ldg(I1w + i) - __ldg(I0 + i);
    }
  }
}

// Per-voxel |w|_inf and ||D w||_inf (max absolute row sum of the Jacobian);
// grid-wide max through atomicMax on the float bit patterns (non-negative
// floats order like their bits; NaN bits sort above +inf).  A thread takes
// four x-consecutive voxels of one row (float4 loads of the voxels and of
// their y- and z-neighbours, two scalars for the x-neighbours outside the
// quad); block (32, 8) covers 128 x 8 voxels of one z-slice.
__global__ void __launch_bounds__(kBX * kBY) k_bound_reduce(Dims d, const float* __restrict__ w,
                                                            unsigned* red, const unsigned* conv) {
  pdl_wait();
  pdl_trigger();
  if (conv != nullptr && conv[kConvOuter]) return;
  const size_t V = (size_t)d.nx * d.ny * d.nz;
  const size_t sy = (size_t)d.nx, sz = (size_t)d.nx * d.ny;
  const int x0 = (blockIdx.x * kBX + threadIdx.x) * 4, y = blockIdx.y * kBY + threadIdx.y;
  const int z = blockIdx.z;
  float mabs = 0.0f, mjac = 0.0f;
  if (x0 < d.nx && y < d.ny) {
    const size_t i = ((size_t)z * d.ny + y) * d.nx + x0;
    const size_t iym = y > 0 ? i - sy : i, iyp = y + 1 < d.ny ? i + sy : i;
    const size_t izm = z > 0 ? i - sz : i, izp = z + 1 < d.nz ? i + sz : i;
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
      const float* f = w + comp * V;
      const float4 q = __ldg(reinterpret_cast<const float4*>(f + i));
      const float xm = x0 > 0 ? __ldg(f + i - 1) : q.x;
      const float xp = x0 + 4 < d.nx ? __ldg(f + i + 4) : q.w;
      const float4 ym = __ldg(reinterpret_cast<const float4*>(f + iym));
      const float4 yp = __ldg(reinterpret_cast<const float4*>(f + iyp));
      const float4 zm = __ldg(reinterpret_cast<const float4*>(f + izm));
      const float4 zp = __ldg(reinterpret_cast<const float4*>(f + izp));
      const float c[4] = {q.x, q.y, q.z, q.w};
      const float lo[4] = {xm, q.x, q.y, q.z}, hi[4] = {q.y, q.z, q.w, xp};
      const float ylo[4] = {ym.x, ym.y, ym.z, ym.w}, yhi[4] = {yp.x, yp.y, yp.z, yp.w};
      const float zlo[4] = {zm.x, zm.y, zm.z, zm.w}, zhi[4] = {zp.x, zp.y, zp.z, zp.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float a = fabsf(c[e]);
        const float row = fabsf(0.5f * (hi[e] - lo[e])) + fabsf(0.5f * (yhi[e] - ylo[e])) +
                          fabsf(0.5f * (zhi[e] - zlo[e]));
        // fmaxf drops NaN; keep it visible through the bit-pattern max instead
        mabs = (a != a || a > mabs) ? a : mabs;
        mjac = (row != row || row > mjac) ? row : mjac;
      }
    }
  }
  unsigned ua = __float_as_uint(mabs), uj = __float_as_uint(mjac);
  for (int off = 16; off > 0; off >>= 1) {
    ua = max(ua, __shfl_xor_sync(0xffffffffu, ua, off));
    uj = max(uj, __shfl_xor_sync(0xffffffffu, uj, off));
  }
  __shared__ unsigned sa[kBY], sj[kBY];
  if (threadIdx.x == 0) {
    sa[threadIdx.y] = ua;
    sj[threadIdx.y] = uj;
  }
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    for (int k = 1; k < kBY; ++k) {
      ua = max(ua, sa[k]);
      uj = max(uj, sj[k]);
    }
    atomicMax(red, ua);
    atomicMax(red + 1, uj);
  }
}

// u_out(x) = v(x) + u_in(x + v(x)), v = s w
template <int ZV>
__global__ void __launch_bounds__(kBX * kBY) k_compose(Dims d, const float* __restrict__ w,
                                                       const float* __restrict__ u_in,
                                                       float* __restrict__ u_out,
                                                       const unsigned* red, float kappa,
                                                       float delta, unsigned* status,
                                                       float* scale_out, unsigned* conv) {
  pdl_wait();
  pdl_trigger();
  const size_t V = (size_t)d.nx * d.ny * d.nz;
  const int x = blockIdx.x * kBX + threadIdx.x, y = blockIdx.y * kBY + threadIdx.y;
  if (conv != nullptr && conv[kConvOuter]) {  // stopped: carry u over to u_out
    if (x >= d.nx || y >= d.ny || u_in == u_out) return;
    for (int zz = 0; zz < ZV; ++zz) {
      const int z = blockIdx.z * ZV + zz;
      if (z >= d.nz) break;
      const size_t i = ((size_t)z * d.ny + y) * d.nx + x;
      u_out[i] = u_in[i];
      u_out[V + i] = u_in[V + i];
      u_out[2 * V + i] = u_in[2 * V + i];
    }
    return;
  }
  if (conv != nullptr && (blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x | threadIdx.y) == 0)
    atomicAdd(conv + kConvOuterRun, 1u);  // one more outer step composed
  const bool first = (blockIdx.x | blockIdx.y | blockIdx.z) == 0 && threadIdx.x == 0 &&
                     threadIdx.y == 0;
  const float s = bound_factor(red, kappa, delta, first ? status : nullptr);
  if (scale_out != nullptr && first) *scale_out = s;
  if (x >= d.nx || y >= d.ny) return;
#pragma unroll
  for (int zz = 0; zz < ZV; ++zz) {
    const int z = blockIdx.z * ZV + zz;
    if (z < d.nz) {
      const size_t i = ((size_t)z * d.ny + y) * d.nx + x;
      const float vx = s * w[i], vy = s * w[V + i], vz = s * w[2 * V + i];
      const float px = (float)x + vx, py = (float)y + vy, pz = (float)z + vz;
      u_out[i] = vx + trilerp(u_in, d, px, py, pz);
      u_out[V + i] = vy + trilerp(u_in + V, d, px, py, pz);
      u_out[2 * V + i] = vz + trilerp(u_in + 2 * V, d, px, py, pz);
    }
  }
}

// det(I + D u) per voxel, count of det <= 0
__global__ void __launch_bounds__(kBX * kBY) k_jacobian(Dims d, const float* __restrict__ u,
                                                        float* __restrict__ det, unsigned* count) {
  pdl_wait();
  pdl_trigger();
  const size_t V = (size_t)d.nx * d.ny * d.nz;
  const size_t sy = (size_t)d.nx, sz = (size_t)d.nx * d.ny;
  const int x = blockIdx.x * kBX + threadIdx.x, y = blockIdx.y * kBY + threadIdx.y;
  const int z = blockIdx.z;
  unsigned local = 0;
  if (x < d.nx && y < d.ny) {
    const size_t i = ((size_t)z * d.ny + y) * d.nx + x;
    const size_t xp = i + (x + 1 < d.nx ? 1 : 0), xm = i - (x > 0 ? 1 : 0);
    const size_t yp = i + (y + 1 < d.ny ? sy : 0), ym = i - (y > 0 ? sy : 0);
    const size_t zp = i + (z + 1 < d.nz ? sz : 0), zm = i - (z > 0 ? sz : 0);
    float A[3][3];
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
      const float* f = u + comp * V;
      A[comp][0] = 0.5f * (__ldg(f + xp) - __ldg(f + xm));
      A[comp][1] = 0.5f * (__ldg(f + yp) - __ldg(f + ym));
      A[comp][2] = 0.5f * (__ldg(f + zp) - __ldg(f + zm));
      A[comp][comp] += 1.0f;
    }
    const float dt = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
                     A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                     A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    if (det != nullptr) det[i] = dt;
    if (!(dt > 0.0f)) local = 1;
  }
  if (count != nullptr) {
    for (int off = 16; off > 0; off >>= 1) local += __shfl_xor_sync(0xffffffffu, local, off);
    if (threadIdx.x == 0 && local) atomicAdd(count, local);
  }
}

// Pyramid (Sec. 4): coarse(x) = mean of the 2 x 2 x 2 fine block at 2x.
__global__ void __launch_bounds__(kBX * kBY) k_downsample2(Dims c, const float* __restrict__ fine,
                                                           float* __restrict__ coarse) {
  pdl_wait();
  pdl_trigger();
  const int x = blockIdx.x * kBX + threadIdx.x, y = blockIdx.y * kBY + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= c.nx || y >= c.ny) return;
  const size_t fx = 2 * (size_t)c.nx, fxy = fx * 2 * (size_t)c.ny;
  const float* p = fine + (2 * (size_t)z) * fxy + (2 * (size_t)y) * fx + 2 * (size_t)x;
  const float s = (__ldg(p) + __ldg(p + 1)) + (__ldg(p + fx) + __ldg(p + fx + 1)) +
                  ((__ldg(p + fxy) + __ldg(p + fxy + 1)) + (__ldg(p + fxy + fx) + __ldg(p + fxy + fx + 1)));
  coarse[((size_t)z * c.ny + y) * c.nx + x] = 0.125f * s;
}

// u_fine(x) = 2 u_coarse((x - 1/2) / 2), trilinear with clamped coordinates.
__global__ void __launch_bounds__(kBX * kBY) k_upsample_u(Dims c, Dims f, const float* __restrict__ uc,
                                                          float* __restrict__ uf) {
  pdl_wait();
  pdl_trigger();
  const int x = blockIdx.x * kBX + threadIdx.x, y = blockIdx.y * kBY + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= f.nx || y >= f.ny) return;
  const size_t Vc = (size_t)c.nx * c.ny * c.nz, Vf = (size_t)f.nx * f.ny * f.nz;
  const size_t i = ((size_t)z * f.ny + y) * f.nx + x;
  const float px = 0.5f * ((float)x - 0.5f), py = 0.5f * ((float)y - 0.5f), pz = 0.5f * ((float)z - 0.5f);
#pragma unroll
  for (int comp = 0; comp < 3; ++comp) uf[comp * Vf + i] = 2.0f * trilerp(uc + comp * Vc, c, px, py, pz);
}

static dim3 grid3(Dims d, int zslices) {
  return dim3((unsigned)((d.nx + kBX - 1) / kBX), (unsigned)((d.ny + kBY - 1) / kBY),
              (unsigned)zslices);
}
static const dim3 kBlock(kBX, kBY);

static unsigned zgroups(Dims d) { return (unsigned)((d.nz + d.zv - 1) / d.zv); }

// The kernel of a ZV-templated family for d.zv (1, 2 or 4; other values run 1).
#define NADMM_ZV_LAUNCH(kernel, d, ...)                                                         \
  ((d).zv == 4 ? launch_pdl(kernel<4>, grid3((d), zgroups(d)), kBlock, 0, __VA_ARGS__)        \
   : (d).zv == 2 ? launch_pdl(kernel<2>, grid3((d), zgroups(d)), kBlock, 0, __VA_ARGS__)      \
                 : launch_pdl(kernel<1>, grid3((d), (d).nz), kBlock, 0, __VA_ARGS__))

cudaError_t launch_warp(Dims d, const float* I1, const float* u, float* I1w, unsigned* red_reset,
                        cudaStream_t s) {
  if (d.zv != 2 && d.zv != 4) d.zv = 1;
  return NADMM_ZV_LAUNCH(k_warp, d, s, d, I1, u, I1w, red_reset, (unsigned*)nullptr,
                         (double*)nullptr, 0.0f, 0);
}

cudaError_t launch_warp_measured(Dims d, const float* I1, const float* u, float* I1w,
                                 unsigned* red_reset, unsigned* conv, double* conv_acc,
                                 float warp_tol, bool measure, cudaStream_t s) {
  if (d.zv != 2 && d.zv != 4) d.zv = 1;
  return NADMM_ZV_LAUNCH(k_warp, d, s, d, I1, u, I1w, red_reset, conv, conv_acc, warp_tol,
                         measure ? 1 : 0);
}

cudaError_t launch_grad_residual(Dims d, const float* I1w, const float* I0, float* J, float* c,
                                 cudaStream_t s) {
  if (d.zv != 2 && d.zv != 4) d.zv = 1;
  return NADMM_ZV_LAUNCH(k_grad_residual, d, s, d, I1w, I0, J, c, (const unsigned*)nullptr);
}

cudaError_t launch_grad_residual_conv(Dims d, const float* I1w, const float* I0, float* J, float* c,
                                      const unsigned* conv, cudaStream_t s) {
  if (d.zv != 2 && d.zv != 4) d.zv = 1;
  return NADMM_ZV_LAUNCH(k_grad_residual, d, s, d, I1w, I0, J, c, conv);
}

cudaError_t launch_bound_reduce(Dims d, const float* w, unsigned* red, cudaStream_t s,
                                const unsigned* conv) {
  const dim3 grid((unsigned)((d.nx + 4 * kBX - 1) / (4 * kBX)), (unsigned)((d.ny + kBY - 1) / kBY),
                  (unsigned)d.nz);
  return launch_pdl(k_bound_reduce, grid, kBlock, 0, s, d, w, red, conv);
}

cudaError_t launch_compose(Dims d, const float* w, const float* u_in, float* u_out,
                           const unsigned* red, float kappa, float delta, unsigned* status,
                           float* scale_out, cudaStream_t s, unsigned* conv) {
  if (d.zv != 2 && d.zv != 4) d.zv = 1;
  return NADMM_ZV_LAUNCH(k_compose, d, s, d, w, u_in, u_out, (const unsigned*)red, kappa, delta,
                         status, scale_out, conv);
}

cudaError_t launch_downsample2(Dims coarse, const float* fine, float* out, cudaStream_t s) {
  return launch_pdl(k_downsample2, grid3(coarse, coarse.nz), kBlock, 0, s, coarse, fine, out);
}

cudaError_t launch_upsample_u(Dims coarse, Dims fine, const float* uc, float* uf, cudaStream_t s) {
  return launch_pdl(k_upsample_u, grid3(fine, fine.nz), kBlock, 0, s, coarse, fine, uc, uf);
}

cudaError_t launch_jacobian(Dims d, const float* u, float* det, unsigned* count, cudaStream_t s) {
  return launch_pdl(k_jacobian, grid3(d, d.nz), kBlock, 0, s, d, u, det, count);
}

}  // namespace nadmm
