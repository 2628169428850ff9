// Reverse mode of the registration (the adjoints of the outer step and of
// the ADMM iterations of Eq. 5 with the s = 2 data step of Eq. 6), and the
// SSD loss 1/2 sum (I1 o (Id + u) - I0)^2 with its gradient.
//
// Conventions at non-smooth points, identical to the forward kernels'
// arithmetic: a sample coordinate clamped to [0, dim - 1] passes no gradient
// unless it lies strictly inside; sign(0) = 0; the maxima of the velocity
// bound share the gradient equally among all entries that attain them
// (bit-equal to the forward maximum); s = min(1, kappa/m_jac, delta/m_abs)
// follows the first candidate, in that order, that attains it.
#include <cuda_runtime.h>
#include <math.h>

#include "grid_common.cuh"
#include "nadmm_internal.h"

namespace nadmm {

namespace {

struct TriGrad {
  float gx, gy, gz;
};

// Gradient of g * trilerp(f, p) with respect to p (masked where the clamp
// is active) and, if gf is not null, the scatter of g times the trilinear
// weights into gf.
__device__ __forceinline__ TriGrad trilerp_vjp(const float* __restrict__ f, float* gf, Dims d,
                                               float px, float py, float pz, float g) {
  const bool inx = px > 0.0f && px < (float)(d.nx - 1);
  const bool iny = py > 0.0f && py < (float)(d.ny - 1);
  const bool inz = pz > 0.0f && pz < (float)(d.nz - 1);
  px = fminf(fmaxf(px, 0.0f), (float)(d.nx - 1));
  py = fminf(fmaxf(py, 0.0f), (float)(d.ny - 1));
  pz = fminf(fmaxf(pz, 0.0f), (float)(d.nz - 1));
  const int ix = min((int)floorf(px), d.nx - 2);
  const int iy = min((int)floorf(py), d.ny - 2);
  const int iz = min((int)floorf(pz), d.nz - 2);
  const float fx = px - (float)ix, fy = py - (float)iy, fz = pz - (float)iz;
  const float ex = 1.0f - fx, ey = 1.0f - fy, ez = 1.0f - fz;
  const size_t sx = 1, sy = (size_t)d.nx, sz = (size_t)d.nx * d.ny;
  const size_t o = (size_t)iz * sz + (size_t)iy * sy + ix;
  const float* p = f + o;
  const float c000 = __ldg(p), c001 = __ldg(p + sx);
  const float c010 = __ldg(p + sy), c011 = __ldg(p + sy + sx);
  const float c100 = __ldg(p + sz), c101 = __ldg(p + sz + sx);
  const float c110 = __ldg(p + sz + sy), c111 = __ldg(p + sz + sy + sx);
  const float dfx = ((c001 - c000) * ey + (c011 - c010) * fy) * ez +
                    ((c101 - c100) * ey + (c111 - c110) * fy) * fz;
  const float dfy = ((c010 - c000) * ex + (c011 - c001) * fx) * ez +
                    ((c110 - c100) * ex + (c111 - c101) * fx) * fz;
  const float dfz = ((c100 - c000) * ex + (c101 - c001) * fx) * ey +
                    ((c110 - c010) * ex + (c111 - c011) * fx) * fy;
  if (gf != nullptr && g != 0.0f) {
    float* q = gf + o;
    atomicAdd(q, g * ex * ey * ez);
    atomicAdd(q + sx, g * fx * ey * ez);
    atomicAdd(q + sy, g * ex * fy * ez);
    atomicAdd(q + sy + sx, g * fx * fy * ez);
    atomicAdd(q + sz, g * ex * ey * fz);
    atomicAdd(q + sz + sx, g * fx * ey * fz);
    atomicAdd(q + sz + sy, g * ex * fy * fz);
    atomicAdd(q + sz + sy + sx, g * fx * fy * fz);
  }
  return TriGrad{inx ? g * dfx : 0.0f, iny ? g * dfy : 0.0f, inz ? g * dfz : 0.0f};
}

// Sum of v over the block, added to *acc (double) by one thread.  All
// threads of the block must call it; the closing barrier lets a following
// call reuse the (single, per-block) shared array.
__device__ __forceinline__ void block_add(double v, double* acc) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  __shared__ double part[kBY];
  if (threadIdx.x == 0) part[threadIdx.y] = v;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    double t = 0.0;
    for (int k = 0; k < kBY; ++k) t += part[k];
    atomicAdd(acc, t);
  }
  __syncthreads();
}

enum BoundBranch { kBranchOne = 0, kBranchJac = 1, kBranchAbs = 2 };

// Which candidate of s = min(1, kappa/m_jac, delta/m_abs) is active.
__device__ __forceinline__ int bound_branch(const unsigned* red, float kappa, float delta) {
  const float mabs = __uint_as_float(red[0]), mjac = __uint_as_float(red[1]);
  if (!isfinite(mabs) || !isfinite(mjac)) return kBranchOne;
  float s = 1.0f;
  int b = kBranchOne;
  if (isfinite(kappa) && mjac > 0.0f && kappa / mjac < s) {
    s = kappa / mjac;
    b = kBranchJac;
  }
  if (isfinite(delta) && mabs > 0.0f && delta / mabs < s) b = kBranchAbs;
  return b;
}

__device__ __forceinline__ float sgn(float v) { return (float)((v > 0.0f) - (v < 0.0f)); }

// ---------------------------------------------------------------- compose
// u_new(x) = v(x) + u_o(x + v(x)), v = s w:  ubar_prev += scatter of ubar
// (adjoint of the sampled u_o), wbar = s vbar with vbar = ubar + (grad of
// the samples in x + v)^T ubar, acc[0] += <vbar, w> (the gradient of s).
__global__ void __launch_bounds__(kBX * kBY)
    k_compose_vjp(Dims d, const float* __restrict__ u_o, const float* __restrict__ w,
                  const unsigned* red, float kappa, float delta, const float* __restrict__ ubar,
                  float* ubar_prev, float* __restrict__ wbar, double* acc) {
  pdl_wait();
  pdl_trigger();
  const size_t V = (size_t)d.nx * d.ny * d.nz;
  const float s = bound_factor(red, kappa, delta, nullptr);
  const int x = blockIdx.x * kBX + threadIdx.x, y = blockIdx.y * kBY + threadIdx.y;
  const int z = blockIdx.z;
  double part = 0.0;
  if (x < d.nx && y < d.ny) {
    const size_t i = ((size_t)z * d.ny + y) * d.nx + x;
    const float w0 = w[i], w1 = w[V + i], w2 = w[2 * V + i];
    const float px = (float)x + s * w0, py = (float)y + s * w1, pz = (float)z + s * w2;
    float gv[3] = {ubar[i], ubar[V + i], ubar[2 * V + i]};
    const float g[3] = {gv[0], gv[1], gv[2]};
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
      const TriGrad t = trilerp_vjp(u_o + comp * V, ubar_prev + comp * V, d, px, py, pz, g[comp]);
      gv[0] += t.gx;
      gv[1] += t.gy;
      gv[2] += t.gz;
    }
    wbar[i] = s * gv[0];
    wbar[V + i] = s * gv[1];
    wbar[2 * V + i] = s * gv[2];
    part = (double)gv[0] * w0 + (double)gv[1] * w1 + (double)gv[2] * w2;
  }
  block_add(part, acc);
}

// ---------------------------------------------------------------- bound
// Entries attaining the active maximum (count), then their share of
// d s / d w times acc[0] added to wbar.
__global__ void __launch_bounds__(kBX * kBY)
    k_bound_vjp_count(Dims d, const float* __restrict__ w, const unsigned* red, float kappa,
                      float delta, unsigned* count) {
  pdl_wait();
  pdl_trigger();
  const int branch = bound_branch(red, kappa, delta);
  if (branch == kBranchOne) return;
  const size_t V = (size_t)d.nx * d.ny * d.nz;
  const int x = blockIdx.x * kBX + threadIdx.x, y = blockIdx.y * kBY + threadIdx.y;
  const int z = blockIdx.z;
  unsigned local = 0;
  if (x < d.nx && y < d.ny) {
    const size_t i = ((size_t)z * d.ny + y) * d.nx + x;
    const Nbr nb = neighbours(d, x, y, z, i);
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
      const float* f = w + comp * V;
      if (branch == kBranchJac)
        local += __float_as_uint(jacobian_row(f, nb)) == red[1] ? 1u : 0u;
      else
        local += __float_as_uint(fabsf(__ldg(f + i))) == red[0] ? 1u : 0u;
    }
  }
  for (int off = 16; off > 0; off >>= 1) local += __shfl_xor_sync(0xffffffffu, local, off);
  if (threadIdx.x == 0 && local) atomicAdd(count, local);
}

__global__ void __launch_bounds__(kBX * kBY)
    k_bound_vjp_apply(Dims d, const float* __restrict__ w, const unsigned* red, float kappa,
                      float delta, const double* acc, const unsigned* count, float* wbar) {
  pdl_wait();
  pdl_trigger();
  const int branch = bound_branch(red, kappa, delta);
  if (branch == kBranchOne || *count == 0u) return;
  const size_t V = (size_t)d.nx * d.ny * d.nz;
  const int x = blockIdx.x * kBX + threadIdx.x, y = blockIdx.y * kBY + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= d.nx || y >= d.ny) return;
  const float mabs = __uint_as_float(red[0]), mjac = __uint_as_float(red[1]);
  const float ds = (branch == kBranchJac) ? -kappa / (mjac * mjac) : -delta / (mabs * mabs);
  const float coef = ds * (float)acc[0] / (float)(*count);
  const size_t i = ((size_t)z * d.ny + y) * d.nx + x;
  const Nbr nb = neighbours(d, x, y, z, i);
#pragma unroll
  for (int comp = 0; comp < 3; ++comp) {
    const float* f = w + comp * V;
    float* gw = wbar + comp * V;
    if (branch == kBranchJac) {
      if (__float_as_uint(jacobian_row(f, nb)) != red[1]) continue;
      const size_t pl[3] = {nb.xp, nb.yp, nb.zp}, mi[3] = {nb.xm, nb.ym, nb.zm};
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const float D = 0.5f * (__ldg(f + pl[j]) - __ldg(f + mi[j]));
        const float c = 0.5f * sgn(D) * coef;
        if (c != 0.0f) {
          atomicAdd(gw + pl[j], c);
          atomicAdd(gw + mi[j], -c);
        }
      }
    } else {
      const float a = __ldg(f + i);
      if (__float_as_uint(fabsf(a)) == red[0]) atomicAdd(gw + i, sgn(a) * coef);
    }
  }
}

// ---------------------------------------------------------------- ADMM
// One reverse step k of Eq. 5 (s = 2): from wbar^k, bbar^k (g = wbar -
// bbar and its filtered Sg = S g) to the contributions to J, c, theta,
// gamma = lambda/theta and to wbar, bbar of iterations k-1 (added) and k-2
// (the first contribution, stored).
__global__ void __launch_bounds__(kBX * kBY) k_adj_step(AdjArgs a) {
  pdl_wait();
  pdl_trigger();
  const Dims d = a.d;
  const size_t V = (size_t)d.nx * d.ny * d.nz;
  const int x = blockIdx.x * kBX + threadIdx.x, y = blockIdx.y * kBY + threadIdx.y;
  const int z = blockIdx.z;
  double p_theta = 0.0, p_gamma = 0.0;
  if (x < d.nx && y < d.ny) {
    const size_t i = ((size_t)z * d.ny + y) * d.nx + x;
    const float beta = a.beta;
    float Jv[3], u[3], yb[3];
    float rho = a.c[i], dd = a.theta;
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
      const size_t j = comp * V + i;
      u[comp] = a.uk[j];
      Jv[comp] = a.J[j];
      rho += Jv[comp] * u[comp];
      dd += Jv[comp] * Jv[comp];
      const float sg = a.Sg[j];
      p_gamma += (double)(a.g_in[j] - sg) * a.wk[j];
      yb[comp] = sg + a.Bk[j];
    }
    const float jy = Jv[0] * yb[0] + Jv[1] * yb[1] + Jv[2] * yb[2];
    const float inv_d = 1.0f / dd;
    const float q = jy * inv_d;
    a.gc[i] += -q;
    p_theta = (double)rho * jy * inv_d * inv_d;
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
      const size_t j = comp * V + i;
      a.gJ[j] += -(rho * inv_d) * yb[comp] - q * u[comp] + 2.0f * rho * q * inv_d * Jv[comp];
      const float ub = yb[comp] - Jv[comp] * q;  // u_bar = w_hat_bar
      const float bb = yb[comp] - ub;             // b_hat_bar
      if (a.W1bar) {
        const float nw = a.W1bar[j] + (1.0f + beta) * ub;
        const float nb = a.B1bar[j] + (1.0f + beta) * bb;
        a.W1bar[j] = nw;
        a.B1bar[j] = nb;
        a.g_out[j] = nw - nb;
      }
      if (a.W2bar) {  // slot of iteration k+1, dead: plain stores
        a.W2bar[j] = -beta * ub;
        a.B2bar[j] = -beta * bb;
      }
    }
    p_gamma *= -(double)a.inv_gamma;
  }
  block_add(p_theta, a.acc + 1);
  block_add(p_gamma, a.acc + 2);
}

// ---------------------------------------------------------------- linearise
// (J, c, I1w) = (grad I1w, I1w - I0, I1 o (Id + u_o)):  I1w_bar = c_bar +
// adjoint of the clamped central differences of J_bar; I0_bar -= c_bar;
// I1_bar += scatter of I1w_bar; ubar_out = ubar_prev + (grad of the I1
// sample)^T I1w_bar.
__device__ __forceinline__ float cdiff_adj(const float* __restrict__ g, size_t i, size_t st, int m,
                                           int n) {
  float t = 0.0f;
  if (m >= 1) t += g[i - st];
  if (m == n - 1) t += g[i];
  if (m <= n - 2) t -= g[i + st];
  if (m == 0) t -= g[i];
  return 0.5f * t;
}

__global__ void __launch_bounds__(kBX * kBY)
    k_linearise_vjp(Dims d, const float* __restrict__ I1, const float* __restrict__ u_o,
                    const float* __restrict__ gJ, const float* __restrict__ gc, float* grad_fixed,
                    float* grad_moving, const float* __restrict__ ubar_prev,
                    float* __restrict__ ubar_out) {
  pdl_wait();
  pdl_trigger();
  const size_t V = (size_t)d.nx * d.ny * d.nz;
  const int x = blockIdx.x * kBX + threadIdx.x, y = blockIdx.y * kBY + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= d.nx || y >= d.ny) return;
  const size_t i = ((size_t)z * d.ny + y) * d.nx + x;
  const float cb = gc[i];
  const float gw = cb + cdiff_adj(gJ, i, 1, x, d.nx) +
                   cdiff_adj(gJ + V, i, (size_t)d.nx, y, d.ny) +
                   cdiff_adj(gJ + 2 * V, i, (size_t)d.nx * d.ny, z, d.nz);
  grad_fixed[i] -= cb;
  const float px = (float)x + u_o[i], py = (float)y + u_o[V + i], pz = (float)z + u_o[2 * V + i];
  const TriGrad t = trilerp_vjp(I1, grad_moving, d, px, py, pz, gw);
  ubar_out[i] = ubar_prev[i] + t.gx;
  ubar_out[V + i] = ubar_prev[V + i] + t.gy;
  ubar_out[2 * V + i] = ubar_prev[2 * V + i] + t.gz;
}

// d/d lambda = g_gamma / theta; d/d theta = (data-step part) - g_gamma lambda / theta^2
__global__ void k_param_grads(const double* acc, float lambda, float theta, float* glam,
                              float* gtheta) {
  pdl_wait();
  pdl_trigger();
  if (threadIdx.x != 0) return;
  const double gg = acc[2];
  if (glam) *glam = (float)(gg / theta);
  if (gtheta) *gtheta = (float)(acc[1] - gg * lambda / ((double)theta * theta));
}

// ---------------------------------------------------------------- SSD loss
__global__ void __launch_bounds__(kBX * kBY)
    k_ssd(Dims d, const float* __restrict__ I0, const float* __restrict__ I1,
          const float* __restrict__ u, double* acc) {
  pdl_wait();
  pdl_trigger();
  const size_t V = (size_t)d.nx * d.ny * d.nz;
  const int x = blockIdx.x * kBX + threadIdx.x, y = blockIdx.y * kBY + threadIdx.y;
  const int z = blockIdx.z;
  double part = 0.0;
  if (x < d.nx && y < d.ny) {
    const size_t i = ((size_t)z * d.ny + y) * d.nx + x;
    const float r = trilerp(I1, d, (float)x + u[i], (float)y + u[V + i], (float)z + u[2 * V + i]) -
                    I0[i];
    part = 0.5 * (double)r * r;
  }
  block_add(part, acc);
}

__global__ void k_store_loss(const double* acc, float* loss) {
  pdl_wait();
  pdl_trigger();
  if (threadIdx.x == 0) *loss = (float)acc[0];
}

__global__ void __launch_bounds__(kBX * kBY)
    k_ssd_vjp(Dims d, const float* __restrict__ I0, const float* __restrict__ I1,
              const float* __restrict__ u, const float* gL, float* __restrict__ grad_fixed,
              float* grad_moving, float* __restrict__ grad_u) {
  pdl_wait();
  pdl_trigger();
  const size_t V = (size_t)d.nx * d.ny * d.nz;
  const int x = blockIdx.x * kBX + threadIdx.x, y = blockIdx.y * kBY + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= d.nx || y >= d.ny) return;
  const size_t i = ((size_t)z * d.ny + y) * d.nx + x;
  const float px = (float)x + u[i], py = (float)y + u[V + i], pz = (float)z + u[2 * V + i];
  const float g = *gL * (trilerp(I1, d, px, py, pz) - I0[i]);
  if (grad_fixed) grad_fixed[i] = -g;
  const TriGrad t = trilerp_vjp(I1, grad_moving, d, px, py, pz, g);
  if (grad_u) {
    grad_u[i] = t.gx;
    grad_u[V + i] = t.gy;
    grad_u[2 * V + i] = t.gz;
  }
}

dim3 grid3(Dims d) {
  return dim3((unsigned)((d.nx + kBX - 1) / kBX), (unsigned)((d.ny + kBY - 1) / kBY),
              (unsigned)d.nz);
}
const dim3 kBlock(kBX, kBY);

}  // namespace

cudaError_t launch_compose_vjp(Dims d, const float* u_o, const float* w, const unsigned* red,
                               float kappa, float delta, const float* ubar, float* ubar_prev,
                               float* wbar, double* acc, cudaStream_t s) {
  return launch_pdl(k_compose_vjp, grid3(d), kBlock, 0, s, d, u_o, w, red, kappa, delta, ubar,
                    ubar_prev, wbar, acc);
}

cudaError_t launch_bound_vjp(Dims d, const float* w, const unsigned* red, float kappa,
                             float delta, const double* acc, unsigned* count, float* wbar,
                             cudaStream_t s) {
  cudaError_t e = launch_pdl(k_bound_vjp_count, grid3(d), kBlock, 0, s, d, w, red, kappa, delta,
                             count);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_bound_vjp_apply, grid3(d), kBlock, 0, s, d, w, red, kappa, delta, acc,
                    (const unsigned*)count, wbar);
}

cudaError_t launch_adj_step(const AdjArgs& a, cudaStream_t s) {
  return launch_pdl(k_adj_step, grid3(a.d), kBlock, 0, s, a);
}

cudaError_t launch_linearise_vjp(Dims d, const float* I1, const float* u_o, const float* gJ,
                                 const float* gc, float* grad_fixed, float* grad_moving,
                                 const float* ubar_prev, float* ubar_out, cudaStream_t s) {
  return launch_pdl(k_linearise_vjp, grid3(d), kBlock, 0, s, d, I1, u_o, gJ, gc, grad_fixed,
                    grad_moving, ubar_prev, ubar_out);
}

cudaError_t launch_param_grads(const double* acc, float lambda, float theta, float* glam,
                               float* gtheta, cudaStream_t s) {
  return launch_pdl(k_param_grads, dim3(1), dim3(32), 0, s, acc, lambda, theta, glam, gtheta);
}

cudaError_t launch_ssd(Dims d, const float* I0, const float* I1, const float* u, double* acc,
                       float* loss, cudaStream_t s) {
  cudaError_t e = launch_pdl(k_ssd, grid3(d), kBlock, 0, s, d, I0, I1, u, acc);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_store_loss, dim3(1), dim3(32), 0, s, (const double*)acc, loss);
}

cudaError_t launch_ssd_vjp(Dims d, const float* I0, const float* I1, const float* u,
                           const float* gL, float* grad_fixed, float* grad_moving, float* grad_u,
                           cudaStream_t s) {
  return launch_pdl(k_ssd_vjp, grid3(d), kBlock, 0, s, d, I0, I1, u, gL, grad_fixed,
                    grad_moving, grad_u);
}

}  // namespace nadmm
