// Inner Nesterov-accelerated ADMM loop (Eq. 5, closed forms of Eq. 6).
//
// One ADMM iteration is two kernels:
//   plane pass  (per R rows of a z-plane, all 3 components):
//       inverse x-DFT of the filtered spectrum -> w^{k-1};
//       b^{k-1} = y^{k-1} - w^{k-1}                         (Eq. 5, line 3)
//       w_hat^k = w^{k-1} + beta_{k-1} (w^{k-1} - w^{k-2}),
//       b_hat^k likewise                                   (Eq. 5, lines 5-6)
//       v^k = closed-form v-step at u = w_hat^k - b_hat^k   (Eq. 6, s = 1 / 2)
//       y^k = v^k + b_hat^k; forward x-DFT of y^k (two real rows per complex
//       line), scattered as a half spectrum [3][nkx][nz][ny];
//   pencil pass (per (component, kx) plane of the half spectrum):
//       forward y- and z-DFTs, multiply by 1/(1 + gamma K^n) / (nx ny nz),
//       inverse z- and y-DFTs                             (Eq. 5 line 2, Eq. 6)
// so the w-step's 3D transform pair costs two global passes and no
// transpose kernels.  The phase functions below are plain C++ over
// (tid, nthr); kernels separate them with barriers.
#include <cuda_runtime.h>

#include "fft_device.cuh"
#include "nadmm_internal.h"

namespace nadmm {

// ---------------------------------------------------------------- v-step
// s = 2 (Eq. 6 middle, Sherman-Morrison): v = u - rho(u) J / (theta + |J|^2)
// s = 1 (Eq. 6 top):  z = theta rho(u) / (|J|^2 + eps),
//                     v = u - z / max(|z|, 1) * J / theta
NADMM_HD void v_step(int data_term, float theta, float eps, const float (&J)[3], float c,
                     const float (&u)[3], float (&v)[3]) {
  float rho = J[0] * u[0] + J[1] * u[1] + J[2] * u[2] + c;
  float jj = J[0] * J[0] + J[1] * J[1] + J[2] * J[2];
  float f;
  if (data_term == 2) {
    f = rho / (theta + jj);
  } else {
    float z = theta * rho / (jj + eps);
    float t = z / fmaxf(fabsf(z), 1.0f);
    f = t / theta;
  }
  v[0] = u[0] - f * J[0];
  v[1] = u[1] - f * J[1];
  v[2] = u[2] - f * J[2];
}

// ---------------------------------------------------------------- plane pass
// Lines: line l = comp * (R/2) + r holds rows (y0 + r) [real part] and
// (y0 + r + R/2) [imaginary part] of component comp, at pitch a.pitch.

// Half spectrum (A, B of the two rows) -> full complex line Z = A + iB.
NADMM_HD void plane_gather(const PlaneArgs& a, float2* lines, int z, int y0, int tid, int nthr) {
  const int h = a.R / 2;
  const int total = 3 * a.nkx * h;
  for (int g = tid; g < total; g += nthr) {
    int r = g % h;
    int rest = g / h;
    int kx = rest % a.nkx;
    int comp = rest / a.nkx;
    const float2* src = a.spec + ((size_t)(comp * a.nkx + kx) * a.nz + z) * a.ny + y0 + r;
    float2 A = src[0];
    float2 B = src[h];
    float2* line = lines + (comp * h + r) * a.pitch;
    if (kx == 0 || 2 * kx == a.nx) {
      line[a.posx[kx]] = make_float2(A.x, B.x);
    } else {
      line[a.posx[kx]] = make_float2(A.x - B.y, A.y + B.x);
      line[a.posx[a.nx - kx]] = make_float2(A.x + B.y, B.x - A.y);
    }
  }
}

// Full complex line Z -> half spectra A = (Z_k + conj Z_{N-k})/2,
// B = (Z_k - conj Z_{N-k})/(2i) of the two real rows.
NADMM_HD void plane_scatter(const PlaneArgs& a, const float2* lines, int z, int y0, int tid,
                            int nthr) {
  const int h = a.R / 2;
  const int total = 3 * a.nkx * h;
  for (int g = tid; g < total; g += nthr) {
    int r = g % h;
    int rest = g / h;
    int kx = rest % a.nkx;
    int comp = rest / a.nkx;
    const float2* line = lines + (comp * h + r) * a.pitch;
    float2 Zk = line[a.posx[kx]];
    float2 Zm = line[a.posx[kx == 0 ? 0 : a.nx - kx]];
    float2* dst = a.spec + ((size_t)(comp * a.nkx + kx) * a.nz + z) * a.ny + y0 + r;
    dst[0] = make_float2(0.5f * (Zk.x + Zm.x), 0.5f * (Zk.y - Zm.y));
    dst[h] = make_float2(0.5f * (Zk.y + Zm.y), 0.5f * (Zm.x - Zk.x));
  }
}

template <int IN, bool PREV, bool STEP>
NADMM_HD void plane_pointwise(const PlaneArgs& a, float2* lines, int z, int y0, int tid,
                              int nthr) {
  const int h = a.R / 2;
  const size_t V = (size_t)a.nx * a.ny * a.nz;
  const int total = h * a.nx;
  for (int g = tid; g < total; g += nthr) {
    int x = g % a.nx;
    int r = g / a.nx;
    float ynew[2][3];
    for (int half = 0; half < 2; ++half) {
      const size_t vox = ((size_t)z * a.ny + (y0 + r + half * h)) * a.nx + x;
      float wk1[3], bk1[3], wh[3], bh[3];
      for (int comp = 0; comp < 3; ++comp) {
        const size_t i = comp * V + vox;
        if (IN == IN_SPEC) {
          float2 l = lines[(comp * h + r) * a.pitch + x];
          wk1[comp] = half ? l.y : l.x;
          bk1[comp] = (a.y != nullptr) ? a.y[i] - wk1[comp] : 0.0f;
        } else if (IN == IN_STATE) {
          wk1[comp] = a.w_in[i];
          bk1[comp] = a.b_in[i];
        } else if (IN == IN_FIELD) {
          wk1[comp] = a.w_in[i];
          bk1[comp] = 0.0f;
        } else {
          wk1[comp] = 0.0f;
          bk1[comp] = 0.0f;
        }
        if (STEP && PREV) {
          const float* wsrc = (IN == IN_STATE) ? a.wprev_in : a.wp;
          const float* bsrc = (IN == IN_STATE) ? a.bprev_in : a.bp;
          wh[comp] = wk1[comp] + a.beta * (wk1[comp] - wsrc[i]);
          bh[comp] = bk1[comp] + a.beta * (bk1[comp] - bsrc[i]);
        } else {
          wh[comp] = wk1[comp];
          bh[comp] = bk1[comp];
        }
        if (!STEP) {
          a.w_out[i] = wk1[comp];
          if (a.b_out != nullptr) a.b_out[i] = bk1[comp];
        } else if (IN == IN_SPEC || IN == IN_STATE) {
          a.wp[i] = wk1[comp];
          a.bp[i] = bk1[comp];
        }
      }
      if (STEP) {
        if (IN == IN_FIELD) {
          for (int comp = 0; comp < 3; ++comp) ynew[half][comp] = wk1[comp];
        } else {
          float Jv[3], u[3], v[3];
          for (int comp = 0; comp < 3; ++comp) {
            Jv[comp] = a.J[comp * V + vox];
            u[comp] = wh[comp] - bh[comp];
          }
          v_step(a.data_term, a.theta, a.eps, Jv, a.c[vox], u, v);
          for (int comp = 0; comp < 3; ++comp) {
            ynew[half][comp] = v[comp] + bh[comp];
            if (a.y != nullptr) a.y[comp * V + vox] = ynew[half][comp];
          }
        }
      }
    }
    if (STEP) {
      for (int comp = 0; comp < 3; ++comp)
        lines[(comp * h + r) * a.pitch + x] = make_float2(ynew[0][comp], ynew[1][comp]);
    }
  }
}

#if defined(__CUDACC__)
#define NADMM_SYNC() __syncthreads()
#else
#define NADMM_SYNC()
#endif

constexpr int kPlaneThreads = 256;
constexpr int kPencilThreads = 512;

template <int IN, bool PREV, bool STEP>
__global__ void __launch_bounds__(kPlaneThreads) k_plane(PlaneArgs a) {
  extern __shared__ float2 lines[];
  const int tiles_y = a.ny / a.R;
  const int z = blockIdx.x / tiles_y;
  const int y0 = (blockIdx.x % tiles_y) * a.R;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int nlines = 3 * (a.R / 2);
  if (IN == IN_SPEC) {
    plane_gather(a, lines, z, y0, tid, nthr);
    NADMM_SYNC();
    for (int s = a.px.nst - 1; s >= 0; --s) {
      fft_stage<true>(a.px, s, lines, nlines, 1, a.pitch, a.twx, tid, nthr);
      NADMM_SYNC();
    }
  }
  plane_pointwise<IN, PREV, STEP>(a, lines, z, y0, tid, nthr);
  if (STEP) {
    NADMM_SYNC();
    for (int s = 0; s < a.px.nst; ++s) {
      fft_stage<false>(a.px, s, lines, nlines, 1, a.pitch, a.twx, tid, nthr);
      NADMM_SYNC();
    }
    plane_scatter(a, lines, z, y0, tid, nthr);
  }
}

// ---------------------------------------------------------------- pencil pass
NADMM_HD void pencil_symbol(const PencilArgs& a, float2* sm, int kx, int tid, int nthr) {
  const int total = a.ny * a.nz;
  const float kxv = a.Kx[kx];
  for (int g = tid; g < total; g += nthr) {
    int yy = g % a.ny;
    int zz = g / a.ny;
    float K = kxv + a.Ky[yy] + a.Kz[zz];
    float Kn = K;
    for (int i = 1; i < a.order_n; ++i) Kn *= K;
    float S = a.scale / (1.0f + a.gamma * Kn);
    float2& e = sm[zz * a.pitch + yy];
    e = cscale(e, S);
  }
}

__global__ void __launch_bounds__(kPencilThreads) k_pencil(PencilArgs a) {
  extern __shared__ float2 sm[];
  const int plane = blockIdx.x;
  const int kx = plane % a.nkx;
  const int tid = threadIdx.x, nthr = blockDim.x;
  float2* g = a.spec + (size_t)plane * a.ny * a.nz;
  const int total = a.ny * a.nz;
  for (int i = tid; i < total; i += nthr) {
    int yy = i % a.ny, zz = i / a.ny;
    sm[zz * a.pitch + yy] = g[i];
  }
  __syncthreads();
  for (int s = 0; s < a.py.nst; ++s) {
    fft_stage<false>(a.py, s, sm, a.nz, 1, a.pitch, a.twy, tid, nthr);
    __syncthreads();
  }
  for (int s = 0; s < a.pz.nst; ++s) {
    fft_stage<false>(a.pz, s, sm, a.ny, a.pitch, 1, a.twz, tid, nthr);
    __syncthreads();
  }
  pencil_symbol(a, sm, kx, tid, nthr);
  __syncthreads();
  for (int s = a.pz.nst - 1; s >= 0; --s) {
    fft_stage<true>(a.pz, s, sm, a.ny, a.pitch, 1, a.twz, tid, nthr);
    __syncthreads();
  }
  for (int s = a.py.nst - 1; s >= 0; --s) {
    fft_stage<true>(a.py, s, sm, a.nz, 1, a.pitch, a.twy, tid, nthr);
    __syncthreads();
  }
  for (int i = tid; i < total; i += nthr) {
    int yy = i % a.ny, zz = i / a.ny;
    g[i] = sm[zz * a.pitch + yy];
  }
}

// ---------------------------------------------------------------- launchers
size_t plane_smem_bytes(int R, int pitch) { return (size_t)3 * (R / 2) * pitch * sizeof(float2); }
size_t pencil_smem_bytes(int ny, int nz, int pitch) {
  (void)ny;
  return (size_t)nz * pitch * sizeof(float2);
}

template <int IN, bool PREV, bool STEP>
static cudaError_t set_plane_attr(size_t smem) {
  return cudaFuncSetAttribute(k_plane<IN, PREV, STEP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
}

cudaError_t configure_admm_kernels(size_t plane_smem, size_t pencil_smem) {
  cudaError_t e;
  if ((e = set_plane_attr<IN_NONE, false, true>(plane_smem)) != cudaSuccess) return e;
  if ((e = set_plane_attr<IN_SPEC, false, true>(plane_smem)) != cudaSuccess) return e;
  if ((e = set_plane_attr<IN_SPEC, true, true>(plane_smem)) != cudaSuccess) return e;
  if ((e = set_plane_attr<IN_SPEC, false, false>(plane_smem)) != cudaSuccess) return e;
  if ((e = set_plane_attr<IN_STATE, false, true>(plane_smem)) != cudaSuccess) return e;
  if ((e = set_plane_attr<IN_STATE, true, true>(plane_smem)) != cudaSuccess) return e;
  if ((e = set_plane_attr<IN_FIELD, false, true>(plane_smem)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_pencil, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)pencil_smem);
}

cudaError_t launch_plane(int in_mode, bool prev, bool step, const PlaneArgs& a, cudaStream_t s) {
  dim3 grid((unsigned)((a.ny / a.R) * a.nz));
  size_t smem = plane_smem_bytes(a.R, a.pitch);
  int key = in_mode * 4 + (prev ? 2 : 0) + (step ? 1 : 0);
  switch (key) {
    case IN_NONE * 4 + 1: k_plane<IN_NONE, false, true><<<grid, kPlaneThreads, smem, s>>>(a); break;
    case IN_SPEC * 4 + 1: k_plane<IN_SPEC, false, true><<<grid, kPlaneThreads, smem, s>>>(a); break;
    case IN_SPEC * 4 + 3: k_plane<IN_SPEC, true, true><<<grid, kPlaneThreads, smem, s>>>(a); break;
    case IN_SPEC * 4 + 0: k_plane<IN_SPEC, false, false><<<grid, kPlaneThreads, smem, s>>>(a); break;
    case IN_STATE * 4 + 1: k_plane<IN_STATE, false, true><<<grid, kPlaneThreads, smem, s>>>(a); break;
    case IN_STATE * 4 + 3: k_plane<IN_STATE, true, true><<<grid, kPlaneThreads, smem, s>>>(a); break;
    case IN_FIELD * 4 + 1: k_plane<IN_FIELD, false, true><<<grid, kPlaneThreads, smem, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_pencil(const PencilArgs& a, cudaStream_t s) {
  dim3 grid((unsigned)(3 * a.nkx));
  k_pencil<<<grid, kPencilThreads, pencil_smem_bytes(a.ny, a.nz, a.pitch), s>>>(a);
  return cudaGetLastError();
}

}  // namespace nadmm
