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
// transpose kernels.
//
// Data movement: the plane pass brings its real-space tiles (y, the w/b state,
// J, c) into shared memory with TMA bulk copies issued at kernel start, so
// they stream in while the spectrum is gathered and inverse-transformed; the
// pencil pass moves its whole (ny x nz) plane in and out with bulk copies.
// Every mbarrier wait is bounded: on expiry the kernel records a status bit
// and returns instead of spinning.
#include <cuda_runtime.h>

#include <mutex>

#include "fft_device.cuh"
#include "lane_fft.cuh"
#include "tma.cuh"
#include "nadmm_internal.h"
#include "plan.h"
#include "vstep.cuh"

namespace nadmm {

// TMA / mbarrier helpers: tma.cuh

// Self-test of the timeout path: one barrier that nothing ever arrives at
// (no copy is issued), waited on with the bounded wait of the passes; the
// expired wait sets the status bit and the kernel returns normally.
__global__ void k_wait_selftest(unsigned* status, int attempts) {
#if defined(__CUDA_ARCH__)
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  const bool ok = __syncthreads_and(mbar_wait_bounded(&bar, 0, attempts));
  if (!ok && threadIdx.x == 0 && status != nullptr) atomicOr(status, kStatusTimeout);
#endif
}

cudaError_t launch_wait_selftest(unsigned* status, int attempts, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(status, attempts);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- plane pass
// Shared-memory staging of the real-space tiles: slot s holds R rows x nx.
struct FieldMap {
  int y, w, b, wp, bp, J, c, n;
};

template <int IN, bool PREV, bool STEP>
NADMM_HD constexpr FieldMap field_map() {
  FieldMap f{-1, -1, -1, -1, -1, -1, -1, 0};
  int n = 0;
  if (IN == IN_SPEC && STEP) { f.y = n; n += 3; }
  if (IN == IN_STATE || IN == IN_FIELD) { f.w = n; n += 3; }
  if (IN == IN_STATE) { f.b = n; n += 3; }
  if (STEP && PREV) { f.wp = n; n += 3; f.bp = n; n += 3; }
  if (STEP && IN != IN_FIELD) { f.J = n; n += 3; f.c = n; n += 1; }
  f.n = n;
  return f;
}

constexpr int kGatherItems = 4;   // spectrum values per thread held in flight per round
enum PlaneExtra : int { kPlanePlain = 0, kPlaneConv = 1, kPlaneHist = 2 };
constexpr int kPlaneThreads = 256;
constexpr int kSpecIssuer = 32;  // lane 0 of warp 1 issues the spectrum-block copy

// Lines: line l = comp * (R/2) + r holds rows (y0 + r) [real part] and
// (y0 + r + R/2) [imaginary part] of component comp, at pitch a.pitch.

// Half spectrum (A, B of the two rows) -> full complex line Z = A + iB.
// All loads of a thread are issued before its first shared-memory store.
NADMM_HD void plane_gather(const PlaneArgs& a, float2* lines, const int* pos, int z, int y0,
                           int tid, int nthr) {
  const int h = a.R / 2;
  const int total = 3 * a.nkx * h;
  for (int base = 0; base < total; base += kGatherItems * nthr) {
    float2 A[kGatherItems], B[kGatherItems];
#pragma unroll
    for (int it = 0; it < kGatherItems; ++it) {
      const int g = base + tid + it * nthr;
      if (g < total) {
        const int rest = (int)fdiv((uint32_t)g, a.half_div);
        const int r = g - rest * h;
        const int comp = (int)fdiv((uint32_t)rest, a.nkx_div);
        const int kx = rest - comp * a.nkx;
        const float2* src = a.spec + ((size_t)(comp * a.nkx + kx) * a.nz + z) * a.ny + y0 + r;
        A[it] = src[0];
        B[it] = src[h];
      }
    }
#pragma unroll
    for (int it = 0; it < kGatherItems; ++it) {
      const int g = base + tid + it * nthr;
      if (g < total) {
        const int rest = (int)fdiv((uint32_t)g, a.half_div);
        const int r = g - rest * h;
        const int comp = (int)fdiv((uint32_t)rest, a.nkx_div);
        const int kx = rest - comp * a.nkx;
        float2* line = lines + (comp * h + r) * a.pitch;
        const float2 Av = A[it], Bv = B[it];
        if (kx == 0 || 2 * kx == a.nx) {
          line[swz_rt(pos[kx], a.xlog2r2)] = make_float2(Av.x, Bv.x);
        } else {
          line[swz_rt(pos[kx], a.xlog2r2)] = make_float2(Av.x - Bv.y, Av.y + Bv.x);
          line[swz_rt(pos[a.nx - kx], a.xlog2r2)] = make_float2(Av.x + Bv.y, Bv.x - Av.y);
        }
      }
    }
  }
}

// Full complex line Z -> half spectra A = (Z_k + conj Z_{N-k})/2,
// B = (Z_k - conj Z_{N-k})/(2i) of the two real rows.
NADMM_HD void plane_scatter(const PlaneArgs& a, const float2* lines, const int* pos, int z, int y0,
                            int tid, int nthr) {
  const int h = a.R / 2;
  const int total = 3 * a.nkx * h;
  for (int g = tid; g < total; g += nthr) {
    const int rest = (int)fdiv((uint32_t)g, a.half_div);
    const int r = g - rest * h;
    const int comp = (int)fdiv((uint32_t)rest, a.nkx_div);
    const int kx = rest - comp * a.nkx;
    const float2* line = lines + (comp * h + r) * a.pitch;
    const float2 Zk = line[swz_rt(pos[kx], a.xlog2r2)];
    const float2 Zm = line[swz_rt(pos[kx == 0 ? 0 : a.nx - kx], a.xlog2r2)];
    float2* dst = a.spec + ((size_t)(comp * a.nkx + kx) * a.nz + z) * a.ny + y0 + r;
    dst[0] = make_float2(0.5f * (Zk.x + Zm.x), 0.5f * (Zk.y - Zm.y));
    dst[h] = make_float2(0.5f * (Zk.y + Zm.y), 0.5f * (Zm.x - Zk.x));
  }
}

// Point-wise part of the iteration on staged tiles (fld) and lines.
template <int IN, bool PREV, bool STEP, bool MEASURE = false, bool HIST = false>
NADMM_HD void plane_pointwise(const PlaneArgs& a, float* fld, float2* lines, int z, int y0,
                              int tid, int nthr, float* racc = nullptr) {
  constexpr FieldMap F = field_map<IN, PREV, STEP>();
  const int h = a.R / 2;
  const int tile = a.R * a.nx;
  const size_t V = (size_t)a.nx * a.ny * a.nz;
  const int total = h * a.nx;
  for (int g = tid; g < total; g += nthr) {
    const int r = (int)fdiv((uint32_t)g, a.nx_div);
    const int x = g - r * a.nx;
    const int xs = swz_rt(x, a.xlog2r2);  // position of x in the line buffer
    float ynew[2][3];
    for (int half = 0; half < 2; ++half) {
      const int row = r + half * h;
      const int so = row * a.nx + x;  // offset inside a staged tile
      const size_t vox = ((size_t)z * a.ny + (y0 + row)) * a.nx + x;
      float wk1[3], bk1[3], wh[3], bh[3];
#pragma unroll
      for (int comp = 0; comp < 3; ++comp) {
        const size_t i = comp * V + vox;
        if (IN == IN_SPEC) {
          const float2 l = lines[(comp * h + r) * a.pitch + xs];
          wk1[comp] = half ? l.y : l.x;
          if (STEP)
            bk1[comp] = fld[(F.y + comp) * tile + so] - wk1[comp];
          else
            bk1[comp] = (a.b_out != nullptr) ? a.y[i] - wk1[comp] : 0.0f;
        } else if (IN == IN_STATE) {
          wk1[comp] = fld[(F.w + comp) * tile + so];
          bk1[comp] = fld[(F.b + comp) * tile + so];
        } else if (IN == IN_FIELD) {
          wk1[comp] = fld[(F.w + comp) * tile + so];
          bk1[comp] = 0.0f;
        } else {
          wk1[comp] = 0.0f;
          bk1[comp] = 0.0f;
        }
        if (STEP && PREV) {
          if (MEASURE) {  // ADMM residual: change of w and its size
            const float dw = wk1[comp] - fld[(F.wp + comp) * tile + so];
            racc[0] += dw * dw;
            racc[1] += wk1[comp] * wk1[comp];
          }
          wh[comp] = wk1[comp] + a.beta * (wk1[comp] - fld[(F.wp + comp) * tile + so]);
          bh[comp] = bk1[comp] + a.beta * (bk1[comp] - fld[(F.bp + comp) * tile + so]);
        } else {
          wh[comp] = wk1[comp];
          bh[comp] = bk1[comp];
        }
        if (!STEP) {
          a.w_out[i] = wk1[comp];
          if (a.b_out != nullptr) a.b_out[i] = bk1[comp];
        } else if (IN == IN_SPEC || IN == IN_STATE) {
          if (F.wp >= 0) {
            // w^{k-2}, b^{k-2} of this element were read above: their staged
            // tiles take w^{k-1}, b^{k-1} and leave by bulk stores
            fld[(F.wp + comp) * tile + so] = wk1[comp];
            fld[(F.bp + comp) * tile + so] = bk1[comp];
          } else {
            a.wp[i] = wk1[comp];
            a.bp[i] = bk1[comp];
          }
        }
      }
      if (STEP) {
        if (IN == IN_FIELD) {
#pragma unroll
          for (int comp = 0; comp < 3; ++comp) ynew[half][comp] = wk1[comp];
        } else {
          float Jv[3], u[3], v[3];
#pragma unroll
          for (int comp = 0; comp < 3; ++comp) {
            Jv[comp] = fld[(F.J + comp) * tile + so];
            u[comp] = wh[comp] - bh[comp];
            if (HIST) a.u_hist[comp * V + vox] = u[comp];  // reverse-mode recompute
          }
          v_step(a.data_term, a.theta, a.eps, Jv, fld[F.c * tile + so], u, v);
#pragma unroll
          for (int comp = 0; comp < 3; ++comp) {
            ynew[half][comp] = v[comp] + bh[comp];
            if (F.y >= 0)  // y^{k-1} of this element was read above
              fld[(F.y + comp) * tile + so] = ynew[half][comp];
            else if (a.y != nullptr)
              a.y[comp * V + vox] = ynew[half][comp];
          }
        }
      }
    }
    if (STEP) {
#pragma unroll
      for (int comp = 0; comp < 3; ++comp)
        lines[(comp * h + r) * a.pitch + xs] = make_float2(ynew[0][comp], ynew[1][comp]);
    }
  }
}

// Shared-memory layout of the plane pass (byte offsets).
struct PlaneSmem {
  size_t fld, lines, total;
};

NADMM_HD PlaneSmem plane_layout(const PlaneArgs& a, int nfields) {
  PlaneSmem L;
  size_t o = 16;  // two mbarriers: field tiles, spectrum block
  L.fld = o;
  o += (size_t)nfields * a.R * a.nx * sizeof(float);
  o = (o + 127) & ~(size_t)127;  // tensor copies land here
  L.lines = o;
  o += (size_t)3 * (a.R / 2) * a.pitch * sizeof(float2);
  L.total = (o + 15) & ~(size_t)15;
  return L;
}

#if defined(__CUDA_ARCH__)
// Spectrum block moved by tensor copies: box {R, 1, 3 nkx} lands densely at
// the start of the line buffer as T[ckx][r] (ckx = comp nkx + kx, r < R).
// Unpack it in place into the complex lines of the two-for-one transform:
// every thread first reads all its items, then (after a barrier) writes.
__device__ __forceinline__ void plane_unpack(const PlaneArgs& a, float2* lines,
                                             const int* __restrict__ pos, int tid, int nthr) {
  const int h = a.R / 2;
  const int total = 3 * a.nkx * h;
  const float2* T = lines;
  float2 A[kGatherItems], B[kGatherItems];
#pragma unroll
  for (int it = 0; it < kGatherItems; ++it) {
    const int g = tid + it * nthr;
    if (g < total) {
      const int rest = (int)fdiv((uint32_t)g, a.half_div);  // ckx
      const int r = g - rest * h;
      A[it] = T[rest * a.R + r];
      B[it] = T[rest * a.R + r + h];
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < kGatherItems; ++it) {
    const int g = tid + it * nthr;
    if (g < total) {
      const int rest = (int)fdiv((uint32_t)g, a.half_div);
      const int r = g - rest * h;
      const int comp = (int)fdiv((uint32_t)rest, a.nkx_div);
      const int kx = rest - comp * a.nkx;
      float2* line = lines + (comp * h + r) * a.pitch;
      const float2 Av = A[it], Bv = B[it];
      if (kx == 0 || 2 * kx == a.nx) {
        line[swz_rt(pos[kx], a.xlog2r2)] = make_float2(Av.x, Bv.x);
      } else {
        line[swz_rt(pos[kx], a.xlog2r2)] = make_float2(Av.x - Bv.y, Av.y + Bv.x);
        line[swz_rt(pos[a.nx - kx], a.xlog2r2)] = make_float2(Av.x + Bv.y, Bv.x - Av.y);
      }
    }
  }
}

// Inverse of plane_unpack for the forward transform's output: half spectra
// of the two rows of each line, packed in place as T[ckx][r].
__device__ __forceinline__ void plane_pack(const PlaneArgs& a, float2* lines,
                                           const int* __restrict__ pos, int tid, int nthr) {
  const int h = a.R / 2;
  const int total = 3 * a.nkx * h;
  float2 A[kGatherItems], B[kGatherItems];
#pragma unroll
  for (int it = 0; it < kGatherItems; ++it) {
    const int g = tid + it * nthr;
    if (g < total) {
      const int rest = (int)fdiv((uint32_t)g, a.half_div);
      const int r = g - rest * h;
      const int comp = (int)fdiv((uint32_t)rest, a.nkx_div);
      const int kx = rest - comp * a.nkx;
      const float2* line = lines + (comp * h + r) * a.pitch;
      const float2 Zk = line[swz_rt(pos[kx], a.xlog2r2)];
      const float2 Zm = line[swz_rt(pos[kx == 0 ? 0 : a.nx - kx], a.xlog2r2)];
      A[it] = make_float2(0.5f * (Zk.x + Zm.x), 0.5f * (Zk.y - Zm.y));
      B[it] = make_float2(0.5f * (Zk.y + Zm.y), 0.5f * (Zm.x - Zk.x));
    }
  }
  __syncthreads();
  float2* T = lines;
#pragma unroll
  for (int it = 0; it < kGatherItems; ++it) {
    const int g = tid + it * nthr;
    if (g < total) {
      const int rest = (int)fdiv((uint32_t)g, a.half_div);
      const int r = g - rest * h;
      T[rest * a.R + r] = A[it];
      T[rest * a.R + r + h] = B[it];
    }
  }
}

// ADMM residual of the pass (w^{k-1} against w^{k-2}): CTA sums into
// conv_acc[0..1]; the last CTA to report decides the ADMM stop.
__device__ __forceinline__ void plane_residual(const PlaneArgs& a, const float (&racc)[2]) {
  float d = racc[0], w = racc[1];
  for (int off = 16; off > 0; off >>= 1) {
    d += __shfl_xor_sync(0xffffffffu, d, off);
    w += __shfl_xor_sync(0xffffffffu, w, off);
  }
  __shared__ float pd[kPlaneThreads / 32], pw[kPlaneThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    pd[warp] = d;
    pw[warp] = w;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sd = 0.0, sw = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      sd += pd[k];
      sw += pw[k];
    }
    atomicAdd(a.conv_acc, sd);
    atomicAdd(a.conv_acc + 1, sw);
    __threadfence();
    if (atomicAdd(a.conv + kConvPlaneDone, 1u) == gridDim.x - 1) {  // last CTA
      __threadfence();
      const double d2 = atomicAdd(a.conv_acc, 0.0), w2 = atomicAdd(a.conv_acc + 1, 0.0);
      a.conv[kConvInner] = (sqrt(d2) <= (double)a.admm_tol * sqrt(w2)) ? 1u : 0u;
      // the velocity is w^{k-1}: iteration k, started by this pass, does not count
      if (a.conv[kConvInner]) atomicSub(a.conv + kConvAdmmRun, 1u);
      a.conv_acc[0] = 0.0;
      a.conv_acc[1] = 0.0;
      a.conv[kConvPlaneDone] = 0u;
    }
  }
}

// x-DFT of the CTA's lines by groups of xr2 lanes (lane FFT, swizzled lines).
template <bool INV>
__device__ __forceinline__ void plane_lane_fft(const PlaneArgs& a, float2* lines,
                                               const float2* __restrict__ tw, int nlines, int tid) {
  const int g = tid >> a.xlog2r2, l = tid & (a.xr2 - 1);
  if (g < nlines) {
    const int lane = tid & 31;
    const unsigned gmask = ((a.xr2 == 32) ? 0xffffffffu : ((1u << a.xr2) - 1u)) << (lane & ~(a.xr2 - 1));
    lane_line_fft_rt<INV>(a.xr1, a.xr2, lines + g * a.pitch, tw, l, gmask);
  }
}

template <int IN, bool PREV, bool STEP>
__device__ __forceinline__ const float* field_src(const PlaneArgs& a, int slot) {
  constexpr FieldMap F = field_map<IN, PREV, STEP>();
  const size_t V = (size_t)a.nx * a.ny * a.nz;
  auto in_range = [](int s, int base, int cnt) { return base >= 0 && s >= base && s < base + cnt; };
  if (in_range(slot, F.y, 3)) return a.y + (slot - F.y) * V;
  if (in_range(slot, F.w, 3)) return a.w_in + (slot - F.w) * V;
  if (in_range(slot, F.b, 3)) return a.b_in + (slot - F.b) * V;
  if (in_range(slot, F.wp, 3)) return (IN == IN_STATE ? a.wprev_in : a.wp) + (slot - F.wp) * V;
  if (in_range(slot, F.bp, 3)) return (IN == IN_STATE ? a.bprev_in : a.bp) + (slot - F.bp) * V;
  if (in_range(slot, F.J, 3)) return a.J + (slot - F.J) * V;
  return a.c;
}
#endif

// XTRA: kPlanePlain, kPlaneConv (threshold stopping), kPlaneHist (reverse-mode
// recompute: u^k history, w^{k-1} to w_tile_out)
template <int IN, bool PREV, bool STEP, int XTRA>
__global__ void __launch_bounds__(kPlaneThreads, 3) k_plane(const __grid_constant__ PlaneArgs a) {
#if defined(__CUDA_ARCH__)
  constexpr FieldMap F = field_map<IN, PREV, STEP>();
  extern __shared__ __align__(128) unsigned char smem[];
  const PlaneSmem L = plane_layout(a, F.n);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  float* fld = reinterpret_cast<float*>(smem + L.fld);
  float2* lines = reinterpret_cast<float2*>(smem + L.lines);
  // the small x-axis tables are read through L1 where they are used
  const float2* __restrict__ tw = a.twx;
  const int* __restrict__ pos = a.posx;
  const int tiles_y = a.ny / a.R;
  const int z = (int)fdiv(blockIdx.x, a.tiles_div);
  const int y0 = (blockIdx.x - z * tiles_y) * a.R;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int nlines = 3 * (a.R / 2);

  // Within an ADMM loop the k >= 1 passes (IN_SPEC) read tiles written by the
  // plane pass four kernels back, while the kernel just before them writes
  // only the spectrum: their bulk loads are issued before waiting on it.
  // Every other variant reads data of the immediately preceding kernel (the
  // gradient kernel, or the caller's own work), so it loads after the wait.
  constexpr bool CONV = (XTRA == kPlaneConv);
  // with thresholds (CONV) the pass may have to stop before loading anything
  constexpr bool kEarlyLoads = (IN == IN_SPEC) && !CONV;
  const uint32_t tile_bytes = (uint32_t)(a.R * a.nx * sizeof(float));
  const size_t tile_off = ((size_t)z * a.ny + y0) * a.nx;
  const bool spec_tma = a.spec_tma != 0;
  const int nckx = 3 * a.nkx;
  if (F.n > 0 || spec_tma) {
    if (tid == 0) {
      mbar_init(bar, 1);
      mbar_init(bar + 1, 1);
      fence_barrier_init();
    }
    __syncthreads();
  }
  if (F.n > 0) {
    if (kEarlyLoads && tid < 32) {
      if (tid == 0) mbar_expect_tx(bar, tile_bytes * F.n);
      __syncwarp();
      for (int s = tid; s < F.n; s += 32)
        bulk_load(fld + (size_t)s * a.R * a.nx, field_src<IN, PREV, STEP>(a, s) + tile_off,
                  tile_bytes, bar);
    }
  }
  pdl_wait();
  pdl_trigger();
  if (CONV) {
    // threshold stop: a new inner loop (k = 0) clears the ADMM stop; later
    // passes of a stopped loop, and every pass after the outer stop, return
    if (a.conv[kConvOuter]) return;
    if (IN == IN_SPEC && a.conv[kConvInner]) return;
    if (tid == 0 && (IN == IN_SPEC || IN == IN_NONE) && STEP) {
      if (IN == IN_NONE && blockIdx.x == 0) a.conv[kConvInner] = 0u;
      if (blockIdx.x == 0) atomicAdd(a.conv + kConvAdmmRun, 1u);
    }
  }
  if (IN == IN_SPEC && spec_tma && tid == kSpecIssuer) {
    // the CTA's spectrum block {R rows, this z, all (comp, kx)}: one box,
    // issued from warp 1 so that it does not wait behind warp 0's issue of
    // the field loads
    mbar_expect_tx(bar + 1, (uint32_t)(nckx * a.R * sizeof(float2)));
    tensor_load_3d(lines, &a.smap, y0, z, 0, bar + 1);
  }
  if (F.n > 0 && !kEarlyLoads && tid < 32) {
    if (tid == 0) mbar_expect_tx(bar, tile_bytes * F.n);
    __syncwarp();
    for (int s = tid; s < F.n; s += 32)
      bulk_load(fld + (size_t)s * a.R * a.nx, field_src<IN, PREV, STEP>(a, s) + tile_off,
                tile_bytes, bar);
  }
  if (IN == IN_SPEC) {
    if (spec_tma) {
      const bool ok = __syncthreads_and(mbar_wait_bounded(bar + 1, 0));
      if (!ok) {
        if (tid == 0 && a.status != nullptr) atomicOr(a.status, kStatusTimeout);
        mbar_wait_bounded(bar + 1, 0);  // let copies still in flight land before exit
        if (F.n > 0) mbar_wait_bounded(bar, 0);
        return;
      }
      plane_unpack(a, lines, pos, tid, nthr);
    } else {
      plane_gather(a, lines, pos, z, y0, tid, nthr);
    }
    __syncthreads();
    if (a.xr2 != 0) {
      plane_lane_fft<true>(a, lines, tw, nlines, tid);
      __syncthreads();
    } else {
      for (int s = a.px.nst - 1; s >= 0; --s) {
        fft_stage<true>(a.px, s, lines, nlines, a.lines_div, 1, a.pitch, tw, tid, nthr);
        __syncthreads();
      }
    }
  }
  if (F.n > 0) {
    const bool ok = __syncthreads_and(mbar_wait_bounded(bar, 0));
    if (!ok) {
      if (tid == 0 && a.status != nullptr) atomicOr(a.status, kStatusTimeout);
      mbar_wait_bounded(bar, 0);  // let copies still in flight land before exit
      return;
    }
  }
  constexpr bool kMeasure = CONV && PREV && STEP && IN == IN_SPEC;  // ADMM residual of this pass
  if (kMeasure && a.admm_tol > 0.0f) {
    float racc[2] = {0.0f, 0.0f};
    plane_pointwise<IN, PREV, STEP, kMeasure>(a, fld, lines, z, y0, tid, nthr, racc);
    plane_residual(a, racc);
  } else if (XTRA == kPlaneHist) {
    plane_pointwise<IN, PREV, STEP, false, STEP && IN != IN_FIELD>(a, fld, lines, z, y0, tid, nthr);
  } else {
    plane_pointwise<IN, PREV, STEP>(a, fld, lines, z, y0, tid, nthr);
  }
  // tiles rewritten in shared memory by the point-wise step (w, b, y state)
  constexpr bool kTileStores = STEP && (F.wp >= 0 || F.y >= 0);
  if (kTileStores) fence_proxy_async();  // make them visible to the bulk copies
  if (STEP) {
    __syncthreads();
    if (kTileStores && tid == 0) {
      const size_t V = (size_t)a.nx * a.ny * a.nz;
      for (int comp = 0; comp < 3; ++comp) {
        const size_t g = comp * V + tile_off;
        if (F.wp >= 0) {
          float* wdst = (XTRA == kPlaneHist && a.w_tile_out != nullptr) ? a.w_tile_out : a.wp;
          bulk_store(wdst + g, fld + (size_t)(F.wp + comp) * a.R * a.nx, tile_bytes);
          bulk_store(a.bp + g, fld + (size_t)(F.bp + comp) * a.R * a.nx, tile_bytes);
        }
        if (F.y >= 0) bulk_store(a.y + g, fld + (size_t)(F.y + comp) * a.R * a.nx, tile_bytes);
      }
      bulk_commit();
    }
    if (a.xr2 != 0) {
      plane_lane_fft<false>(a, lines, tw, nlines, tid);
      __syncthreads();
    } else {
      for (int s = 0; s < a.px.nst; ++s) {
        fft_stage<false>(a.px, s, lines, nlines, a.lines_div, 1, a.pitch, tw, tid, nthr);
        __syncthreads();
      }
    }
    if (spec_tma) {
      plane_pack(a, lines, pos, tid, nthr);
      fence_proxy_async();
      __syncthreads();
      if (tid == 0) {
        tensor_store_3d(&a.smap, y0, z, 0, lines);
        bulk_commit();
      }
    } else {
      plane_scatter(a, lines, pos, z, y0, tid, nthr);
    }
    // shared memory must stay until the bulk stores have read it
    if ((kTileStores || spec_tma) && tid == 0) bulk_wait_read();
  }
#endif
}

// ---------------------------------------------------------------- pipelined plane pass
// The k >= 2 pass of a fixed schedule as persistent CTAs (two per SM): CTA
// c handles tiles c, c + G, c + 2G, ... (G CTAs).  A second line buffer lets
// the next tile's spectrum block load while this tile is transformed, and
// the next tile's field tiles load as soon as this tile's outputs have been
// read out of the field buffer by their bulk stores.  The last thread of the
// CTA (in a warp the lane FFTs leave idle) issues and retires the copies.
// Same arithmetic as k_plane<IN_SPEC, true, true, kPlanePlain>.
constexpr int kPipeCtasPerSm = 2;

struct PipeSmem {
  size_t fld, lines0, lines1, total;
};

NADMM_HD PipeSmem pipe_layout(const PlaneArgs& a, int nfields) {
  PipeSmem L;
  L.fld = 128;  // three mbarriers before it
  size_t o = L.fld + (size_t)nfields * a.R * a.nx * sizeof(float);
  const size_t lines = (((size_t)3 * (a.R / 2) * a.pitch * sizeof(float2)) + 127) & ~(size_t)127;
  L.lines0 = (o + 127) & ~(size_t)127;
  L.lines1 = L.lines0 + lines;
  L.total = L.lines1 + lines;
  return L;
}

__global__ void __launch_bounds__(kPlaneThreads, kPipeCtasPerSm)
    k_plane_pipe(const __grid_constant__ PlaneArgs a) {
#if defined(__CUDA_ARCH__)
  constexpr int IN = IN_SPEC;
  constexpr bool PREV = true, STEP = true;
  constexpr FieldMap F = field_map<IN, PREV, STEP>();
  extern __shared__ __align__(128) unsigned char smem[];
  const PipeSmem L = pipe_layout(a, F.n);
  uint64_t* fbar = reinterpret_cast<uint64_t*>(smem);  // field tiles
  uint64_t* sbar = fbar + 1;                            // spectrum blocks, per line buffer
  float* fld = reinterpret_cast<float*>(smem + L.fld);
  float2* const lbuf[2] = {reinterpret_cast<float2*>(smem + L.lines0),
                           reinterpret_cast<float2*>(smem + L.lines1)};
  const float2* __restrict__ tw = a.twx;
  const int* __restrict__ pos = a.posx;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int X = nthr - 1;  // copy thread
  const int nlines = 3 * (a.R / 2);
  const int tiles_y = a.ny / a.R;
  const int ntiles = tiles_y * a.nz;
  const int G = gridDim.x;
  const int mine = (ntiles - (int)blockIdx.x + G - 1) / G;  // tiles of this CTA
  const uint32_t tile_bytes = (uint32_t)(a.R * a.nx * sizeof(float));
  const uint32_t spec_bytes = (uint32_t)(3 * a.nkx * a.R * sizeof(float2));
  const size_t V = (size_t)a.nx * a.ny * a.nz;
  auto tile_zy = [&](int i, int& z, int& y0) {
    const int t = (int)blockIdx.x + i * G;
    z = (int)fdiv((uint32_t)t, a.tiles_div);
    y0 = (t - z * tiles_y) * a.R;
  };
  auto load_fields = [&](int i) {  // thread X
    int z, y0;
    tile_zy(i, z, y0);
    const size_t off = ((size_t)z * a.ny + y0) * a.nx;
    mbar_expect_tx(fbar, tile_bytes * F.n);
    for (int sl = 0; sl < F.n; ++sl)
      bulk_load(fld + (size_t)sl * a.R * a.nx, field_src<IN, PREV, STEP>(a, sl) + off, tile_bytes,
                fbar);
  };
  auto load_spec = [&](int i) {  // thread X
    int z, y0;
    tile_zy(i, z, y0);
    mbar_expect_tx(sbar + (i & 1), spec_bytes);
    tensor_load_3d(lbuf[i & 1], &a.smap, y0, z, 0, sbar + (i & 1));
  };
  if (tid == 0) {
    mbar_init(fbar, 1);
    mbar_init(sbar, 1);
    mbar_init(sbar + 1, 1);
    fence_barrier_init();
  }
  __syncthreads();
  int f_issued = 0, s_issued[2] = {0, 0};  // loads issued per barrier (thread X's view)
  if (tid == X && mine > 0) {  // fields of the first tile: written four kernels back
    load_fields(0);
    f_issued = 1;
  }
  pdl_wait();
  pdl_trigger();
  if (tid == X && mine > 0) {
    load_spec(0);
    s_issued[0] = 1;
  }
  bool failed = false;
  int i = 0;
  for (; i < mine; ++i) {
    const int b = i & 1;
    float2* lines = lbuf[b];
    int z, y0;
    tile_zy(i, z, y0);
    const size_t tile_off = ((size_t)z * a.ny + y0) * a.nx;
    if (!__syncthreads_and(mbar_wait_bounded(sbar + b, (uint32_t)((i >> 1) & 1)))) {
      failed = true;
      break;
    }
    plane_unpack(a, lines, pos, tid, nthr);
    __syncthreads();
    if (tid == X && i + 1 < mine) {
      // the other line buffer is free once the previous tile's spectrum
      // store has read it: prefetch the next tile's block there
      bulk_wait_read();
      load_spec(i + 1);
      s_issued[(i + 1) & 1] += 1;
    }
    if (a.xr2 != 0) {
      plane_lane_fft<true>(a, lines, tw, nlines, tid);
    } else {
      for (int s = a.px.nst - 1; s >= 0; --s) {
        fft_stage<true>(a.px, s, lines, nlines, a.lines_div, 1, a.pitch, tw, tid, nthr);
        __syncthreads();
      }
    }
    if (!__syncthreads_and(mbar_wait_bounded(fbar, (uint32_t)(i & 1)))) {
      failed = true;
      break;
    }
    plane_pointwise<IN, PREV, STEP>(a, fld, lines, z, y0, tid, nthr);
    fence_proxy_async();
    __syncthreads();
    if (tid == X) {
      for (int comp = 0; comp < 3; ++comp) {
        const size_t g = comp * V + tile_off;
        bulk_store(a.wp + g, fld + (size_t)(F.wp + comp) * a.R * a.nx, tile_bytes);
        bulk_store(a.bp + g, fld + (size_t)(F.bp + comp) * a.R * a.nx, tile_bytes);
        bulk_store(a.y + g, fld + (size_t)(F.y + comp) * a.R * a.nx, tile_bytes);
      }
      bulk_commit();
      if (i + 1 < mine) {  // the field buffer is free once the stores have read it
        bulk_wait_read();
        load_fields(i + 1);
        f_issued += 1;
      }
    }
    if (a.xr2 != 0) {
      plane_lane_fft<false>(a, lines, tw, nlines, tid);
      __syncthreads();
    } else {
      for (int s = 0; s < a.px.nst; ++s) {
        fft_stage<false>(a.px, s, lines, nlines, a.lines_div, 1, a.pitch, tw, tid, nthr);
        __syncthreads();
      }
    }
    plane_pack(a, lines, pos, tid, nthr);
    fence_proxy_async();
    __syncthreads();
    if (tid == X) {
      tensor_store_3d(&a.smap, y0, z, 0, lines);
      bulk_commit();
    }
  }
  if (tid == X) {
    if (failed) {
      if (a.status != nullptr) atomicOr(a.status, kStatusTimeout);
      // let every copy still in flight land before the CTA leaves: the
      // barrier phases not yet waited for, from the issued counts
      const int f_done = i;                       // tiles whose fields were consumed
      if (f_issued > f_done) mbar_wait_bounded(fbar, (uint32_t)(f_done & 1));
      for (int bb = 0; bb < 2; ++bb) {
        const int s_done = (i + 1 - bb) / 2;      // uses of buffer bb consumed before tile i
        if (s_issued[bb] > s_done) mbar_wait_bounded(sbar + bb, (uint32_t)(s_done & 1));
      }
    }
    bulk_wait_read();  // shared memory must stay until the last stores have read it
  }
#endif
}

// ---------------------------------------------------------------- y / z passes
// The pencil work of Eq. 6's 3D DFT on the half spectrum [3][nkx][nz][ny]:
//   y-pass  (forward, then inverse after the z-pass): y-DFT of `yrows`
//           consecutive (component, kx, z) rows per CTA;
//   z-pass: for a (component, kx) plane and `zcols` consecutive y positions,
//           forward z-DFT, multiply by 1/(1 + gamma K^n)/(nx ny nz), inverse
//           z-DFT (last forward stage, filter and first inverse stage fused).
// The spectrum stays L2-resident between them; each CTA is small, so the
// grid covers every SM several times whatever the grid size.

// Gain 1/(1 + gamma K^n)/(nx ny nz) for y position `line` of the tile and
// z position `zpos` (Ky holds the tile's slice, Kz the whole axis).
struct PencilFilter {
  const float* Ky;
  const float* Kz;
  float kx_term, gamma, scale;
  int order;
  NADMM_HD float operator()(int line, int zpos) const {
    const float K = kx_term + Ky[line] + Kz[zpos];
    float Kn = K;
    for (int i = 1; i < order; ++i) Kn *= K;
#if defined(__CUDA_ARCH__)
    return __fdividef(scale, 1.0f + gamma * Kn);
#else
    return scale / (1.0f + gamma * Kn);
#endif
  }
};

constexpr int kYThreads = 128;
constexpr int kZThreads = 128;

NADMM_HD size_t ypass_smem(const PencilArgs& a) {
  return 16 + (size_t)a.yrows * a.ypitch * sizeof(float2) + (size_t)a.py.tw_count * sizeof(float2);
}

NADMM_HD size_t zpass_smem(const PencilArgs& a) {
  return 16 + 128 + (size_t)a.nz * a.zcols * sizeof(float2) + (size_t)a.pz.tw_count * sizeof(float2) +
         (size_t)(a.nz + a.zcols) * sizeof(float) + 16;
}

// y-DFT (forward or inverse) of `nrows` rows held at `rows` with pitch ypitch.
template <bool INV>
NADMM_HD void ypass_transform(const PencilArgs& a, float2* rows, const float2* tw, int tid,
                              int nthr, bool sync_between) {
#if defined(__CUDA_ARCH__)
#define NADMM_PSYNC() \
  if (sync_between) __syncthreads()
#else
#define NADMM_PSYNC() (void)sync_between
#endif
  if (!INV) {
    for (int s = 0; s < a.py.nst; ++s) {
      fft_stage<false>(a.py, s, rows, a.yrows, a.yrows_div, 1, a.ypitch, tw, tid, nthr);
      NADMM_PSYNC();
    }
  } else {
    for (int s = a.py.nst - 1; s >= 0; --s) {
      fft_stage<true>(a.py, s, rows, a.yrows, a.yrows_div, 1, a.ypitch, tw, tid, nthr);
      NADMM_PSYNC();
    }
  }
#undef NADMM_PSYNC
}

// z-DFT, filter, inverse z-DFT of a [nz][zcols] tile (lines = y positions).
NADMM_HD void zpass_transform(const PencilArgs& a, float2* tile, const float2* tw,
                              const PencilFilter& filt, int tid, int nthr, bool sync_between) {
#if defined(__CUDA_ARCH__)
#define NADMM_PSYNC() \
  if (sync_between) __syncthreads()
#else
#define NADMM_PSYNC() (void)sync_between
#endif
  if (a.pz.root_off[a.pz.nst - 1] >= 0) {
    // last stage generic (nz a product of primes > 7): transform, filter and
    // transform back as separate steps
    for (int s = 0; s < a.pz.nst; ++s) {
      fft_stage<false>(a.pz, s, tile, a.zcols, a.zcols_div, a.zcols, 1, tw, tid, nthr);
      NADMM_PSYNC();
    }
    for (int g = tid; g < a.nz * a.zcols; g += nthr) {
      const int zpos = (int)fdiv((uint32_t)g, a.zcols_div), line = g - zpos * a.zcols;
      tile[g] = cscale(tile[g], filt(line, zpos));
    }
    NADMM_PSYNC();
    for (int s = a.pz.nst - 1; s >= 0; --s) {
      fft_stage<true>(a.pz, s, tile, a.zcols, a.zcols_div, a.zcols, 1, tw, tid, nthr);
      NADMM_PSYNC();
    }
    return;
  }
  for (int s = 0; s + 1 < a.pz.nst; ++s) {
    fft_stage<false>(a.pz, s, tile, a.zcols, a.zcols_div, a.zcols, 1, tw, tid, nthr);
    NADMM_PSYNC();
  }
  fft_filter_last(a.pz, tile, a.zcols, a.zcols_div, a.zcols, 1, filt, tid, nthr);
  NADMM_PSYNC();
  for (int s = a.pz.nst - 2; s >= 0; --s) {
    fft_stage<true>(a.pz, s, tile, a.zcols, a.zcols_div, a.zcols, 1, tw, tid, nthr);
    NADMM_PSYNC();
  }
#undef NADMM_PSYNC
}

template <bool INV>
__global__ void __launch_bounds__(kYThreads) k_ypass(PencilArgs a) {
#if defined(__CUDA_ARCH__)
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  float2* rows = reinterpret_cast<float2*>(smem + 16);
  float2* tw = rows + (size_t)a.yrows * a.ypitch;
  const int tid = threadIdx.x, nthr = blockDim.x;
  float2* g = a.spec + (size_t)blockIdx.x * a.yrows * a.ny;
  const uint32_t row_bytes = (uint32_t)(a.ny * sizeof(float2));
  for (int i = tid; i < a.py.tw_count; i += nthr) tw[i] = a.twy[i];
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  pdl_wait();  // the spectrum comes from the previous kernel
  if (a.conv != nullptr && (a.conv[kConvInner] | a.conv[kConvOuter])) return;  // threshold stop
  if (tid < 32) {
    if (tid == 0) mbar_expect_tx(bar, row_bytes * a.yrows);
    __syncwarp();
    for (int r = tid; r < a.yrows; r += 32)
      bulk_load(rows + (size_t)r * a.ypitch, g + (size_t)r * a.ny, row_bytes, bar);
  }
  pdl_trigger();
  const bool ok = __syncthreads_and(mbar_wait_bounded(bar, 0));
  if (!ok) {
    if (tid == 0 && a.status != nullptr) atomicOr(a.status, kStatusTimeout);
    mbar_wait_bounded(bar, 0);
    return;
  }
  ypass_transform<INV>(a, rows, tw, tid, nthr, true);
  fence_proxy_async();
  __syncthreads();
  if (tid < 32) {
    for (int r = tid; r < a.yrows; r += 32)
      bulk_store(g + (size_t)r * a.ny, rows + (size_t)r * a.ypitch, row_bytes);
    bulk_commit();
    bulk_wait_read();
  }
#endif
}

__global__ void __launch_bounds__(kZThreads) k_zpass(const __grid_constant__ PencilArgs a) {
#if defined(__CUDA_ARCH__)
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  // TMA box destination: round up to 128 bytes (the layout reserves the slack)
  unsigned char* tile_p = smem + 16;
  tile_p += (128u - (smem_addr(tile_p) & 127u)) & 127u;
  float2* tile = reinterpret_cast<float2*>(tile_p);
  float2* tw = tile + (size_t)a.nz * a.zcols;
  float* Kz = reinterpret_cast<float*>(tw + a.pz.tw_count);
  float* Ky = Kz + a.nz;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int tiles = a.ny / a.zcols;
  const int plane = (int)fdiv(blockIdx.x, a.ztiles_div);
  const int y0 = (blockIdx.x - plane * tiles) * a.zcols;
  const int kx = plane - (int)fdiv((uint32_t)plane, a.nkx_div) * a.nkx;
  const int row0 = plane * a.nz;  // first row of this plane in the 2D view
  for (int i = tid; i < a.pz.tw_count; i += nthr) tw[i] = a.twz[i];
  for (int i = tid; i < a.nz; i += nthr) Kz[i] = a.Kz[i];
  for (int i = tid; i < a.zcols; i += nthr) Ky[i] = a.Ky[y0 + i];
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  pdl_wait();
  if (a.conv != nullptr && (a.conv[kConvInner] | a.conv[kConvOuter])) return;  // threshold stop
  if (tid == 0) {
    mbar_expect_tx(bar, (uint32_t)(a.nz * a.zcols * sizeof(float2)));
    tensor_load_2d(tile, &a.zmap, y0, row0, bar);
  }
  pdl_trigger();
  const bool ok = __syncthreads_and(mbar_wait_bounded(bar, 0));
  if (!ok) {
    if (tid == 0 && a.status != nullptr) atomicOr(a.status, kStatusTimeout);
    mbar_wait_bounded(bar, 0);
    return;
  }
  // Kx by the natural frequency kx < nkx (the x-transform is scattered in
  // natural order); Ky and Kz by position.
  const PencilFilter filt{Ky, Kz, a.Kx[kx], a.gamma, a.scale, a.order_n};
  zpass_transform(a, tile, tw, filt, tid, nthr, true);
  fence_proxy_async();
  __syncthreads();
  if (tid == 0) {
    tensor_store_2d(&a.zmap, y0, row0, tile);
    bulk_commit();
    bulk_wait_read();
  }
#endif
}

// ---------------------------------------------------------------- launchers
int rows_per_tile(int ny) { return (ny % 8 == 0) ? 8 : (ny % 4 == 0) ? 4 : 2; }

void finish_plane_args(PlaneArgs& a) {
  a.nkx = a.nx / 2 + 1;
  a.R = rows_per_tile(a.ny);
  const AxisPlan& p = a.px;
  const bool lane = p.nst == 2 && p.m[1] == 1 && lane_pair_supported(p.radix[0], p.radix[1]) &&
                    3 * (a.R / 2) * p.radix[1] <= kPlaneThreads;
  if (lane) {
    a.xr1 = p.radix[0];
    a.xr2 = p.radix[1];
    a.xlog2r2 = (a.xr2 == 8) ? 3 : 4;
    a.pitch = a.nx + 8;  // even; two 8-lane groups of a half-warp on different banks
  } else {
    a.xr1 = a.xr2 = 0;
    a.xlog2r2 = -1;
    a.pitch = a.nx + 3;  // odd: lanes on different lines hit different banks
  }
  // The spectrum block (3 nkx R values) fits the line buffer (3 R/2 lines of
  // pitch >= nx + 2 = 2 nkx) and moves by one tensor copy when the box spans
  // all (comp, kx) (3 nkx <= 256, i.e. nx <= 168) and each thread holds at
  // most kGatherItems (comp, kx, row) items in the in-place (un)pack.
  a.spec_tma = (3 * a.nkx <= 256 && 3 * a.nkx * (a.R / 2) <= kGatherItems * kPlaneThreads) ? 1 : 0;
  a.pipe = 0;  // opt-in: the persistent pass measured slower than one CTA per tile
  a.nx_div = make_fastdiv((uint32_t)a.nx);
  a.lines_div = make_fastdiv((uint32_t)(3 * (a.R / 2)));
  a.half_div = make_fastdiv((uint32_t)(a.R / 2));
  a.nkx_div = make_fastdiv((uint32_t)a.nkx);
  a.tiles_div = make_fastdiv((uint32_t)(a.ny / a.R));
}

void finish_pencil_args(PencilArgs& a) {
  a.yrows = (a.nz % 16 == 0) ? 16 : (a.nz % 8 == 0) ? 8 : (a.nz % 4 == 0) ? 4 : (a.nz % 2 == 0) ? 2 : 1;
  a.ypitch = a.ny + 2;  // even: row starts stay 16-byte aligned for bulk copies
  a.zcols = (a.ny % 16 == 0) ? 16 : (a.ny % 8 == 0) ? 8 : (a.ny % 4 == 0) ? 4 : 2;
  a.yrows_div = make_fastdiv((uint32_t)a.yrows);
  a.zcols_div = make_fastdiv((uint32_t)a.zcols);
  a.ztiles_div = make_fastdiv((uint32_t)(a.ny / a.zcols));
  a.nkx_div = make_fastdiv((uint32_t)a.nkx);
  a.fused = 0;  // the caller opts in (NADMM_FLAG_FUSED_PENCIL) where fused_pencil_supported
}

cudaError_t encode_pencil_map(PencilArgs& a) {
  using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeFn encode = nullptr;
  if (encode == nullptr) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || fn == nullptr) return cudaErrorSymbolNotFound;
    encode = reinterpret_cast<EncodeFn>(fn);
  }
  // complex64 values as 8-byte elements: dims {ny, 3 nkx nz}, row stride ny * 8 bytes
  const cuuint64_t dims[2] = {(cuuint64_t)a.ny, (cuuint64_t)3 * a.nkx * a.nz};
  const cuuint64_t strides[1] = {(cuuint64_t)a.ny * sizeof(float2)};
  const cuuint32_t box[2] = {(cuuint32_t)a.zcols, (cuuint32_t)a.nz};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(&a.zmap, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, a.spec, dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t encode_plane_map(PlaneArgs& a) {
  using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeFn encode = nullptr;
  if (encode == nullptr) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || fn == nullptr) return cudaErrorSymbolNotFound;
    encode = reinterpret_cast<EncodeFn>(fn);
  }
  // complex64 values as 8-byte elements: dims {ny, nz, 3 nkx}; box {R, 1, <= 256}
  const int nckx = 3 * a.nkx;
  const cuuint64_t dims[3] = {(cuuint64_t)a.ny, (cuuint64_t)a.nz, (cuuint64_t)nckx};
  const cuuint64_t strides[2] = {(cuuint64_t)a.ny * sizeof(float2),
                                 (cuuint64_t)a.ny * a.nz * sizeof(float2)};
  if (nckx > 256) return cudaErrorInvalidValue;  // one box must span every (comp, kx)
  const cuuint32_t box[3] = {(cuuint32_t)a.R, 1u, (cuuint32_t)nckx};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encode(&a.smap, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, a.spec, dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

static int field_count(int in_mode, bool prev, bool step) {
  switch (in_mode * 4 + (prev ? 2 : 0) + (step ? 1 : 0)) {
    case IN_NONE * 4 + 1: return field_map<IN_NONE, false, true>().n;
    case IN_SPEC * 4 + 1: return field_map<IN_SPEC, false, true>().n;
    case IN_SPEC * 4 + 3: return field_map<IN_SPEC, true, true>().n;
    case IN_SPEC * 4 + 0: return field_map<IN_SPEC, false, false>().n;
    case IN_STATE * 4 + 1: return field_map<IN_STATE, false, true>().n;
    case IN_STATE * 4 + 3: return field_map<IN_STATE, true, true>().n;
    case IN_FIELD * 4 + 1: return field_map<IN_FIELD, false, true>().n;
  }
  return 0;
}

size_t plane_smem_bytes(const PlaneArgs& a, int in_mode, bool prev, bool step) {
  return plane_layout(a, field_count(in_mode, prev, step)).total;
}

size_t plane_smem_max(const PlaneArgs& a) {
  const size_t p = a.spec_tma ? pipe_layout(a, 16).total : 0, q = plane_layout(a, 16).total;
  return p > q ? p : q;
}

size_t pencil_smem_bytes(const PencilArgs& a) {
  const size_t y = ypass_smem(a), z = zpass_smem(a);
  return y > z ? y : z;
}

// Dynamic shared-memory limit of a kernel: the request, capped so that the
// kernel's static shared memory still fits the opt-in maximum per block.
template <typename K>
static cudaError_t set_smem_limit(K kernel, size_t smem) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  int dev = 0, optin = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
    return e;
  const size_t cap = (size_t)optin - fa.sharedSizeBytes;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(smem < cap ? smem : cap));
}

template <int IN, bool PREV, bool STEP>
static cudaError_t set_plane_attr(size_t smem) {
  cudaError_t e = set_smem_limit(k_plane<IN, PREV, STEP, kPlanePlain>, smem);
  if (e == cudaSuccess) e = set_smem_limit(k_plane<IN, PREV, STEP, kPlaneConv>, smem);
  return e != cudaSuccess ? e : set_smem_limit(k_plane<IN, PREV, STEP, kPlaneHist>, smem);
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
  if ((e = set_smem_limit(k_plane_pipe, plane_smem)) != cudaSuccess) return e;
  if ((e = set_smem_limit(k_ypass<false>, pencil_smem)) != cudaSuccess) return e;
  if ((e = set_smem_limit(k_ypass<true>, pencil_smem)) != cudaSuccess) return e;
  if ((e = configure_fused_pencil()) != cudaSuccess) return e;
  if ((e = configure_slab_kernels()) != cudaSuccess) return e;
  return set_smem_limit(k_zpass, pencil_smem);
}

// cudaFuncSetAttribute applies to the device that is current when it is
// called (each device holds its own copy of the module), so the limits are
// raised once per device ordinal, the first time a handle or a no-alloc call
// runs there.
cudaError_t configure_admm_kernels_on_current_device() {
  constexpr int kMaxDev = 64;
  static std::mutex mu;
  static bool done[kMaxDev] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return cudaSuccess;
  constexpr size_t kOptinMax = 227 * 1024;
  e = configure_admm_kernels(kOptinMax, kOptinMax);
  if (e == cudaSuccess) done[dev] = true;
  return e;
}

template <int CONV>
static cudaError_t launch_plane_t(int in_mode, bool prev, bool step, const PlaneArgs& a,
                                  cudaStream_t s) {
  dim3 grid((unsigned)((a.ny / a.R) * a.nz));
  dim3 block(kPlaneThreads);
  const size_t smem = plane_smem_bytes(a, in_mode, prev, step);
  switch (in_mode * 4 + (prev ? 2 : 0) + (step ? 1 : 0)) {
    case IN_NONE * 4 + 1: return launch_pdl(k_plane<IN_NONE, false, true, CONV>, grid, block, smem, s, a);
    case IN_SPEC * 4 + 1: return launch_pdl(k_plane<IN_SPEC, false, true, CONV>, grid, block, smem, s, a);
    case IN_SPEC * 4 + 3:
      if (CONV == kPlanePlain && a.pipe && a.spec_tma) {  // persistent, pipelined
        int dev = 0, sms = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        const int ntiles = (a.ny / a.R) * a.nz;
        const int G = ntiles < kPipeCtasPerSm * sms ? ntiles : kPipeCtasPerSm * sms;
        return launch_pdl(k_plane_pipe, dim3((unsigned)G), block,
                          pipe_layout(a, field_map<IN_SPEC, true, true>().n).total, s, a);
      }
      return launch_pdl(k_plane<IN_SPEC, true, true, CONV>, grid, block, smem, s, a);
    case IN_SPEC * 4 + 0: return launch_pdl(k_plane<IN_SPEC, false, false, CONV>, grid, block, smem, s, a);
    case IN_STATE * 4 + 1: return launch_pdl(k_plane<IN_STATE, false, true, CONV>, grid, block, smem, s, a);
    case IN_STATE * 4 + 3: return launch_pdl(k_plane<IN_STATE, true, true, CONV>, grid, block, smem, s, a);
    case IN_FIELD * 4 + 1: return launch_pdl(k_plane<IN_FIELD, false, true, CONV>, grid, block, smem, s, a);
  }
  return cudaErrorInvalidValue;
}

// Fixed schedules use the kernels without the threshold or history code.
cudaError_t launch_plane(int in_mode, bool prev, bool step, const PlaneArgs& a, cudaStream_t s) {
  if (a.conv != nullptr) return launch_plane_t<kPlaneConv>(in_mode, prev, step, a, s);
  if (a.u_hist != nullptr) return launch_plane_t<kPlaneHist>(in_mode, prev, step, a, s);
  return launch_plane_t<kPlanePlain>(in_mode, prev, step, a, s);
}

cudaError_t launch_pencil(const PencilArgs& a, cudaStream_t s) {
  if (a.fused) return launch_fused_pencil(a, s);
  const unsigned yblocks = (unsigned)(3 * a.nkx * a.nz / a.yrows);
  const unsigned zblocks = (unsigned)(3 * a.nkx * (a.ny / a.zcols));
  const bool ly = lane_y_supported(a), lz = lane_z_supported(a);
  cudaError_t e = ly ? launch_lane_y(a, false, s)
                     : launch_pdl(k_ypass<false>, dim3(yblocks), dim3(kYThreads), ypass_smem(a), s, a);
  if (e == cudaSuccess)
    e = lz ? launch_lane_z(a, s)
           : launch_pdl(k_zpass, dim3(zblocks), dim3(kZThreads), zpass_smem(a), s, a);
  if (e == cudaSuccess)
    e = ly ? launch_lane_y(a, true, s)
           : launch_pdl(k_ypass<true>, dim3(yblocks), dim3(kYThreads), ypass_smem(a), s, a);
  return e;
}

}  // namespace nadmm
