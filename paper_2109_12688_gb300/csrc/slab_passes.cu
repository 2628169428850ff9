// The ADMM iteration of Eq. 5 in two kernels ("slab path").
//
// The w-step (Eq. 5 line 2, Eq. 6 last line) is a 3D real DFT, a division
// by 1 + (lambda/theta) K^n in the spectrum and the inverse DFT.  Here the
// half spectrum lives as [z][component][y][kx] and one iteration is
//
//   slab pass  (one cluster of three CTAs per z-plane; CTA c holds the whole
//              ny x (nx/2+1) half-spectrum plane of component c in shared
//              memory):
//     A  inverse y-DFT of the plane's columns, inverse x-DFT of its rows
//        (real output, in place) -> w^{k-1} of component c;
//     B  point-wise: b^{k-1} = y^{k-1} - w^{k-1} (Eq. 5 line 3), the
//        Nesterov extrapolation (lines 4-6), the closed-form v-step (Eq. 6,
//        s = 1 / 2) and y^k = v^k + b_hat^k.  The v-step couples the three
//        components at each voxel, so CTA r of the cluster takes a third of
//        the plane's voxels for all three components and reads / writes the
//        other CTAs' planes through distributed shared memory;
//     C  forward x-DFT of the rows, forward y-DFT of the columns, store;
//   z-pass: forward z-DFT, multiply by 1/(1 + gamma K^n)/(nx ny nz), inverse
//     z-DFT, per (component, y, kx) column.
//
// Real x-DFTs of length nx use one complex DFT of length nx/2 per row: the
// even and odd samples form z[m] = x[2m] + i x[2m+1]; the forward spectrum
// is X_k = E_k + e^{-2 pi i k/nx} O_k with E_k = (Z_k + conj Z_{M-k})/2,
// O_k = (Z_k - conj Z_{M-k})/(2i); the inverse forms Z_k = (X_k + conj
// X_{M-k}) + i e^{+2 pi i k/nx} (X_k - conj X_{M-k}) and transforms back
// (M = nx/2, unnormalised both ways).  Each row is held by a group of 8
// lanes (lane FFT [xr1, 8]); the row's nx reals occupy nx/2 of its nx/2+1
// complex slots, starting at slot (y & 1) so that every real row starts on a
// 16-byte boundary (nx/2 + 1 is odd).
//
// Every wait on a bulk copy is bounded; on expiry a CTA records the status
// bit and still takes part in both cluster barriers, so no peer waits on it.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "fft_device.cuh"
#include "lane_fft.cuh"
#include "nadmm_internal.h"
#include "plan.h"
#include "tma.cuh"
#include "vstep.cuh"

namespace cg = cooperative_groups;

namespace nadmm {

constexpr int kSlabThreads = 256;
constexpr int kSlabWarps = kSlabThreads / 32;
constexpr int kSlabPad = 8;       // padding of an exchange line (float2)
constexpr int kSlabXR2 = 8;       // lanes per row of the x-DFT

// Exchange space of one warp (float2): 32/xr2 rows or 32/yr2 columns.
NADMM_HD size_t slab_xch_per_warp(const SlabArgs& a) {
  const size_t x = (size_t)(32 / kSlabXR2) * (a.mx + kSlabPad);
  const size_t y = (size_t)(32 / a.yr2) * (a.ny + kSlabPad);
  return x > y ? x : y;
}

// [mbarrier, 16 B][plane: ny nkx float2][exchange: kSlabWarps warps]
size_t slab_smem_bytes(const SlabArgs& a) {
  return 16 + (size_t)a.ny * a.nkx * sizeof(float2) +
         (size_t)kSlabWarps * slab_xch_per_warp(a) * sizeof(float2);
}

#if defined(__CUDA_ARCH__)
// ---------------------------------------------------------------- x-DFT of rows
// The x plan is [R1, R2] of M = nx/2 (R2 = 8): frequency k sits at position
// (k mod R1) R2 + k / R1 after the forward transform, position p holds
// frequency (p mod R2) R1 + p / R2.  Lane l's twiddles and the factors
// e^{-2 pi i k / nx} of its pre- and post-processing are loop-invariant and
// held in registers for all rows.
template <int R1, int R2>
struct RowLane {
  float2 tw[R1 - 1];
  float2 rt_post[R1 + 1];  // e^{-2 pi i k / nx}, k = l + R2 j (j <= R1; k <= M)
  float2 rt_pre[R1 > R2 ? 2 * R2 : R2];  // e^{-2 pi i k / nx}, k = b + R1 j of lane l's blocks
};

template <int R1, int R2>
__device__ __forceinline__ int row_pos(int k) {
  return (k % R1) * R2 + k / R1;
}

template <int R1, int R2>
__device__ __forceinline__ void row_inverse(float2* row, float2* buf, int l, unsigned gmask, int y,
                                            const RowLane<R1, R2>& L) {
  constexpr int M = R1 * R2;
  int blk = 0;
  for (int b = l; b < R1; b += R2, ++blk) {
    float2 w[R2];
#pragma unroll
    for (int j = 0; j < R2; ++j) {
      const int k = b + R1 * j;  // frequency held at position b R2 + j
      const float2 xa = row[k], xb = row[M - k];
      const float2 A = make_float2(xa.x + xb.x, xa.y - xb.y);  // X_k + conj X_{M-k}
      const float2 D = make_float2(xa.x - xb.x, xa.y + xb.y);  // X_k - conj X_{M-k}
      const float2 B = cmulc(D, L.rt_pre[blk * R2 + j]);       // D e^{+2 pi i k / nx}
      w[j] = make_float2(A.x - B.y, A.y + B.x);                // A + i B
    }
    dft<R2, true>(w);
#pragma unroll
    for (int j = 0; j < R2; ++j) buf[swz<R2>(b * R2 + j)] = w[j];
  }
  __syncwarp(gmask);
  float2 v[R1];
#pragma unroll
  for (int k = 0; k < R1; ++k) v[k] = buf[swz<R2>(l + R2 * k)];
  lane_stage1_reg<R1, R2, true>(v, L.tw);
  float2* re = row + (y & 1);
#pragma unroll
  for (int j = 0; j < R1; ++j) re[l + R2 * j] = v[j];
  __syncwarp(gmask);
}

template <int R1, int R2>
__device__ __forceinline__ void row_forward(float2* row, float2* buf, int l, unsigned gmask, int y,
                                            const RowLane<R1, R2>& L) {
  constexpr int M = R1 * R2;
  const float2* re = row + (y & 1);
  float2 v[R1];
#pragma unroll
  for (int j = 0; j < R1; ++j) v[j] = re[l + R2 * j];
  lane_stage1_reg<R1, R2, false>(v, L.tw);
#pragma unroll
  for (int k = 0; k < R1; ++k) buf[swz<R2>(l + R2 * k)] = v[k];
  __syncwarp(gmask);
  lane_stage2<R1, R2, false>(buf, l);
  __syncwarp(gmask);
#pragma unroll
  for (int j = 0; j <= R1; ++j) {
    const int k = l + R2 * j;
    if (k <= M) {
      const int k1 = (k == M) ? 0 : k;
      const int k2 = (k == 0 || k == M) ? 0 : M - k;
      const float2 zk = buf[swz<R2>(row_pos<R1, R2>(k1))];
      const float2 zm = buf[swz<R2>(row_pos<R1, R2>(k2))];
      const float2 E = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
      const float2 O = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
      row[k] = cadd(E, cmul(O, L.rt_post[j]));
    }
  }
  __syncwarp(gmask);
}

// All rows of the plane, groups of R2 lanes per row.
template <int R1, int R2>
__device__ __noinline__ void slab_rows(const SlabArgs& a, float2* plane, float2* xch, bool inv) {
  constexpr int M = R1 * R2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int G = 32 / R2;
  const int g = lane / R2, l = lane % R2;
  const unsigned gmask = ((1u << R2) - 1u) << (g * R2);
  float2* buf = xch + (size_t)warp * slab_xch_per_warp(a) + (size_t)g * (a.mx + kSlabPad);
  RowLane<R1, R2> L;
  lane_twiddles<R1, R2>(a.twx, l, L.tw);
#pragma unroll
  for (int j = 0; j <= R1; ++j) {
    const int k = l + R2 * j;
    L.rt_post[j] = __ldg(a.rtx + (k <= M ? k : 0));
  }
  {
    int blk = 0;
    for (int b = l; b < R1; b += R2, ++blk) {
#pragma unroll
      for (int j = 0; j < R2; ++j) L.rt_pre[blk * R2 + j] = __ldg(a.rtx + b + R1 * j);
    }
  }
  const int ny16 = a.ny & ~15;
  for (int y0 = warp * G; y0 < a.ny; y0 += kSlabWarps * G) {
    // Row r = y0 + g is transformed at y: within each block of 16 rows the two
    // groups of a half-warp take rows 8 apart, whose slots lie 8 (nx/2 + 1)
    // float2 = 16 banks (mod 32) apart (nx/2 + 1 is odd), so their accesses
    // never share a bank; adjacent rows (2 banks apart) would.
    const int r = y0 + g;
    const int y = (G == 4 && r < ny16)
                      ? (r & ~15) + ((r >> 1) & 6) + ((r & 3) >> 1) + ((r & 1) << 3)
                      : r;
    if (y < a.ny) {  // uniform over the group
      float2* row = plane + (size_t)y * a.nkx;
      if (inv)
        row_inverse<R1, R2>(row, buf, l, gmask, y, L);
      else
        row_forward<R1, R2>(row, buf, l, gmask, y, L);
    }
  }
}

// ---------------------------------------------------------------- y-DFT of columns
// Columns kx = 1 .. M-1 one by one; the columns kx = 0 and kx = M (M = nx/2)
// as one complex column Z = X_0 + i X_M.  Both hold the y-DFT of a real
// sequence (the x-DFT of real rows at frequency 0 and M is real), so
//   inverse: IDFT(X_0 + i X_M) = x_0 + i x_M with x_0, x_M real;
//   forward: Z = x_0 + i x_M, X_0[f] = (Z_f + conj Z_{-f}) / 2,
//            X_M[f] = (Z_f - conj Z_{-f}) / (2i),
// which makes M transforms of the plane's M + 1 columns.  Position p of the
// forward output holds frequency (p mod R2) R1 + p / R2; frequency f sits at
// position (f mod R1) R2 + f / R1.
template <int R1, int R2>
__device__ __forceinline__ int col_neg_pos(int p) {
  constexpr int N = R1 * R2;
  const int f = (p % R2) * R1 + p / R2;
  const int nf = f == 0 ? 0 : N - f;
  return (nf % R1) * R2 + nf / R1;
}

template <int R1, int R2>
__device__ __noinline__ void slab_cols(const SlabArgs& a, float2* plane, float2* xch, bool inv) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int G = 32 / R2;
  const int g = lane / R2, l = lane % R2;
  const unsigned gmask = (R2 == 32 ? 0xffffffffu : ((1u << R2) - 1u)) << (g * R2);
  float2* buf = xch + (size_t)warp * slab_xch_per_warp(a) + (size_t)g * (a.ny + kSlabPad);
  const int st = a.nkx;
  float2 twr[R1 - 1];
  lane_twiddles<R1, R2>(a.twy, l, twr);
  for (int c0 = warp * G; c0 < a.mx; c0 += kSlabWarps * G) {
    const int t = c0 + g;
    if (t >= a.mx) continue;  // uniform over the group
    const bool pair = (t == 0);  // columns 0 and M together
    float2* col = plane + t;
    float2* colm = plane + a.mx;
    float2 v[R1];
    if (!inv) {
#pragma unroll
      for (int j = 0; j < R1; ++j) {
        const int y = l + R2 * j;
        v[j] = pair ? make_float2(col[y * st].x, colm[y * st].x) : col[y * st];
      }
      lane_stage1_reg<R1, R2, false>(v, twr);
#pragma unroll
      for (int k = 0; k < R1; ++k) buf[swz<R2>(l + R2 * k)] = v[k];
      __syncwarp(gmask);
      lane_stage2<R1, R2, false>(buf, l);
      __syncwarp(gmask);
      if (pair) {
#pragma unroll
        for (int k = 0; k < R1; ++k) {
          const int p = l + R2 * k;
          const float2 zp = buf[swz<R2>(p)], zq = buf[swz<R2>(col_neg_pos<R1, R2>(p))];
          col[p * st] = make_float2(0.5f * (zp.x + zq.x), 0.5f * (zp.y - zq.y));
          colm[p * st] = make_float2(0.5f * (zp.y + zq.y), -0.5f * (zp.x - zq.x));
        }
      } else {
#pragma unroll
        for (int k = 0; k < R1; ++k) col[(l + R2 * k) * st] = buf[swz<R2>(l + R2 * k)];
      }
    } else {
#pragma unroll
      for (int k = 0; k < R1; ++k) {
        const int p = l + R2 * k;
        float2 z = col[p * st];
        if (pair) {  // X_0 + i X_M
          const float2 b = colm[p * st];
          z = make_float2(z.x - b.y, z.y + b.x);
        }
        buf[swz<R2>(p)] = z;
      }
      __syncwarp(gmask);
      lane_stage2<R1, R2, true>(buf, l);
      __syncwarp(gmask);
#pragma unroll
      for (int k = 0; k < R1; ++k) v[k] = buf[swz<R2>(l + R2 * k)];
      lane_stage1_reg<R1, R2, true>(v, twr);
#pragma unroll
      for (int j = 0; j < R1; ++j) {
        const int y = l + R2 * j;
        if (pair) {
          col[y * st] = make_float2(v[j].x, 0.0f);
          colm[y * st] = make_float2(v[j].y, 0.0f);
        } else {
          col[y * st] = v[j];
        }
      }
    }
    __syncwarp(gmask);
  }
}

#define NADMM_SLAB_X_CASES(X) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(12) X(14) X(16)

__device__ __forceinline__ void rows_rt(const SlabArgs& a, float2* plane, float2* xch, bool inv) {
#define X(A) \
  if (a.xr1 == A) { slab_rows<A, kSlabXR2>(a, plane, xch, inv); return; }
  NADMM_SLAB_X_CASES(X)
#undef X
}

__device__ __forceinline__ void cols_rt(const SlabArgs& a, float2* plane, float2* xch, bool inv) {
#define X(A, B) \
  if (a.yr1 == A && a.yr2 == B) { slab_cols<A, B>(a, plane, xch, inv); return; }
  NADMM_LANE_CASES(X)
#undef X
}

// ---------------------------------------------------------------- point-wise step
__device__ __forceinline__ float4 f4sub(float4 p, float4 q) {
  return make_float4(p.x - q.x, p.y - q.y, p.z - q.z, p.w - q.w);
}
__device__ __forceinline__ float4 f4extra(float4 p, float4 q, float beta) {  // p + beta (p - q)
  return make_float4(p.x + beta * (p.x - q.x), p.y + beta * (p.y - q.y), p.z + beta * (p.z - q.z),
                     p.w + beta * (p.w - q.w));
}
__device__ __forceinline__ float f4get(const float4& v, int e) {
  return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w;
}
__device__ __forceinline__ void f4set(float4& v, int e, float x) {
  if (e == 0) v.x = x; else if (e == 1) v.y = x; else if (e == 2) v.z = x; else v.w = x;
}

// Real row y of a plane (x0 a multiple of 4).
__device__ __forceinline__ float4* real_quad(float2* plane, int nkx, int y, int x0) {
  return reinterpret_cast<float4*>(reinterpret_cast<float*>(plane + (size_t)y * nkx + (y & 1)) + x0);
}

// The coupled point-wise step on voxel quads [q0, q1) of the plane at z for
// all three components (planes[c] is component c's plane, local or remote).
// RST (adaptive restart, SPEC modes): the factor comes from beta_dev[k], u^k
// is kept, and the thread's share of c_{k-1} is returned.
template <int MODE, bool RST>
__device__ __forceinline__ float slab_pointwise(const SlabArgs& a, float2* const (&planes)[3], int z,
                                                int q0, int q1, float beta_k, int k) {
  const size_t V = (size_t)a.nx * a.ny * a.nz;
  const int qrow = a.nx >> 2;
  constexpr bool kPrev = (MODE == SLAB_SPEC_PREV) || (MODE == SLAB_STATE_PREV);
  constexpr bool kState = (MODE == SLAB_STATE) || (MODE == SLAB_STATE_PREV);
  constexpr bool kSpec = (MODE == SLAB_SPEC) || (MODE == SLAB_SPEC_PREV);
  const float beta = RST ? a.beta_dev[k] : beta_k;
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  float racc = 0.0f;
  for (int q = q0 + (int)threadIdx.x; q < q1; q += kSlabThreads) {
    const int yy = (int)fdiv((uint32_t)q, a.qdiv);
    const int x0 = (q - yy * qrow) << 2;
    const size_t vox = ((size_t)z * a.ny + yy) * a.nx + x0;
    // every load of the quad is issued before the first store (the stores
    // may alias nothing the quad reads, but the compiler cannot know that)
    float4 wk1[3], yq[3], wq[3], bq[3], Jq[3], up[3];
    const float4 cq = __ldg(reinterpret_cast<const float4*>(a.c + vox));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t i = c * V + vox;
      Jq[c] = __ldg(reinterpret_cast<const float4*>(a.J + i));
      if (kSpec) {
        wk1[c] = *real_quad(planes[c], a.nkx, yy, x0);
        yq[c] = __ldcg(reinterpret_cast<const float4*>(a.y + i));
      } else if (kState) {
        wk1[c] = __ldg(reinterpret_cast<const float4*>(a.w_in + i));
        yq[c] = __ldg(reinterpret_cast<const float4*>(a.b_in + i));  // b^{k-1} itself
      } else {
        wk1[c] = yq[c] = zero4;
      }
      if (kPrev) {
        wq[c] = (MODE == SLAB_STATE_PREV) ? __ldg(reinterpret_cast<const float4*>(a.wprev_in + i))
                                          : __ldcg(reinterpret_cast<const float4*>(a.wp + i));
        bq[c] = (MODE == SLAB_STATE_PREV) ? __ldg(reinterpret_cast<const float4*>(a.bprev_in + i))
                                          : __ldcg(reinterpret_cast<const float4*>(a.bp + i));
      }
      if (RST) up[c] = (MODE == SLAB_SPEC_PREV) ? __ldcg(reinterpret_cast<const float4*>(a.u_prev + i))
                                                : zero4;
    }
    float4 bk1[3], wh[3], bh[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      bk1[c] = kSpec ? f4sub(yq[c], wk1[c]) : yq[c];
      wh[c] = kPrev ? f4extra(wk1[c], wq[c], beta) : wk1[c];
      bh[c] = kPrev ? f4extra(bk1[c], bq[c], beta) : bk1[c];
    }
    if (RST) {
      // c_{k-1}: w_hat^{k-1}, b_hat^{k-1} from u^{k-1} = w_hat - b_hat and
      // y^{k-1} = v^{k-1} + b_hat^{k-1}, v^{k-1} the v-step at u^{k-1}
      // (both zero for k = 1)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (MODE == SLAB_SPEC_PREV) {
          float Jv[3], u[3], v[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            Jv[c] = f4get(Jq[c], e);
            u[c] = f4get(up[c], e);
          }
          v_step(a.data_term, a.theta, a.eps, Jv, f4get(cq, e), u, v);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float bhat = f4get(yq[c], e) - v[c];
            const float dw = f4get(wk1[c], e) - (u[c] + bhat);
            const float db = f4get(bk1[c], e) - bhat;
            racc += dw * dw + db * db;
          }
        } else {
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float dw = f4get(wk1[c], e), db = f4get(bk1[c], e);
            racc += dw * dw + db * db;
          }
        }
      }
    }
    float4 yn[3];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float Jv[3], u[3], v[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        Jv[c] = f4get(Jq[c], e);
        u[c] = f4get(wh[c], e) - f4get(bh[c], e);
      }
      v_step(a.data_term, a.theta, a.eps, Jv, f4get(cq, e), u, v);
#pragma unroll
      for (int c = 0; c < 3; ++c) f4set(yn[c], e, v[c] + f4get(bh[c], e));
    }
    float* const wdst = a.wp_out != nullptr ? a.wp_out : a.wp;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t i = c * V + vox;
      if (MODE != SLAB_FIRST) {  // w^{k-1}, b^{k-1} into the state slots
        __stcg(reinterpret_cast<float4*>(wdst + i), wk1[c]);
        __stcg(reinterpret_cast<float4*>(a.bp + i), bk1[c]);
      }
      if (RST) __stcg(reinterpret_cast<float4*>(a.u_prev + i), f4sub(wh[c], bh[c]));
      if (a.u_hist != nullptr) __stcg(reinterpret_cast<float4*>(a.u_hist + i), f4sub(wh[c], bh[c]));
      __stcg(reinterpret_cast<float4*>(a.y + i), yn[c]);
      *real_quad(planes[c], a.nkx, yy, x0) = yn[c];
    }
  }
  return racc;
}

// Reverse step k of Eq. 5 with the s = 2 data step (the adjoint of the
// point-wise part of the iteration) on voxel quads [q0, q1) of plane z, all
// three components: the planes hold S g^k on entry and g^{k-1} (MODE
// SLAB_ADJ) on exit.  Per voxel, with rho = c + J.u^k, d = theta + |J|^2,
// y_bar = S g^k + bbar^k, q = J.y_bar / d:
//   c_bar -= q,  J_bar += -(rho/d) y_bar - q u^k + 2 rho q J / d,
//   u_bar = y_bar - J q (the adjoint of w_hat), b_hat_bar = y_bar - u_bar,
//   wbar^{k-1} += (1 + beta_k) u_bar, bbar^{k-1} += (1 + beta_k) b_hat_bar,
//   wbar^{k-2} = -beta_k u_bar, bbar^{k-2} = -beta_k b_hat_bar,
// and the thread's shares of dL/dtheta (rho J.y_bar / d^2) and dL/dgamma
// (-<g^k - S g^k, w^k> theta / lambda).
template <int MODE>
__device__ __forceinline__ void slab_adjoint(const SlabArgs& a, float2* const (&planes)[3], int z,
                                             int q0, int q1, double& p_theta, double& p_gamma) {
  const size_t V = (size_t)a.nx * a.ny * a.nz;
  const int qrow = a.nx >> 2;
  const SlabAdj& d = a.adj;
  const float beta = a.beta;
  for (int q = q0 + (int)threadIdx.x; q < q1; q += kSlabThreads) {
    const int yy = (int)fdiv((uint32_t)q, a.qdiv);
    const int x0 = (q - yy * qrow) << 2;
    const size_t vox = ((size_t)z * a.ny + yy) * a.nx + x0;
    float4 J4[3], u4[3], yb4[3];
    const float4 c4 = __ldg(reinterpret_cast<const float4*>(a.c + vox));
    double pg = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t i = c * V + vox;
      J4[c] = __ldg(reinterpret_cast<const float4*>(a.J + i));
      u4[c] = __ldg(reinterpret_cast<const float4*>(d.uk + i));
      const float4 sg = *real_quad(planes[c], a.nkx, yy, x0);
      const float4 gi = __ldcg(reinterpret_cast<const float4*>(d.g_in + i));
      const float4 wv = __ldg(reinterpret_cast<const float4*>(d.wk + i));
      const float4 bk = __ldg(reinterpret_cast<const float4*>(d.Bk + i));
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        pg += (double)(f4get(gi, e) - f4get(sg, e)) * f4get(wv, e);
        f4set(yb4[c], e, f4get(sg, e) + f4get(bk, e));
      }
    }
    p_gamma += pg;
    float qv[4], ri[4], tt[4];
    float4 gc4 = __ldcg(reinterpret_cast<const float4*>(d.gc + vox));
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float rho = f4get(c4, e), dd = a.theta, jy = 0.0f;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float Jv = f4get(J4[c], e);
        rho += Jv * f4get(u4[c], e);
        dd += Jv * Jv;
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) jy += f4get(J4[c], e) * f4get(yb4[c], e);
      const float inv_d = 1.0f / dd;
      const float qq = jy * inv_d;
      f4set(gc4, e, f4get(gc4, e) + -qq);
      p_theta += (double)rho * jy * inv_d * inv_d;
      qv[e] = qq;
      ri[e] = rho * inv_d;
      tt[e] = 2.0f * rho * qq * inv_d;
    }
    __stcg(reinterpret_cast<float4*>(d.gc + vox), gc4);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t i = c * V + vox;
      float4 gJ4 = __ldcg(reinterpret_cast<const float4*>(d.gJ + i));
      float4 ub4, bb4;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float yb = f4get(yb4[c], e), Jv = f4get(J4[c], e);
        f4set(gJ4, e, f4get(gJ4, e) + (-ri[e] * yb - qv[e] * f4get(u4[c], e) + tt[e] * Jv));
        const float ub = yb - Jv * qv[e];
        f4set(ub4, e, ub);
        f4set(bb4, e, yb - ub);
      }
      __stcg(reinterpret_cast<float4*>(d.gJ + i), gJ4);
      if (MODE == SLAB_ADJ) {
        float4 w1 = __ldcg(reinterpret_cast<const float4*>(d.W1bar + i));
        float4 b1 = __ldcg(reinterpret_cast<const float4*>(d.B1bar + i));
        float4 go;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float nw = f4get(w1, e) + (1.0f + beta) * f4get(ub4, e);
          const float nb = f4get(b1, e) + (1.0f + beta) * f4get(bb4, e);
          f4set(w1, e, nw);
          f4set(b1, e, nb);
          f4set(go, e, nw - nb);
        }
        __stcg(reinterpret_cast<float4*>(d.W1bar + i), w1);
        __stcg(reinterpret_cast<float4*>(d.B1bar + i), b1);
        __stcg(reinterpret_cast<float4*>(d.g_out + i), go);
        *real_quad(planes[c], a.nkx, yy, x0) = go;
      }
      if (d.W2bar != nullptr) {  // slot of iteration k + 1, dead: plain stores
        __stcg(reinterpret_cast<float4*>(d.W2bar + i),
               make_float4(-beta * ub4.x, -beta * ub4.y, -beta * ub4.z, -beta * ub4.w));
        __stcg(reinterpret_cast<float4*>(d.B2bar + i),
               make_float4(-beta * bb4.x, -beta * bb4.y, -beta * bb4.z, -beta * bb4.w));
      }
    }
  }
  p_gamma *= -(double)d.inv_gamma;
}

// Sum of two doubles over the CTA, added to acc[0], acc[1] by one thread.
__device__ __forceinline__ void slab_cta_add2(double v0, double v1, double* acc) {
  __shared__ double part[2][kSlabWarps];
  for (int off = 16; off > 0; off >>= 1) {
    v0 += __shfl_xor_sync(0xffffffffu, v0, off);
    v1 += __shfl_xor_sync(0xffffffffu, v1, off);
  }
  if ((threadIdx.x & 31) == 0) {
    part[0][threadIdx.x >> 5] = v0;
    part[1][threadIdx.x >> 5] = v1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int w = 0; w < kSlabWarps; ++w) {
      t0 += part[0][w];
      t1 += part[1][w];
    }
    atomicAdd(acc, t0);
    atomicAdd(acc + 1, t1);
  }
}

// Restart test of iteration k - 1 (reading of Goldstein et al.'s rule): the
// CTA's share of c_{k-1} goes into racc[0]; the last CTA of the grid to
// report compares c_{k-1} with eta cbar and, on a restart, rewrites the
// factors of iterations k + 1 .. kmax as beta_0, beta_1, ...  All threads of
// the CTA call this.
__device__ __forceinline__ void slab_restart_test(const SlabArgs& a, float part, int k,
                                                  unsigned nctas) {
  __shared__ float warp_sum[kSlabWarps];
  for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double cta = 0.0;
    for (int w = 0; w < kSlabWarps; ++w) cta += warp_sum[w];
    atomicAdd(a.racc, cta);
    __threadfence();
    if (atomicAdd(a.rwords, 1u) == nctas - 1) {  // every CTA of the pair has reported
      __threadfence();
      const double ck = atomicAdd(a.racc, 0.0);
      const double cbar = a.racc[1];
      if (a.eta > 0.0f && ck < (double)a.eta * cbar) {
        a.racc[1] = ck;
      } else {
        if (a.eta > 0.0f) a.racc[1] = cbar / (double)a.eta;
        for (int m = 0; k + 1 + m <= a.kmax; ++m) a.beta_dev[k + 1 + m] = a.beta_seq[m];
        if (k + 1 <= a.kmax) a.rwords[1] += 1u;  // count restarts that take effect
      }
      a.racc[0] = 0.0;
      a.rwords[0] = 0u;
      __threadfence();
    }
  }
}
#endif

#if defined(__CUDA_ARCH__)
// The slab pass of z-plane z of one grid (pair), run by the cluster of three
// CTAs that owns it: beta_k and k are the factor and index of the iteration
// the pass starts, nctas the pair's CTA count, lead the CTA that resets the
// restart state of a new inner loop.
// pass: how many planes this CTA has already taken in this launch (the
// mbarrier is set up on the first and its phase alternates).
template <int MODE>
__device__ __forceinline__ void slab_body(const SlabArgs& a, int z, float beta_k, int k,
                                          unsigned nctas, bool lead, int pass) {
  constexpr bool kAdjoint = (MODE == SLAB_ADJ || MODE == SLAB_ADJ_LAST);
  constexpr bool kInverse = (MODE == SLAB_SPEC || MODE == SLAB_SPEC_PREV || MODE == SLAB_FINAL ||
                             kAdjoint);
  constexpr bool kForward = (MODE != SLAB_FINAL && MODE != SLAB_ADJ_LAST);
  constexpr bool kCoupled = (MODE != SLAB_FINAL && MODE != SLAB_FIELD);
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  float2* plane = reinterpret_cast<float2*>(smem + 16);
  float2* xch = plane + (size_t)a.ny * a.nkx;
  cg::cluster_group cluster = cg::this_cluster();
  const int comp = (int)cluster.block_rank();
  const int tid = threadIdx.x;
  const uint32_t plane_bytes = (uint32_t)((size_t)a.ny * a.nkx * sizeof(float2));
  float2* gplane = a.spec + ((size_t)z * 3 + comp) * a.ny * a.nkx;
  if (pass == 0) {
    if (kInverse) {
      if (tid == 0) {
        mbar_init(bar, 1);
        fence_barrier_init();
      }
      __syncthreads();
    }
    pdl_wait();  // the spectrum, J and c come from the kernels before
    pdl_trigger();
  }
  if (kInverse) {
    const uint32_t parity = (uint32_t)(pass & 1);
    if (tid == 0) {  // the previous plane's store has read the buffer (bulk_wait_read)
      mbar_expect_tx(bar, plane_bytes);
      bulk_load(plane, gplane, plane_bytes, bar);
    }
    const bool ok = __syncthreads_and(mbar_wait_bounded(bar, parity));
    if (!ok) {
      if (tid == 0 && a.status != nullptr) atomicOr(a.status, kStatusTimeout);
      mbar_wait_bounded(bar, parity);  // let the copy land before the plane is touched
    }
    cols_rt(a, plane, xch, true);
    __syncthreads();
    rows_rt(a, plane, xch, true);
  }
  const size_t V = (size_t)a.nx * a.ny * a.nz;
  if (kCoupled) {
    cluster.sync();  // every component's plane holds w^{k-1} (or is to be written)
    float2* const planes[3] = {cluster.map_shared_rank(plane, 0), cluster.map_shared_rank(plane, 1),
                               cluster.map_shared_rank(plane, 2)};
    const int Q = a.ny * (a.nx >> 2);
    const int q0 = (int)((long long)Q * comp / 3), q1 = (int)((long long)Q * (comp + 1) / 3);
    if (MODE == SLAB_FIRST && a.restart && lead && tid == 0) {
      // a new inner loop: the factors of Eq. 5, cbar = +inf
      for (int i = 0; i <= a.kmax; ++i) a.beta_dev[i] = (i == 0) ? 0.0f : a.beta_seq[i - 1];
      a.racc[0] = 0.0;
      a.racc[1] = __longlong_as_double(0x7ff0000000000000ll);
      a.rwords[0] = 0u;
    }
    if (kAdjoint) {
      double p_theta = 0.0, p_gamma = 0.0;
      slab_adjoint<MODE>(a, planes, z, q0, q1, p_theta, p_gamma);
      slab_cta_add2(p_theta, p_gamma, a.adj.acc + 1);
    } else if ((MODE == SLAB_SPEC || MODE == SLAB_SPEC_PREV) && a.restart) {
      const float part = slab_pointwise<MODE, true>(a, planes, z, q0, q1, beta_k, k);
      slab_restart_test(a, part, k, nctas);
    } else {
      slab_pointwise<MODE, false>(a, planes, z, q0, q1, beta_k, k);
    }
    cluster.sync();  // every plane holds y^k; no remote access after this
  } else {
    __syncthreads();
    const int Q = a.ny * (a.nx >> 2);
    const int qrow = a.nx >> 2;
    for (int q = tid; q < Q; q += kSlabThreads) {
      const int yy = (int)fdiv((uint32_t)q, a.qdiv);
      const int x0 = (q - yy * qrow) << 2;
      const size_t i = comp * V + ((size_t)z * a.ny + yy) * a.nx + x0;
      float4* rq = real_quad(plane, a.nkx, yy, x0);
      if (MODE == SLAB_FIELD) {
        *rq = __ldg(reinterpret_cast<const float4*>(a.w_in + i));
      } else {  // FINAL
        const float4 w = *rq;
        *reinterpret_cast<float4*>(a.w_out + i) = w;
        if (a.b_out != nullptr)
          *reinterpret_cast<float4*>(a.b_out + i) = f4sub(*reinterpret_cast<const float4*>(a.y + i), w);
      }
    }
    __syncthreads();
  }
  if (kForward) {
    rows_rt(a, plane, xch, false);
    __syncthreads();
    cols_rt(a, plane, xch, false);
    fence_proxy_async();  // the plane's generic-proxy writes, seen by the bulk store
    __syncthreads();
    if (tid == 0) {
      bulk_store(gplane, plane, plane_bytes);
      bulk_commit();
      bulk_wait_read();  // shared memory must stay until the store has read it
    }
  }
}
#endif

// MODE: SLAB_FIRST, SLAB_SPEC (k = 1), SLAB_SPEC_PREV (k >= 2), SLAB_FINAL,
// SLAB_FIELD, SLAB_STATE (k = 1), SLAB_STATE_PREV (k >= 2), SLAB_ADJ,
// SLAB_ADJ_LAST (reverse steps k >= 1 and k = 0).
// A cluster takes planes z = cluster, cluster + clusters, ... (one plane
// each when the grid has nz clusters; a.zper planes each with fewer).
template <int MODE>
__global__ void __cluster_dims__(3, 1, 1) __launch_bounds__(kSlabThreads, 2)
    k_slab(const __grid_constant__ SlabArgs a) {
#if defined(__CUDA_ARCH__)
  const int clusters = (int)(gridDim.x / 3);
  int pass = 0;
  for (int z = (int)(blockIdx.x / 3); z < a.nz; z += clusters, ++pass)
    slab_body<MODE>(a, z, a.beta, a.k, 3u * (unsigned)a.nz, blockIdx.x == 0 && pass == 0, pass);
#endif
}

// The slab pass of many grids in one launch: pair p owns CTAs
// [start[p], start[p+1]) (3 nz_p of them, so no cluster straddles two pairs).
template <int MODE>
__global__ void __cluster_dims__(3, 1, 1) __launch_bounds__(kSlabThreads, 2)
    k_slab_multi(const SlabArgs* __restrict__ pairs, const int* __restrict__ start, int npairs,
                 float beta_k, int k) {
#if defined(__CUDA_ARCH__)
  int lo = 0, hi = npairs - 1;  // the last pair whose first CTA is <= blockIdx.x
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(start + mid) <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const int local = (int)blockIdx.x - __ldg(start + lo);
  slab_body<MODE>(pairs[lo], local / 3, beta_k, k, (unsigned)(__ldg(start + lo + 1) - __ldg(start + lo)),
                  local == 0, 0);
#endif
}


// ---------------------------------------------------------------- z-pass
constexpr int kZSlabThreads = 128;  // 4 independent warps

template <int R1, int R2>
constexpr int zslab_min_blocks() {
  return (R2 == 8 && R1 <= 12) ? 8 : 6;
}

// One warp: 32/R2 consecutive kx columns of one (component, y) row, R2 lanes
// per column; lane l holds z positions l + R2 j.  The second stage fuses the
// last forward stage, the multiply by 1/(1 + gamma K^n)/(nx ny nz) and the
// first inverse stage.
template <int R1, int R2>
__device__ __forceinline__ void zslab_body(const PencilArgs& a, int blk) {
  constexpr int N = R1 * R2, CPW = 32 / R2;
  constexpr int P = N + (R2 == 8 ? 4 : 8);
  extern __shared__ float2 sm_all[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int l = lane / CPW, col = lane % CPW;
  float2* sm = sm_all + (warp * CPW + col) * P;
  const int groups = (a.nkx + CPW - 1) / CPW;  // kx groups per (component, y) row
  const int tasks = 3 * a.ny * groups;
  const int task = blk * (kZSlabThreads / 32) + warp;
  const bool task_ok = task < tasks;
  const int row = task_ok ? task / groups : 0;  // component * ny + y
  const int kx0 = (task_ok ? task - row * groups : 0) * CPW + col;
  const bool active = task_ok && kx0 < a.nkx;
  const int kx = active ? kx0 : 0;
  const int y = row % a.ny;
  pdl_wait();
  pdl_trigger();
  float2* base = a.spec + (size_t)row * a.nkx + kx;
  const size_t zs = (size_t)3 * a.ny * a.nkx;
  float2 v[R1];
#pragma unroll
  for (int j = 0; j < R1; ++j) v[j] = active ? __ldcg(base + (l + R2 * j) * zs) : make_float2(0.f, 0.f);
  lane_stage1<R1, R2, false>(v, a.twz, l);
#pragma unroll
  for (int k = 0; k < R1; ++k) sm[swz<R2>(l + R2 * k)] = v[k];
  __syncwarp();
  const float kxy = __ldg(a.Kx + kx) + __ldg(a.Ky + y);
  const int order = a.order_n;
  for (int b = l; b < R1; b += R2) {
    float2 w[R2];
#pragma unroll
    for (int j = 0; j < R2; ++j) w[j] = sm[swz<R2>(b * R2 + j)];
    dft<R2, false>(w);
    float Kn[R2];
#pragma unroll
    for (int k = 0; k < R2; ++k) Kn[k] = kxy + __ldg(a.Kz + b * R2 + k);
    if (order == 2) {  // the orders of the paper's experiments without a loop
#pragma unroll
      for (int k = 0; k < R2; ++k) Kn[k] *= Kn[k];
    } else if (order == 3) {
#pragma unroll
      for (int k = 0; k < R2; ++k) Kn[k] *= Kn[k] * Kn[k];
    } else if (order != 1) {
#pragma unroll
      for (int k = 0; k < R2; ++k) {
        const float K = Kn[k];
        for (int i = 1; i < order; ++i) Kn[k] *= K;
      }
    }
#pragma unroll
    for (int k = 0; k < R2; ++k) w[k] = cscale(w[k], __fdividef(a.scale, 1.0f + a.gamma * Kn[k]));
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

template <int R1, int R2>
__global__ void __launch_bounds__(kZSlabThreads, zslab_min_blocks<R1, R2>())
    k_zslab(const __grid_constant__ PencilArgs a) {
  zslab_body<R1, R2>(a, (int)blockIdx.x);
}

// The z-pass of many grids sharing the z plan [R1, R2] in one launch: pair p
// owns blocks [start[p], start[p+1]).
template <int R1, int R2>
__global__ void __launch_bounds__(kZSlabThreads, zslab_min_blocks<R1, R2>())
    k_zslab_multi(const PencilArgs* __restrict__ pairs, const int* __restrict__ start, int npairs) {
  int lo = 0, hi = npairs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(start + mid) <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  zslab_body<R1, R2>(pairs[lo], (int)blockIdx.x - __ldg(start + lo));
}

// ---------------------------------------------------------------- host side
namespace {

bool slab_x_case(int r1) {
  for (int r : {2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 14, 16})
    if (r == r1) return true;
  return false;
}

bool lane_case(const AxisPlan& p) {
  return p.nst == 2 && p.m[1] == 1 && lane_pair_supported(p.radix[0], p.radix[1]);
}

template <int R1, int R2>
cudaError_t launch_z(const PencilArgs& a, cudaStream_t s) {
  constexpr int N = R1 * R2, CPW = 32 / R2;
  const int groups = (a.nkx + CPW - 1) / CPW;
  const int tasks = 3 * a.ny * groups;
  const int per_cta = kZSlabThreads / 32;
  const dim3 grid((unsigned)((tasks + per_cta - 1) / per_cta));
  const size_t smem = (size_t)per_cta * CPW * (N + (R2 == 8 ? 4 : 8)) * sizeof(float2);
  return launch_pdl(k_zslab<R1, R2>, grid, dim3(kZSlabThreads), smem, s, a);
}

template <typename K>
cudaError_t raise_smem(K kernel) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  int dev = 0, optin = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
    return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - (int)fa.sharedSizeBytes);
}

}  // namespace

bool slab_supported(int nx, int ny, int nz, const AxisPlan& pxh, const AxisPlan& py,
                    const AxisPlan& pz) {
  if (nx % 4 != 0 || pxh.n * 2 != nx) return false;
  if (!(pxh.nst == 2 && pxh.radix[1] == kSlabXR2 && slab_x_case(pxh.radix[0]))) return false;
  if (!lane_case(py) || !lane_case(pz) || py.n != ny || pz.n != nz) return false;
  SlabArgs a{};
  a.nx = nx;
  a.ny = ny;
  a.nz = nz;
  a.nkx = nx / 2 + 1;
  a.mx = nx / 2;
  a.yr2 = py.radix[1];
  return slab_smem_bytes(a) <= 227 * 1024;
}

cudaError_t launch_slab(int mode, const SlabArgs& a, cudaStream_t s) {
  const int zper = a.zper > 1 ? a.zper : 1;
  const dim3 grid((unsigned)(3 * ((a.nz + zper - 1) / zper))), block(kSlabThreads);
  const size_t smem = slab_smem_bytes(a);
  switch (mode) {
    case SLAB_FIRST: return launch_whole(k_slab<SLAB_FIRST>, grid, block, smem, s, a);
    case SLAB_SPEC: return launch_whole(k_slab<SLAB_SPEC>, grid, block, smem, s, a);
    case SLAB_SPEC_PREV: return launch_whole(k_slab<SLAB_SPEC_PREV>, grid, block, smem, s, a);
    case SLAB_FINAL: return launch_whole(k_slab<SLAB_FINAL>, grid, block, smem, s, a);
    case SLAB_FIELD: return launch_whole(k_slab<SLAB_FIELD>, grid, block, smem, s, a);
    case SLAB_STATE: return launch_whole(k_slab<SLAB_STATE>, grid, block, smem, s, a);
    case SLAB_STATE_PREV: return launch_whole(k_slab<SLAB_STATE_PREV>, grid, block, smem, s, a);
    case SLAB_ADJ: return launch_whole(k_slab<SLAB_ADJ>, grid, block, smem, s, a);
    case SLAB_ADJ_LAST: return launch_whole(k_slab<SLAB_ADJ_LAST>, grid, block, smem, s, a);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_zslab(const PencilArgs& a, cudaStream_t s) {
  const int r1 = a.pz.radix[0], r2 = a.pz.radix[1];
#define X(A, B) \
  if (r1 == A && r2 == B) return launch_z<A, B>(a, s);
  NADMM_LANE_CASES(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t slab_max_clusters(const SlabArgs& a, int* clusters) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(3 * a.nz));
  cfg.blockDim = dim3(kSlabThreads);
  cfg.dynamicSmemBytes = slab_smem_bytes(a);
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 3;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaOccupancyMaxActiveClusters(clusters, (void*)k_slab<SLAB_SPEC_PREV>, &cfg);
}

cudaError_t launch_slab_multi(int mode, const SlabArgs* pairs, const int* start, int npairs,
                              int total_ctas, size_t smem, float beta, int k, cudaStream_t s) {
  const dim3 grid((unsigned)total_ctas), block(kSlabThreads);
  switch (mode) {
    case SLAB_FIRST:
      return launch_whole(k_slab_multi<SLAB_FIRST>, grid, block, smem, s, pairs, start, npairs, beta, k);
    case SLAB_SPEC:
      return launch_whole(k_slab_multi<SLAB_SPEC>, grid, block, smem, s, pairs, start, npairs, beta, k);
    case SLAB_SPEC_PREV:
      return launch_whole(k_slab_multi<SLAB_SPEC_PREV>, grid, block, smem, s, pairs, start, npairs,
                        beta, k);
    case SLAB_FINAL:
      return launch_whole(k_slab_multi<SLAB_FINAL>, grid, block, smem, s, pairs, start, npairs, beta, k);
  }
  return cudaErrorInvalidValue;
}

int zslab_blocks(const PencilArgs& a) {
  const int cpw = 32 / a.pz.radix[1];
  const int tasks = 3 * a.ny * ((a.nkx + cpw - 1) / cpw);
  const int per_cta = kZSlabThreads / 32;
  return (tasks + per_cta - 1) / per_cta;
}

namespace {
template <int R1, int R2>
cudaError_t launch_z_multi(const PencilArgs* pairs, const int* start, int npairs, int blocks,
                           cudaStream_t s) {
  constexpr int N = R1 * R2, CPW = 32 / R2;
  const size_t smem = (size_t)(kZSlabThreads / 32) * CPW * (N + (R2 == 8 ? 4 : 8)) * sizeof(float2);
  return launch_pdl(k_zslab_multi<R1, R2>, dim3((unsigned)blocks), dim3(kZSlabThreads), smem, s,
                    pairs, start, npairs);
}
}  // namespace

cudaError_t launch_zslab_multi(int r1, int r2, const PencilArgs* pairs, const int* start, int npairs,
                               int total_blocks, cudaStream_t s) {
#define X(A, B) \
  if (r1 == A && r2 == B) return launch_z_multi<A, B>(pairs, start, npairs, total_blocks, s);
  NADMM_LANE_CASES(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t configure_slab_kernels() {
  cudaError_t e;
  if ((e = raise_smem(k_slab_multi<SLAB_FIRST>)) != cudaSuccess) return e;
  if ((e = raise_smem(k_slab_multi<SLAB_SPEC>)) != cudaSuccess) return e;
  if ((e = raise_smem(k_slab_multi<SLAB_SPEC_PREV>)) != cudaSuccess) return e;
  if ((e = raise_smem(k_slab_multi<SLAB_FINAL>)) != cudaSuccess) return e;
  if ((e = raise_smem(k_slab<SLAB_FIRST>)) != cudaSuccess) return e;
  if ((e = raise_smem(k_slab<SLAB_SPEC>)) != cudaSuccess) return e;
  if ((e = raise_smem(k_slab<SLAB_SPEC_PREV>)) != cudaSuccess) return e;
  if ((e = raise_smem(k_slab<SLAB_FINAL>)) != cudaSuccess) return e;
  if ((e = raise_smem(k_slab<SLAB_FIELD>)) != cudaSuccess) return e;
  if ((e = raise_smem(k_slab<SLAB_STATE>)) != cudaSuccess) return e;
  if ((e = raise_smem(k_slab<SLAB_ADJ>)) != cudaSuccess) return e;
  if ((e = raise_smem(k_slab<SLAB_ADJ_LAST>)) != cudaSuccess) return e;
  return raise_smem(k_slab<SLAB_STATE_PREV>);
}

}  // namespace nadmm
