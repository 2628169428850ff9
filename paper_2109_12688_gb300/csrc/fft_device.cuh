// In-place mixed-radix FFT building blocks for lines held in shared memory.
//
// The regulariser step of the method (Eq. 6, last line) is a division in the
// spectrum of the 3D DFT.  Because the symbol 1/(1 + gamma K^n) is applied
// point-wise, the forward transform may leave its output in any known order:
// the forward pass is a decimation-in-frequency (DIF) FFT that stores each
// stage's outputs back into the positions it read (no reordering), so its
// result is in mixed-radix digit-reversed order; the inverse is the exact
// stage-by-stage inverse (decimation in time, conjugate twiddles, stages in
// reverse order), which takes that order back to natural order.  No
// transposition or bit-reversal pass is ever made.
//
// Stage i (1-based) of a length-N transform with radices r_1..r_S works on
// blocks of length L_i = N / (r_1...r_{i-1}); with m_i = L_i / r_i it reads
// x[n1 + m_i j] (j < r_i) of each block, forms the r_i-point DFT over j,
// multiplies output k by w_{L_i}^{n1 k} and stores it at n1 + m_i k.  The
// frequency stored at position p = sum_i d_i m_i is k = sum_i d_i r_1..r_{i-1}.
//
// A prime factor r > 7 of N (sizes with no codelet radix) gets a generic
// stage: the same stage with the r-point DFT evaluated directly as a sum of r
// terms with the roots w_r^q (q < r) from the axis table.  It costs O(r) per
// element instead of O(log r), needs no padding (unlike a chirp-z transform
// of length >= 2r - 1), and the plan puts such stages first.
//
// Every function here is __host__ __device__ and takes (tid, nthr) so that a
// block-level loop is plain C++; the kernels separate phases with barriers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#if defined(__CUDACC__)
#define NADMM_HD __host__ __device__ __forceinline__
#else
#define NADMM_HD inline
#endif

namespace nadmm {

constexpr int kMaxStages = 5;
// Largest prime factor an axis may have (a generic stage of radix r keeps at
// most kPrimeItems outputs per thread per round; r <= 4 x 128 threads).
constexpr int kMaxPrime = 509;
constexpr int kPrimeItems = 4;

// Division by a runtime-invariant divisor d >= 1 for 0 <= n < 2^31, by the
// round-up multiplier method (Granlund & Montgomery, "Division by invariant
// integers using multiplication", 1994): with l = ceil(log2 d), p = 31 + l,
// mul = ceil(2^p / d), q = floor(n * mul / 2^p).
struct FastDiv {
  uint32_t d, mul, shift;  // shift = p - 32 (unused when d == 1)
};

inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  if (d <= 1) {
    f.mul = 0;
    f.shift = 0;
    return f;
  }
  uint32_t l = 0;
  while ((1ull << l) < d) ++l;
  uint64_t p2 = 1ull << (31 + l);
  f.mul = (uint32_t)((p2 + d - 1) / d);
  f.shift = l - 1;
  return f;
}

#if defined(__CUDACC__)
// Device-side construction (slow path for ragged tails only).
__device__ __forceinline__ FastDiv make_fastdiv_dev(uint32_t d) {
  FastDiv f;
  f.d = d;
  if (d <= 1) {
    f.mul = 0;
    f.shift = 0;
    return f;
  }
  uint32_t l = 0;
  while ((1ull << l) < d) ++l;
  const unsigned long long p2 = 1ull << (31 + l);
  f.mul = (uint32_t)((p2 + d - 1) / d);
  f.shift = l - 1;
  return f;
}
#endif

NADMM_HD uint32_t fdiv(uint32_t n, const FastDiv& f) {
  if (f.d <= 1) return n;
#if defined(__CUDA_ARCH__)
  return __umulhi(n, f.mul) >> f.shift;
#else
  return (uint32_t)(((uint64_t)n * f.mul) >> 32) >> f.shift;
#endif
}

// Radix plan of one axis, passed to kernels by value.
struct AxisPlan {
  int n;                     // transform length
  int nst;                   // number of stages
  int radix[kMaxStages];     // r_i
  int L[kMaxStages];         // block length at stage i
  int m[kMaxStages];         // L_i / r_i
  int tw_off[kMaxStages];    // offset of stage i's twiddles in the axis table
  int root_off[kMaxStages];  // generic prime stage: offset of its roots w_r^q, q < r,
                             // in the axis table; -1 for codelet stages
  int tw_count;              // entries in the axis table
  FastDiv mdiv[kMaxStages];  // division by m_i
};

NADMM_HD float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
NADMM_HD float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
NADMM_HD float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
NADMM_HD float2 cmulc(float2 a, float2 b) {  // a * conj(b)
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
NADMM_HD float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
NADMM_HD float2 rot90(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// ----------------------------------------------------------------- codelets
// Forward: X_k = sum_j x_j exp(-2 pi i jk/R); inverse uses exp(+2 pi i jk/R)
// and is unnormalised.
template <bool INV>
NADMM_HD void dft2(float2& a, float2& b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <bool INV>
NADMM_HD void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
  float2 t0 = cadd(x0, x2), t1 = csub(x0, x2);
  float2 t2 = cadd(x1, x3), t3 = rot90<INV>(csub(x1, x3));
  x0 = cadd(t0, t2);
  x2 = csub(t0, t2);
  x1 = cadd(t1, t3);
  x3 = csub(t1, t3);
}

// cos/sin of 2 pi m / 16 for m = 0..3 (the rest follow by symmetry)
struct C16 {
  static constexpr float c1 = 0.92387953251128674f;  // cos(pi/8)
  static constexpr float s1 = 0.38268343236508978f;  // sin(pi/8)
  static constexpr float h = 0.70710678118654752f;   // cos(pi/4)
};

// multiply by w_8^k (k = 0..3), forward w = exp(-i pi/4)
template <bool INV, int K>
NADMM_HD float2 tw8(float2 a) {
  if (K == 0) return a;
  if (K == 2) return rot90<INV>(a);
  const float h = C16::h;
  if (K == 1) {  // (1 - i)/sqrt2 forward, (1 + i)/sqrt2 inverse
    return INV ? make_float2(h * (a.x - a.y), h * (a.x + a.y))
               : make_float2(h * (a.x + a.y), h * (a.y - a.x));
  }
  // K == 3: (-1 - i)/sqrt2 forward, (-1 + i)/sqrt2 inverse
  return INV ? make_float2(-h * (a.x + a.y), h * (a.x - a.y))
             : make_float2(h * (a.y - a.x), -h * (a.x + a.y));
}

template <bool INV>
NADMM_HD void dft8(float2 (&x)[8]) {
  // even/odd split: E = DFT4(x0,x2,x4,x6), O = DFT4(x1,x3,x5,x7)
  float2 e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
  float2 o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  o1 = tw8<INV, 1>(o1);
  o2 = tw8<INV, 2>(o2);
  o3 = tw8<INV, 3>(o3);
  x[0] = cadd(e0, o0); x[4] = csub(e0, o0);
  x[1] = cadd(e1, o1); x[5] = csub(e1, o1);
  x[2] = cadd(e2, o2); x[6] = csub(e2, o2);
  x[3] = cadd(e3, o3); x[7] = csub(e3, o3);
}

// multiply by w_16^m for m in [0, 9]
template <bool INV>
NADMM_HD float2 tw16(float2 a, int m) {
  float c, s;  // exp(-2 pi i m/16) = c - i s  (forward)
  switch (m) {
    case 0: return a;
    case 1: c = C16::c1; s = C16::s1; break;
    case 2: c = C16::h; s = C16::h; break;
    case 3: c = C16::s1; s = C16::c1; break;
    case 4: return rot90<INV>(a);
    case 6: c = -C16::h; s = C16::h; break;
    case 9: c = -C16::c1; s = -C16::s1; break;
    default: c = 1.f; s = 0.f; break;
  }
  float sg = INV ? -s : s;  // forward multiplies by (c - i s)
  return make_float2(a.x * c + a.y * sg, a.y * c - a.x * sg);
}

template <bool INV>
NADMM_HD void dft16(float2 (&x)[16]) {
  // 16 = 4 x 4: inner DFT4 over n1 of x[4 n1 + n2], twiddle w16^{n2 k1},
  // outer DFT4 over n2; output index k1 + 4 k2.
  float2 y[16];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    float2 a = x[n2], b = x[4 + n2], c = x[8 + n2], d = x[12 + n2];
    dft4<INV>(a, b, c, d);
    y[0 * 4 + n2] = a;
    y[1 * 4 + n2] = tw16<INV>(b, n2);
    y[2 * 4 + n2] = tw16<INV>(c, 2 * n2);
    y[3 * 4 + n2] = tw16<INV>(d, 3 * n2);
  }
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    float2 a = y[k1 * 4 + 0], b = y[k1 * 4 + 1], c = y[k1 * 4 + 2], d = y[k1 * 4 + 3];
    dft4<INV>(a, b, c, d);
    x[k1] = a;
    x[k1 + 4] = b;
    x[k1 + 8] = c;
    x[k1 + 12] = d;
  }
}

// odd prime radices: cos/sin(2 pi m/R), m = 1..(R-1)/2
template <int R> struct OddTab;
template <> struct OddTab<3> {
  NADMM_HD static float c(int m) { (void)m; return -0.5f; }
  NADMM_HD static float s(int m) { (void)m; return 0.86602540378443865f; }
};
template <> struct OddTab<5> {
  NADMM_HD static float c(int m) { return m == 1 ? 0.30901699437494742f : -0.80901699437494742f; }
  NADMM_HD static float s(int m) { return m == 1 ? 0.95105651629515357f : 0.58778525229247313f; }
};
template <> struct OddTab<7> {
  NADMM_HD static float c(int m) {
    return m == 1 ? 0.62348980185873353f : (m == 2 ? -0.22252093395631440f : -0.90096886790241913f);
  }
  NADMM_HD static float s(int m) {
    return m == 1 ? 0.78183148246802981f : (m == 2 ? 0.97492791218182361f : 0.43388373911755812f);
  }
};

// cos(2 pi q/R) and sin(2 pi q/R) for any integer q, from the half table
template <int R>
NADMM_HD void odd_cs(int q, float& c, float& s) {
  q %= R;
  if (q == 0) { c = 1.f; s = 0.f; return; }
  if (q <= (R - 1) / 2) { c = OddTab<R>::c(q); s = OddTab<R>::s(q); return; }
  c = OddTab<R>::c(R - q);
  s = -OddTab<R>::s(R - q);
}

template <int R, bool INV>
NADMM_HD void dft_odd(float2 (&x)[R]) {
  constexpr int H = (R - 1) / 2;
  float2 a[H], d[H];
#pragma unroll
  for (int j = 1; j <= H; ++j) {
    a[j - 1] = cadd(x[j], x[R - j]);
    d[j - 1] = csub(x[j], x[R - j]);
  }
  float2 x0 = x[0];
  float2 sum = x0;
#pragma unroll
  for (int j = 0; j < H; ++j) sum = cadd(sum, a[j]);
#pragma unroll
  for (int k = 1; k <= H; ++k) {
    float2 P = x0, Q = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 1; j <= H; ++j) {
      float c, s;
      odd_cs<R>(j * k, c, s);
      P = cadd(P, cscale(a[j - 1], c));
      Q = cadd(Q, cscale(d[j - 1], s));
    }
    // forward: X_k = P - i Q, X_{R-k} = P + i Q
    float2 iQ = rot90<INV>(Q);  // -iQ forward, +iQ inverse
    x[k] = cadd(P, iQ);
    x[R - k] = csub(P, iQ);
  }
  x[0] = sum;
}

// cos/sin(2 pi m / R) for m = 0..6, R in {6, 9, 10, 12}: the internal
// twiddles of the composite codelets (m = n2 k1 never exceeds 6 there).
template <int R> struct CompTab;
template <> struct CompTab<6> {
  NADMM_HD static float c(int m) {
    const float t[7] = {1.f, 0.5f, -0.5f, -1.f, -0.5f, 0.5f, 1.f};
    return t[m];
  }
  NADMM_HD static float s(int m) {
    const float t[7] = {0.f, 0.86602540378443865f, 0.86602540378443865f, 0.f,
                        -0.86602540378443865f, -0.86602540378443865f, 0.f};
    return t[m];
  }
};
template <> struct CompTab<9> {
  NADMM_HD static float c(int m) {
    const float t[7] = {1.f, 0.76604444311897801f, 0.17364817766693041f, -0.5f,
                        -0.93969262078590832f, -0.93969262078590843f, -0.5f};
    return t[m];
  }
  NADMM_HD static float s(int m) {
    const float t[7] = {0.f, 0.64278760968653925f, 0.98480775301220802f, 0.86602540378443865f,
                        0.34202014332566888f, -0.34202014332566866f, -0.86602540378443865f};
    return t[m];
  }
};
template <> struct CompTab<10> {
  NADMM_HD static float c(int m) {
    const float t[7] = {1.f, 0.80901699437494745f, 0.30901699437494745f, -0.30901699437494734f,
                        -0.80901699437494734f, -1.f, -0.80901699437494756f};
    return t[m];
  }
  NADMM_HD static float s(int m) {
    const float t[7] = {0.f, 0.58778525229247314f, 0.95105651629515353f, 0.95105651629515364f,
                        0.58778525229247325f, 0.f, -0.58778525229247303f};
    return t[m];
  }
};
template <> struct CompTab<12> {
  NADMM_HD static float c(int m) {
    const float t[7] = {1.f, 0.86602540378443865f, 0.5f, 0.f, -0.5f, -0.86602540378443865f, -1.f};
    return t[m];
  }
  NADMM_HD static float s(int m) {
    const float t[7] = {0.f, 0.5f, 0.86602540378443865f, 1.f, 0.86602540378443865f, 0.5f, 0.f};
    return t[m];
  }
};

template <> struct CompTab<14> {
  NADMM_HD static float c(int m) {
    const float t[7] = {1.f, 0.90096886790241915f, 0.62348980185873359f, 0.22252093395631445f,
                        -0.22252093395631434f, -0.62348980185873348f, -0.90096886790241903f};
    return t[m];
  }
  NADMM_HD static float s(int m) {
    const float t[7] = {0.f, 0.43388373911755812f, 0.7818314824680298f, 0.97492791218182362f,
                        0.97492791218182362f, 0.78183148246802991f, 0.43388373911755823f};
    return t[m];
  }
};

template <int R, bool INV>
NADMM_HD void dft(float2 (&x)[R]);

// R = A * B in registers: inner A-point DFTs over n1 of x[B n1 + n2],
// twiddle w_R^{n2 k1}, outer B-point DFTs over n2; output X[k1 + A k2].
template <int A, int B, bool INV>
NADMM_HD void dft_composite(float2 (&x)[A * B]) {
  constexpr int R = A * B;
  float2 y[R];
#pragma unroll
  for (int n2 = 0; n2 < B; ++n2) {
    float2 a[A];
#pragma unroll
    for (int n1 = 0; n1 < A; ++n1) a[n1] = x[B * n1 + n2];
    dft<A, INV>(a);
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) {
      const int m = n2 * k1;
      float2 v = a[k1];
      if (m != 0) {
        const float c = CompTab<R>::c(m), s = CompTab<R>::s(m);
        const float sg = INV ? -s : s;
        v = make_float2(v.x * c + v.y * sg, v.y * c - v.x * sg);
      }
      y[k1 * B + n2] = v;
    }
  }
#pragma unroll
  for (int k1 = 0; k1 < A; ++k1) {
    float2 b[B];
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) b[n2] = y[k1 * B + n2];
    dft<B, INV>(b);
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) x[k1 + A * k2] = b[k2];
  }
}

template <int R, bool INV>
NADMM_HD void dft(float2 (&x)[R]) {
  if constexpr (R == 2) {
    dft2<INV>(x[0], x[1]);
  } else if constexpr (R == 4) {
    dft4<INV>(x[0], x[1], x[2], x[3]);
  } else if constexpr (R == 8) {
    dft8<INV>(x);
  } else if constexpr (R == 16) {
    dft16<INV>(x);
  } else if constexpr (R == 6) {
    dft_composite<3, 2, INV>(x);
  } else if constexpr (R == 9) {
    dft_composite<3, 3, INV>(x);
  } else if constexpr (R == 10) {
    dft_composite<5, 2, INV>(x);
  } else if constexpr (R == 12) {
    dft_composite<4, 3, INV>(x);
  } else if constexpr (R == 14) {
    dft_composite<7, 2, INV>(x);
  } else {
    dft_odd<R, INV>(x);
  }
}

// One radix-R butterfly of a stage: positions base[j * step], j < R.
// Forward: DFT then twiddle w_L^{n1 k}; inverse: conjugate twiddle then
// inverse DFT.  tw points at the stage table [(k-1) * m + n1].
template <int R, bool INV>
NADMM_HD void butterfly(float2* base, int step, const float2* tw, int m, int n1) {
  float2 x[R];
#pragma unroll
  for (int j = 0; j < R; ++j) x[j] = base[j * step];
  if (!INV) {
    dft<R, false>(x);
    if (m > 1) {
#pragma unroll
      for (int k = 1; k < R; ++k) x[k] = cmul(x[k], tw[(k - 1) * m + n1]);
    }
  } else {
    if (m > 1) {
#pragma unroll
      for (int k = 1; k < R; ++k) x[k] = cmulc(x[k], tw[(k - 1) * m + n1]);
    }
    dft<R, true>(x);
  }
#pragma unroll
  for (int j = 0; j < R; ++j) base[j * step] = x[j];
}

// All butterflies of stage s over a batch of `nlines` lines: element e of
// line l lives at buf[l * ls + e * es].  Work item g -> (line fastest, then
// n1, then block) so that a warp's lanes sit on different lines.
template <int R, bool INV>
NADMM_HD void stage_loop(float2* buf, int nlines, const FastDiv& ldiv, int es, int ls, int L, int m,
                         const FastDiv& mdiv, const float2* tw, int nblk, int tid, int nthr) {
  const int total = nlines * nblk * m;
  const int step = m * es;
  for (int g = tid; g < total; g += nthr) {
    const int q = (int)fdiv((uint32_t)g, ldiv);
    const int line = g - q * nlines;
    const int blk = (int)fdiv((uint32_t)q, mdiv);
    const int n1 = q - blk * m;
    float2* base = buf + line * ls + (blk * L + n1) * es;
    butterfly<R, INV>(base, step, tw, m, n1);
  }
}

// Output k of the r-point butterfly at `base` (elements base[j * step]):
// forward  X_k = (sum_j x_j w_r^{jk}) w_L^{n1 k};
// inverse  X_k = sum_j (x_j conj(w_L^{n1 j})) conj(w_r)^{jk}.
template <bool INV>
NADMM_HD float2 prime_output(const float2* base, int step, int r, int k, const float2* tw,
                             const float2* root, int m, int n1) {
  float2 acc = make_float2(0.0f, 0.0f);
  int e = 0;  // j k mod r
  for (int j = 0; j < r; ++j) {
    float2 xj = base[j * step];
    if (INV && j > 0 && m > 1) xj = cmulc(xj, tw[(j - 1) * m + n1]);
    acc = cadd(acc, INV ? cmulc(xj, root[e]) : cmul(xj, root[e]));
    e += k;
    if (e >= r) e -= r;
  }
  if (!INV && k > 0 && m > 1) acc = cmul(acc, tw[(k - 1) * m + n1]);
  return acc;
}

// Generic stage of prime radix r (every thread of the block calls it).  The
// butterflies are taken in rounds of whole butterflies, at most kPrimeItems
// outputs per thread: each round computes its outputs into registers, waits
// for the block, then writes them over the round's own inputs (the rounds'
// butterflies are disjoint, so no later round reads what a round writes).
template <bool INV>
NADMM_HD void prime_stage(const AxisPlan& p, int s, float2* buf, int nlines, int es, int ls,
                          const float2* tw_axis, int tid, int nthr) {
  const int r = p.radix[s], L = p.L[s], m = p.m[s], nblk = p.n / L;
  const float2* tw = tw_axis + p.tw_off[s];
  const float2* root = tw_axis + p.root_off[s];
  const int step = m * es;
  const int nbf = nlines * nblk * m;
#if defined(__CUDA_ARCH__)
  int per_round = (nthr * kPrimeItems) / r;
  if (per_round < 1) per_round = 1;  // excluded by the plan (r <= kMaxPrime)
  const int rounds = (nbf + per_round - 1) / per_round;
  for (int rd = 0; rd < rounds; ++rd) {
    float2 out[kPrimeItems];
    int dst[kPrimeItems];
#pragma unroll
    for (int it = 0; it < kPrimeItems; ++it) {
      dst[it] = -1;
      const int g = tid + it * nthr;  // (butterfly in round, output k)
      const int b = g / r, k = g - b * r;
      const int bf = rd * per_round + b;
      if (b < per_round && bf < nbf) {
        const int q = bf / nlines, line = bf - q * nlines;
        const int blk = q / m, n1 = q - blk * m;
        const int off = line * ls + (blk * L + n1) * es;
        out[it] = prime_output<INV>(buf + off, step, r, k, tw, root, m, n1);
        dst[it] = off + k * step;
      }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kPrimeItems; ++it)
      if (dst[it] >= 0) buf[dst[it]] = out[it];
    __syncthreads();
  }
#else
  (void)tid;
  (void)nthr;
  float2 out[kMaxPrime];
  for (int bf = 0; bf < nbf; ++bf) {
    const int q = bf / nlines, line = bf - q * nlines;
    const int blk = q / m, n1 = q - blk * m;
    float2* base = buf + line * ls + (blk * L + n1) * es;
    for (int k = 0; k < r; ++k) out[k] = prime_output<INV>(base, step, r, k, tw, root, m, n1);
    for (int k = 0; k < r; ++k) base[k * step] = out[k];
  }
#endif
}

// Stage s of plan p (forward or inverse); tw_axis is the axis table.
template <bool INV>
NADMM_HD void fft_stage(const AxisPlan& p, int s, float2* buf, int nlines, const FastDiv& ldiv,
                        int es, int ls, const float2* tw_axis, int tid, int nthr) {
  if (p.root_off[s] >= 0) {
    prime_stage<INV>(p, s, buf, nlines, es, ls, tw_axis, tid, nthr);
    return;
  }
  const int L = p.L[s], m = p.m[s], nblk = p.n / L;
  const float2* tw = tw_axis + p.tw_off[s];
  const FastDiv& md = p.mdiv[s];
  switch (p.radix[s]) {
    case 2: stage_loop<2, INV>(buf, nlines, ldiv, es, ls, L, m, md, tw, nblk, tid, nthr); break;
    case 3: stage_loop<3, INV>(buf, nlines, ldiv, es, ls, L, m, md, tw, nblk, tid, nthr); break;
    case 4: stage_loop<4, INV>(buf, nlines, ldiv, es, ls, L, m, md, tw, nblk, tid, nthr); break;
    case 5: stage_loop<5, INV>(buf, nlines, ldiv, es, ls, L, m, md, tw, nblk, tid, nthr); break;
    case 6: stage_loop<6, INV>(buf, nlines, ldiv, es, ls, L, m, md, tw, nblk, tid, nthr); break;
    case 7: stage_loop<7, INV>(buf, nlines, ldiv, es, ls, L, m, md, tw, nblk, tid, nthr); break;
    case 8: stage_loop<8, INV>(buf, nlines, ldiv, es, ls, L, m, md, tw, nblk, tid, nthr); break;
    case 9: stage_loop<9, INV>(buf, nlines, ldiv, es, ls, L, m, md, tw, nblk, tid, nthr); break;
    case 10: stage_loop<10, INV>(buf, nlines, ldiv, es, ls, L, m, md, tw, nblk, tid, nthr); break;
    case 12: stage_loop<12, INV>(buf, nlines, ldiv, es, ls, L, m, md, tw, nblk, tid, nthr); break;
    case 14: stage_loop<14, INV>(buf, nlines, ldiv, es, ls, L, m, md, tw, nblk, tid, nthr); break;
    default: stage_loop<16, INV>(buf, nlines, ldiv, es, ls, L, m, md, tw, nblk, tid, nthr); break;
  }
}

// Last forward stage (m = 1), point-wise multiply by the filter, and the
// first inverse stage, fused in registers: each group of R consecutive
// positions (step es) is transformed, scaled and transformed back.
// filt(pos) returns the real gain for position pos of the line.
template <int R, class Filt>
NADMM_HD void filter_loop(float2* buf, int nlines, const FastDiv& ldiv, int es, int ls, int n,
                          Filt filt, int tid, int nthr) {
  const int nblk = n / R;
  const int total = nlines * nblk;
  for (int g = tid; g < total; g += nthr) {
    const int blk = (int)fdiv((uint32_t)g, ldiv);
    const int line = g - blk * nlines;
    float2* base = buf + line * ls + blk * R * es;
    float2 x[R];
#pragma unroll
    for (int j = 0; j < R; ++j) x[j] = base[j * es];
    dft<R, false>(x);
#pragma unroll
    for (int k = 0; k < R; ++k) x[k] = cscale(x[k], filt(line, blk * R + k));
    dft<R, true>(x);
#pragma unroll
    for (int j = 0; j < R; ++j) base[j * es] = x[j];
  }
}

template <class Filt>
NADMM_HD void fft_filter_last(const AxisPlan& p, float2* buf, int nlines, const FastDiv& ldiv,
                              int es, int ls, Filt filt, int tid, int nthr) {
  switch (p.radix[p.nst - 1]) {
    case 2: filter_loop<2>(buf, nlines, ldiv, es, ls, p.n, filt, tid, nthr); break;
    case 3: filter_loop<3>(buf, nlines, ldiv, es, ls, p.n, filt, tid, nthr); break;
    case 4: filter_loop<4>(buf, nlines, ldiv, es, ls, p.n, filt, tid, nthr); break;
    case 5: filter_loop<5>(buf, nlines, ldiv, es, ls, p.n, filt, tid, nthr); break;
    case 6: filter_loop<6>(buf, nlines, ldiv, es, ls, p.n, filt, tid, nthr); break;
    case 7: filter_loop<7>(buf, nlines, ldiv, es, ls, p.n, filt, tid, nthr); break;
    case 8: filter_loop<8>(buf, nlines, ldiv, es, ls, p.n, filt, tid, nthr); break;
    case 9: filter_loop<9>(buf, nlines, ldiv, es, ls, p.n, filt, tid, nthr); break;
    case 10: filter_loop<10>(buf, nlines, ldiv, es, ls, p.n, filt, tid, nthr); break;
    case 12: filter_loop<12>(buf, nlines, ldiv, es, ls, p.n, filt, tid, nthr); break;
    case 14: filter_loop<14>(buf, nlines, ldiv, es, ls, p.n, filt, tid, nthr); break;
    default: filter_loop<16>(buf, nlines, ldiv, es, ls, p.n, filt, tid, nthr); break;
  }
}

}  // namespace nadmm
