// Host-side FFT plans and tables for the spectral regulariser step (Eq. 6).
// Twiddles are evaluated in double precision with the host C library and
// rounded once to float.
#pragma once
#include <cmath>
#include <vector>

#include "fft_device.cuh"

namespace nadmm {

// Radices with register codelets.  The plan uses the fewest stages (each
// stage is one pass over shared memory), larger radices first on ties.
constexpr int kRadices[] = {16, 14, 12, 10, 9, 8, 7, 6, 5, 4, 3, 2};

// Lane-FFT plans: n = R1 * R2 with R2 in {8, 16} lanes per line and R1 values
// per lane (a codelet radix); first stage R1, second stage R2.  Returns R2
// (0 if n has no such split), trying R2 = 8 first.
constexpr int kLaneR1[] = {3, 4, 6, 8, 9, 10, 12, 14, 16};

// Whether a two-stage plan [r1, r2] has lane-FFT kernels.
inline bool lane_pair_supported(int r1, int r2) {
  if (r2 != 8 && r2 != 16) return false;
  for (int r : kLaneR1)
    if (r == r1) return true;
  return false;
}

// R2 of the lane plan of n (0 if none); `first` (8 or 16) is tried first.
inline int lane_split(int n, int first = 8) {
  for (int r2 : {first, 24 - first}) {
    if (n % r2) continue;
    for (int r1 : kLaneR1)
      if (r1 == n / r2) return r2;
  }
  return 0;
}

inline bool best_factors(int n, int depth, int* out, int& best_len, int* cur, int len) {
  if (n == 1) {
    if (len < best_len) {
      best_len = len;
      for (int i = 0; i < len; ++i) out[i] = cur[i];
    }
    return true;
  }
  if (len >= depth || len + 1 >= best_len) return false;
  bool found = false;
  for (int r : kRadices) {
    if (n % r) continue;
    cur[len] = r;
    found |= best_factors(n / r, depth, out, best_len, cur, len + 1);
  }
  return found;
}

// Prime factors of n above 7 (the ones without a codelet), ascending, with
// multiplicity; the rest of n (only factors 2, 3, 5, 7) is returned in smooth.
inline int generic_primes(int n, int* out, int cap, int& smooth) {
  int cnt = 0;
  smooth = 1;
  for (int q : {2, 3, 5, 7})
    while (n % q == 0) {
      n /= q;
      smooth *= q;
    }
  for (int q = 11; n > 1 && q <= n; q += 2)
    while (n % q == 0) {
      n /= q;
      if (cnt < cap) out[cnt] = q;
      ++cnt;
    }
  return cnt;
}

inline bool factor_axis(int n, AxisPlan& p, bool lane_plan = false, int lane_first = 8) {
  if (n < 2) return false;
  int out[kMaxStages], cur[kMaxStages], best = kMaxStages + 1;
  int smooth = 1;
  const int ng = generic_primes(n, out, kMaxStages, smooth);
  if (ng > 0) {
    // generic prime stages first, then the fewest codelet stages for the rest
    if (ng > kMaxStages || out[ng - 1] > kMaxPrime) return false;
    if (smooth == 1) {
      best = ng;
    } else {
      int rest[kMaxStages], rbest = kMaxStages + 1;
      if (!best_factors(smooth, kMaxStages - ng, rest, rbest, cur, 0)) return false;
      for (int i = 0; i < rbest; ++i) out[ng + i] = rest[i];
      best = ng + rbest;
    }
  } else {
    const int r2 = lane_plan ? lane_split(n, lane_first) : 0;
    if (r2) {
      out[0] = n / r2;
      out[1] = r2;
      best = 2;
    } else if (!best_factors(n, kMaxStages, out, best, cur, 0)) {
      return false;
    }
  }
  p.n = n;
  p.nst = best;
  int L = n, off = 0;
  for (int i = 0; i < kMaxStages; ++i) {
    if (i < best) {
      p.radix[i] = out[i];
      p.L[i] = L;
      p.m[i] = L / out[i];
      p.tw_off[i] = off;
      if (p.m[i] > 1) off += (out[i] - 1) * p.m[i];
      L /= out[i];
    } else {
      p.radix[i] = 1; p.L[i] = 1; p.m[i] = 1; p.tw_off[i] = off;
    }
    p.mdiv[i] = make_fastdiv((uint32_t)p.m[i]);
  }
  // the roots of the generic stages follow the stage twiddles
  for (int i = 0; i < kMaxStages; ++i) {
    p.root_off[i] = (i < ng) ? off : -1;
    if (i < ng) off += out[i];
  }
  p.tw_count = off > 0 ? off : 1;
  return true;
}

// The two-stage plan [r1, r2] of n = r1 r2 (a lane plan when r2 is 8 or 16).
inline void two_stage_plan(int n, int r1, int r2, AxisPlan& p) {
  p.n = n;
  p.nst = 2;
  const int rad[2] = {r1, r2};
  int L = n, off = 0;
  for (int i = 0; i < kMaxStages; ++i) {
    if (i < 2) {
      p.radix[i] = rad[i];
      p.L[i] = L;
      p.m[i] = L / rad[i];
      p.tw_off[i] = off;
      if (p.m[i] > 1) off += (rad[i] - 1) * p.m[i];
      L /= rad[i];
    } else {
      p.radix[i] = 1; p.L[i] = 1; p.m[i] = 1; p.tw_off[i] = off;
    }
    p.root_off[i] = -1;
    p.mdiv[i] = make_fastdiv((uint32_t)p.m[i]);
  }
  p.tw_count = off > 0 ? off : 1;
}

// Stage twiddles: stage i holds w_{L_i}^{n1 k} at [(k-1) m_i + n1].
inline std::vector<float2> axis_twiddles(const AxisPlan& p) {
  std::vector<float2> tw;
  const double two_pi = 6.283185307179586476925286766559;
  for (int i = 0; i < p.nst; ++i) {
    if (p.m[i] <= 1) continue;
    for (int k = 1; k < p.radix[i]; ++k)
      for (int n1 = 0; n1 < p.m[i]; ++n1) {
        long long e = (long long)n1 * k % p.L[i];
        double a = -two_pi * (double)e / (double)p.L[i];
        tw.push_back(make_float2((float)std::cos(a), (float)std::sin(a)));
      }
  }
  for (int i = 0; i < p.nst; ++i) {
    if (p.root_off[i] < 0) continue;
    for (int q = 0; q < p.radix[i]; ++q) {
      double a = -two_pi * (double)q / (double)p.radix[i];
      tw.push_back(make_float2((float)std::cos(a), (float)std::sin(a)));
    }
  }
  if (tw.empty()) tw.push_back(make_float2(1.f, 0.f));
  return tw;
}

// Position holding frequency k after the forward transform.
inline int freq_to_pos(const AxisPlan& p, int k) {
  int pos = 0;
  for (int i = 0; i < p.nst; ++i) {
    int d = k % p.radix[i];
    k /= p.radix[i];
    pos += d * p.m[i];
  }
  return pos;
}

inline std::vector<int> pos_table(const AxisPlan& p) {
  std::vector<int> t(p.n);
  for (int k = 0; k < p.n; ++k) t[k] = freq_to_pos(p, k);
  return t;
}

// 4 sin^2(pi k / n) stored at the position that holds frequency k, i.e. the
// per-axis term of K = 2 (3 - cos - cos - cos) (text after Eq. 6).
inline std::vector<float> symbol_by_position(const AxisPlan& p) {
  std::vector<float> t(p.n);
  const double pi = 3.14159265358979323846264338328;
  for (int k = 0; k < p.n; ++k) {
    double s = std::sin(pi * (double)k / (double)p.n);
    t[freq_to_pos(p, k)] = (float)(4.0 * s * s);
  }
  return t;
}

inline std::vector<float> symbol_natural(int n, int count) {
  std::vector<float> t(count);
  const double pi = 3.14159265358979323846264338328;
  for (int k = 0; k < count; ++k) {
    double s = std::sin(pi * (double)k / (double)n);
    t[k] = (float)(4.0 * s * s);
  }
  return t;
}

}  // namespace nadmm
