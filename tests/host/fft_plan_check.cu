// Host-side check of the FFT plans and stage arithmetic shared with the
// kernels (plan.h, fft_device.cuh): for each length n on the command line,
// plan it, run the forward stages on random lines through the host build of
// fft_stage, and print the plan, the largest error against a direct DFT
// (frequency k read at the position the plan assigns it) and the largest
// round-trip error (inverse stages, divided by n).
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "plan.h"

using namespace nadmm;

int main(int argc, char** argv) {
  for (int a = 1; a < argc; ++a) {
    const int n = std::atoi(argv[a]);
    AxisPlan p;
    if (!factor_axis(n, p, true)) {
      std::printf("%d none\n", n);
      continue;
    }
    const std::vector<float2> tw = axis_twiddles(p);
    const std::vector<int> pos = pos_table(p);
    const int nlines = 3;
    std::mt19937 rng(n);
    std::normal_distribution<double> N(0.0, 1.0);
    std::vector<float2> buf(nlines * n);
    for (auto& v : buf) v = make_float2((float)N(rng), (float)N(rng));
    const std::vector<float2> orig = buf;
    const FastDiv ld = make_fastdiv(nlines);
    for (int s = 0; s < p.nst; ++s) fft_stage<false>(p, s, buf.data(), nlines, ld, 1, n, tw.data(), 0, 1);
    double err = 0.0, mag = 0.0;
    const double two_pi = 6.283185307179586476925286766559;
    for (int l = 0; l < nlines; ++l)
      for (int k = 0; k < n; ++k) {
        std::complex<double> acc = 0.0;
        for (int j = 0; j < n; ++j) {
          const double ang = -two_pi * (double)((long long)j * k % n) / n;
          acc += std::complex<double>(orig[l * n + j].x, orig[l * n + j].y) * std::polar(1.0, ang);
        }
        const float2 g = buf[l * n + pos[k]];
        err = std::fmax(err, std::abs(acc - std::complex<double>(g.x, g.y)));
        mag = std::fmax(mag, std::abs(acc));
      }
    for (int s = p.nst - 1; s >= 0; --s) fft_stage<true>(p, s, buf.data(), nlines, ld, 1, n, tw.data(), 0, 1);
    double rt = 0.0;
    for (int i = 0; i < nlines * n; ++i)
      rt = std::fmax(rt, std::fabs(buf[i].x / n - orig[i].x) + std::fabs(buf[i].y / n - orig[i].y));
    std::printf("%d", n);
    for (int s = 0; s < p.nst; ++s) std::printf(" %d%s", p.radix[s], p.root_off[s] >= 0 ? "g" : "");
    std::printf(" | %.3e %.3e %d\n", err / mag, rt, p.tw_count);
  }
  return 0;
}
