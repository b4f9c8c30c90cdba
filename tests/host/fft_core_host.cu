// Host-side check of the batched FFT building blocks (csrc/fft.cuh): the per-thread
// pass pieces are run for every thread of one transform in the order the kernel's
// barriers impose, with the pass-twiddle table built from the same exponent formula in
// double precision, and compared with a direct O(M^2) DFT in double precision.
// Prints one line per size: "M max_rel_err".
#include <cmath>
#include <complex>
#include <cstdio>
#include <random>
#include <vector>

#include "fft.cuh"

using namespace scd;

template <int M>
double check_size(std::mt19937_64& g) {
  using PI = PlanInfo<M>;
  using F = FftPieces<M>;
  constexpr int E = PI::E, T = PI::T;
  std::normal_distribution<double> nd;
  std::vector<float2> x(M);
  for (auto& v : x) v = make_float2((float)nd(g), (float)nd(g));
  // pass-twiddle table from the shared exponent formula
  const int len = PI::tw_len();
  std::vector<float2> tw(len);
  for (int e = 0; e < len && PI::n > 1; ++e) {
    const double ang = 2.0 * M_PI * (double)pass_twiddle_exponent(e, M, PI::r0, PI::r1, PI::r2) / M;
    tw[e] = make_float2((float)std::cos(ang), (float)-std::sin(ang));
  }
  std::vector<float2> sm(PI::stride(1) + 16);
  std::vector<float2> out(M, make_float2(NAN, NAN));
  std::vector<std::vector<float2>> v(T, std::vector<float2>(E));
  auto src = [&](int c, int i) -> float2 { (void)c; return x[i]; };
  auto dst = [&](int c, int f, float2 val) { (void)c; out[f] = val; };
  for (int t = 0; t < T; ++t) F::pass0_load(0, t, src, v[t].data());
  if constexpr (PI::n == 1) {
    for (int t = 0; t < T; ++t) F::template pass_out<0>(0, t, dst, v[t].data());
  } else {
    for (int t = 0; t < T; ++t) F::pass0_store(t, sm.data(), v[t].data());
    for (int t = 0; t < T; ++t) F::template pass_load<1>(t, sm.data(), tw.data(), v[t].data());
    if constexpr (PI::n == 2) {
      for (int t = 0; t < T; ++t) F::template pass_out<1>(0, t, dst, v[t].data());
    } else {
      for (int t = 0; t < T; ++t) F::template pass_store<1>(t, sm.data(), v[t].data());
      for (int t = 0; t < T; ++t) F::template pass_load<2>(t, sm.data(), tw.data(), v[t].data());
      for (int t = 0; t < T; ++t) F::template pass_out<2>(0, t, dst, v[t].data());
    }
  }
  double err = 0, mx = 0;
  for (int f = 0; f < M; ++f) {
    std::complex<double> acc = 0;
    for (int n = 0; n < M; ++n) {
      const double ang = -2.0 * M_PI * (double)(((long long)f * n) % M) / M;
      acc += std::complex<double>(x[n].x, x[n].y) * std::complex<double>(std::cos(ang), std::sin(ang));
    }
    const std::complex<double> got(out[f].x, out[f].y);
    err = std::max(err, std::abs(got - acc));
    mx = std::max(mx, std::abs(acc));
  }
  return err / mx;
}

int main() {
  std::mt19937_64 g(1234);
#define RUN(M) std::printf("%d %.3e\n", M, check_size<M>(g));
  RUN(2) RUN(4) RUN(8) RUN(16) RUN(32) RUN(64) RUN(128) RUN(256) RUN(512) RUN(1024) RUN(2048) RUN(4096)
  RUN(8192) RUN(16384)
  return 0;
}
