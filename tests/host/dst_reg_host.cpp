// Host run of the register DST phases (one simulated thread at a time, a
// barrier between phases) for checking their index arithmetic on the CPU.
// stdin: N RS, then 32 columns of N-1 values; stdout: the 32 transformed
// columns.
#include <cmath>
#include <cstdio>
#include <vector>

#include "dst_reg.cuh"

using namespace kfbi::regdst;

template <int N, int RS>
int run() {
  using G = Geo<N, RS>;
  const double pi = 3.14159265358979323846;
  std::vector<float> s((size_t)N * RS, 0.0f), tot(256, 0.0f), sinv(N);
  std::vector<cf2> tw2(2 * N);
  for (int j = 0; j < 2 * N; ++j) tw2[j] = cf2{(float)std::cos(pi * j / N), (float)std::sin(pi * j / N)};
  for (int j = 0; j < N; ++j) sinv[j] = (float)std::sin(pi * j / N);
  for (int c = 0; c < 32; ++c)
    for (int j = 1; j < N; ++j) {
      double v;
      if (std::scanf("%lf", &v) != 1) return 1;
      s[(size_t)j * RS + c] = (float)v;
    }
  std::vector<State<G>> st(256);
  cf2* ex = reinterpret_cast<cf2*>(s.data());
  for (int t = 0; t < 256; ++t) phase_a1<G>(st[t], s.data(), sinv.data(), tw2.data(), t >> 5, t & 31);
  for (int t = 0; t < 256; ++t) phase_a2<G>(st[t], ex, t >> 5, t & 31);
  for (int t = 0; t < 256; ++t) phase_c<G>(st[t], ex, t >> 5, t & 31);
  for (int t = 0; t < 256; ++t) phase_d<G>(st[t], s.data(), tw2.data(), t >> 5, t & 31, Identity());
  for (int t = 0; t < 256; ++t) phase_e1<G>(st[t], s.data(), tot.data(), t >> 5, t & 31);
  for (int t = 0; t < 256; ++t) phase_e2<G>(st[t], s.data(), tot.data(), t >> 5, t & 31, Identity());
  for (int c = 0; c < 32; ++c) {
    for (int j = 1; j < N; ++j) std::printf("%.9g ", s[(size_t)j * RS + c]);
    std::printf("\n");
  }
  return 0;
}

int main() {
  int N, RS;
  if (std::scanf("%d %d", &N, &RS) != 2) return 1;
  const bool pad = RS != 32;
  switch (N) {
    case 32: return pad ? run<32, 33>() : run<32, 32>();
    case 64: return pad ? run<64, 33>() : run<64, 32>();
    case 128: return pad ? run<128, 33>() : run<128, 32>();
    case 256: return pad ? run<256, 33>() : run<256, 32>();
    case 384: return pad ? run<384, 33>() : run<384, 32>();
    case 512: return pad ? run<512, 33>() : run<512, 32>();
    default: return 2;
  }
}
