// Host run of the register DST / DCT phases (one simulated thread at a
// time, a barrier between phases) for checking their index arithmetic on the
// CPU.  stdin: N RS KIND (0 sine, 1 cosine), then 32 columns of N-1 (sine)
// or N+1 (cosine) values; stdout: the 32 transformed columns.
#include <cmath>
#include <cstdio>
#include <vector>

#include "dst_reg.cuh"

using namespace kfbi::regdst;

template <int N, int RS>
int run(int kind) {
  using G = Geo<N, RS>;
  const double pi = 3.14159265358979323846;
  std::vector<float> s((size_t)(N + 1) * RS, 0.0f), tot(256, 0.0f), sinv(N), x1v(32, 0.0f);
  std::vector<cf2> tw2(2 * N);
  for (int j = 0; j < 2 * N; ++j) tw2[j] = cf2{(float)std::cos(pi * j / N), (float)std::sin(pi * j / N)};
  for (int j = 0; j < N; ++j) sinv[j] = (float)std::sin(pi * j / N);
  const int j0 = kind == 0 ? 1 : 0, j1 = kind == 0 ? N - 1 : N;
  for (int c = 0; c < 32; ++c)
    for (int j = j0; j <= j1; ++j) {
      double v;
      if (std::scanf("%lf", &v) != 1) return 1;
      s[(size_t)j * RS + c] = (float)v;
    }
  std::vector<State<G>> st(256);
  cf2* ex = reinterpret_cast<cf2*>(s.data());
  if (kind == 0) {
    for (int t = 0; t < 256; ++t) phase_a1<G>(st[t], s.data(), sinv.data(), tw2.data(), t >> 5, t & 31);
  } else {
    for (int t = 0; t < 256; ++t) phase_a1_cos<G>(st[t], s.data(), sinv.data(), tw2.data(), tot.data(), t >> 5, t & 31);
  }
  for (int t = 0; t < 256; ++t) phase_a2<G>(st[t], ex, t >> 5, t & 31);
  if (kind == 1)
    for (int t = 0; t < 256; ++t) phase_x1<G>(tot.data(), x1v.data(), t >> 5, t & 31);
  for (int t = 0; t < 256; ++t) phase_c<G>(st[t], ex, t >> 5, t & 31);
  if (kind == 0) {
    for (int t = 0; t < 256; ++t) phase_d<G>(st[t], s.data(), tw2.data(), t >> 5, t & 31, Identity());
  } else {
    for (int t = 0; t < 256; ++t) phase_d_cos<G>(st[t], s.data(), tw2.data(), t >> 5, t & 31, Identity());
  }
  for (int t = 0; t < 256; ++t) phase_e1<G>(st[t], s.data(), tot.data(), t >> 5, t & 31);
  if (kind == 0) {
    for (int t = 0; t < 256; ++t) phase_e2<G>(st[t], s.data(), tot.data(), t >> 5, t & 31, Identity());
  } else {
    for (int t = 0; t < 256; ++t)
      phase_e2_cos<G>(st[t], s.data(), tot.data(), x1v.data(), t >> 5, t & 31, Identity());
  }
  for (int c = 0; c < 32; ++c) {
    for (int j = j0; j <= j1; ++j) std::printf("%.9g ", s[(size_t)j * RS + c]);
    std::printf("\n");
  }
  return 0;
}

int main() {
  int N, RS, kind;
  if (std::scanf("%d %d %d", &N, &RS, &kind) != 3) return 1;
  const bool pad = RS != 32;
  switch (N) {
    case 32: return pad ? run<32, 33>(kind) : run<32, 32>(kind);
    case 64: return pad ? run<64, 33>(kind) : run<64, 32>(kind);
    case 128: return pad ? run<128, 33>(kind) : run<128, 32>(kind);
    case 256: return pad ? run<256, 33>(kind) : run<256, 32>(kind);
    case 384: return pad ? run<384, 33>(kind) : run<384, 32>(kind);
    case 512: return pad ? run<512, 33>(kind) : run<512, 32>(kind);
    default: return 2;
  }
}
