// Register-resident DST-I of the W = 32 columns of a float32 tile, 256
// threads (8 warps) per tile (Sections 5.2-5.3: the box solve is a sine
// transform along each axis).
//
// The DST-I of length N-1 is computed as in the shared-memory Stockham path:
// sine pre-fold into a real sequence y of length N, complex FFT of length
// L = N/2 on z_m = y_{2m} + i y_{2m+1}, real-DFT split, prefix sum for the
// odd outputs.  Here the FFT is one two-level decomposition m = a + 8q,
// k = k1 + P k2 (P = L/8): thread (a = warp, c = lane = column) pre-folds its
// P points straight from the tile, does a radix-P DFT over q in registers and
// the twiddle w_L^{a k1}; after one exchange through shared memory, the
// thread that owns the column-pair group {k1, P - k1} does the radix-8 DFTs
// over a, so both halves of every split pair Z_k, Z_{L-k} sit in its
// registers and the split needs no further exchange.  A segmented scan (one
// P-long segment per warp) finishes the odd outputs.  Every shared-memory
// access of a warp touches one row of 32 consecutive columns (or 32
// consecutive float2 of the exchange buffer), so none has bank conflicts.
//
// The phases are plain functions of (a, c) and per-thread state so that the
// same source runs on the host, one simulated thread at a time, to check the
// index arithmetic against a library DST.
#pragma once

#ifdef __CUDACC__
#define KFBI_HD __host__ __device__ __forceinline__
#else
#define KFBI_HD inline
#endif

namespace kfbi {
namespace regdst {

struct cf2 {
  float x, y;
};

// b_p = sum_q a_q e^{+2 pi i p q / R}, in place
template <int R>
struct Dft;

template <>
struct Dft<1> {
  static KFBI_HD void run(float*, float*) {}
};

template <>
struct Dft<2> {
  static KFBI_HD void run(float* xr, float* xi) {
    const float ar = xr[0] + xr[1], ai = xi[0] + xi[1];
    xr[1] = xr[0] - xr[1];
    xi[1] = xi[0] - xi[1];
    xr[0] = ar;
    xi[0] = ai;
  }
};

// b_p = sum_q a_q e^{+2 pi i p q / 3}
template <>
struct Dft<3> {
  static KFBI_HD void run(float* xr, float* xi) {
    const float s3 = 0.86602540378443864676f;
    const float tr = xr[1] + xr[2], ti = xi[1] + xi[2];
    const float ur = xr[1] - xr[2], ui = xi[1] - xi[2];
    const float mr = xr[0] - 0.5f * tr, mi = xi[0] - 0.5f * ti;
    xr[0] += tr;
    xi[0] += ti;
    xr[1] = mr - s3 * ui;  // m + i s3 u
    xi[1] = mi + s3 * ur;
    xr[2] = mr + s3 * ui;  // m - i s3 u
    xi[2] = mi - s3 * ur;
  }
};

template <>
struct Dft<4> {
  static KFBI_HD void run(float* xr, float* xi) {
    const float t0r = xr[0] + xr[2], t0i = xi[0] + xi[2];
    const float t1r = xr[0] - xr[2], t1i = xi[0] - xi[2];
    const float t2r = xr[1] + xr[3], t2i = xi[1] + xi[3];
    const float t3r = xr[1] - xr[3], t3i = xi[1] - xi[3];
    xr[0] = t0r + t2r;
    xi[0] = t0i + t2i;
    xr[2] = t0r - t2r;
    xi[2] = t0i - t2i;
    xr[1] = t1r - t3i;  // t1 + i t3
    xi[1] = t1i + t3r;
    xr[3] = t1r + t3i;  // t1 - i t3
    xi[3] = t1i - t3r;
  }
};

template <>
struct Dft<8> {
  static KFBI_HD void run(float* xr, float* xi) {
    float er[4] = {xr[0], xr[2], xr[4], xr[6]}, ei[4] = {xi[0], xi[2], xi[4], xi[6]};
    float orr[4] = {xr[1], xr[3], xr[5], xr[7]}, oi[4] = {xi[1], xi[3], xi[5], xi[7]};
    Dft<4>::run(er, ei);
    Dft<4>::run(orr, oi);
    const float c = 0.70710678118654752440f;
    const float w1r = c * (orr[1] - oi[1]), w1i = c * (orr[1] + oi[1]);  // e^{i pi/4} O_1
    const float w2r = -oi[2], w2i = orr[2];                               // i O_2
    const float w3r = -c * (orr[3] + oi[3]), w3i = c * (orr[3] - oi[3]);  // e^{3 i pi/4} O_3
    xr[0] = er[0] + orr[0];
    xi[0] = ei[0] + oi[0];
    xr[4] = er[0] - orr[0];
    xi[4] = ei[0] - oi[0];
    xr[1] = er[1] + w1r;
    xi[1] = ei[1] + w1i;
    xr[5] = er[1] - w1r;
    xi[5] = ei[1] - w1i;
    xr[2] = er[2] + w2r;
    xi[2] = ei[2] + w2i;
    xr[6] = er[2] - w2r;
    xi[6] = ei[2] - w2i;
    xr[3] = er[3] + w3r;
    xi[3] = ei[3] + w3i;
    xr[7] = er[3] - w3r;
    xi[7] = ei[3] - w3i;
  }
};

// 16 = 4 x 4: q = 4 q1 + q2, p = p1 + 4 p2; radix 4 over q1, twiddle
// e^{2 pi i p1 q2 / 16}, radix 4 over q2
template <>
struct Dft<16> {
  static KFBI_HD void run(float* xr, float* xi) {
    // cos(pi k / 8), k = 0..15
    const float C8[16] = {1.0f,
                          0.92387953251128675613f,
                          0.70710678118654752440f,
                          0.38268343236508977173f,
                          0.0f,
                          -0.38268343236508977173f,
                          -0.70710678118654752440f,
                          -0.92387953251128675613f,
                          -1.0f,
                          -0.92387953251128675613f,
                          -0.70710678118654752440f,
                          -0.38268343236508977173f,
                          0.0f,
                          0.38268343236508977173f,
                          0.70710678118654752440f,
                          0.92387953251128675613f};
#pragma unroll
    for (int q2 = 0; q2 < 4; ++q2) {
      float tr[4] = {xr[q2], xr[q2 + 4], xr[q2 + 8], xr[q2 + 12]};
      float ti[4] = {xi[q2], xi[q2 + 4], xi[q2 + 8], xi[q2 + 12]};
      Dft<4>::run(tr, ti);
#pragma unroll
      for (int p1 = 0; p1 < 4; ++p1) {
        const int e = (p1 * q2) & 15;
        const float wr = C8[e], wi = C8[(e + 12) & 15];  // sin(pi e / 8) = cos(pi (e - 4) / 8)
        xr[q2 + 4 * p1] = tr[p1] * wr - ti[p1] * wi;
        xi[q2 + 4 * p1] = tr[p1] * wi + ti[p1] * wr;
      }
    }
    float outr[16], outi[16];
#pragma unroll
    for (int p1 = 0; p1 < 4; ++p1) {
      float tr[4] = {xr[4 * p1], xr[4 * p1 + 1], xr[4 * p1 + 2], xr[4 * p1 + 3]};
      float ti[4] = {xi[4 * p1], xi[4 * p1 + 1], xi[4 * p1 + 2], xi[4 * p1 + 3]};
      Dft<4>::run(tr, ti);
#pragma unroll
      for (int p2 = 0; p2 < 4; ++p2) {
        outr[p1 + 4 * p2] = tr[p2];
        outi[p1 + 4 * p2] = ti[p2];
      }
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      xr[i] = outr[i];
      xi[i] = outi[i];
    }
  }
};

// P = R1 R2 with twiddles from the shared table tw2 (tw2[j] = e^{i pi j/N},
// so e^{2 pi i e / P} = tw2[e * 2N/P]): q = R2 q1 + q2, p = p1 + R1 p2;
// radix R1 over q1, twiddle e^{2 pi i p1 q2 / P}, radix R2 over q2
template <int R1, int R2>
struct DftT {
  static KFBI_HD void run(float* xr, float* xi, const cf2* tw2, int jstep) {
    constexpr int P = R1 * R2;
#pragma unroll
    for (int q2 = 0; q2 < R2; ++q2) {
      float tr[R1], ti[R1];
#pragma unroll
      for (int q1 = 0; q1 < R1; ++q1) {
        tr[q1] = xr[q2 + R2 * q1];
        ti[q1] = xi[q2 + R2 * q1];
      }
      Dft<R1>::run(tr, ti);
#pragma unroll
      for (int p1 = 0; p1 < R1; ++p1) {
        const int e = (p1 * q2) % P;
        if (e == 0) {
          xr[q2 + R2 * p1] = tr[p1];
          xi[q2 + R2 * p1] = ti[p1];
        } else {
          const cf2 w = tw2[e * jstep];
          xr[q2 + R2 * p1] = tr[p1] * w.x - ti[p1] * w.y;
          xi[q2 + R2 * p1] = tr[p1] * w.y + ti[p1] * w.x;
        }
      }
    }
    float outr[P], outi[P];
#pragma unroll
    for (int p1 = 0; p1 < R1; ++p1) {
      Dft<R2>::run(xr + R2 * p1, xi + R2 * p1);
#pragma unroll
      for (int p2 = 0; p2 < R2; ++p2) {
        outr[p1 + R1 * p2] = xr[R2 * p1 + p2];
        outi[p1 + R1 * p2] = xi[R2 * p1 + p2];
      }
    }
#pragma unroll
    for (int i = 0; i < P; ++i) {
      xr[i] = outr[i];
      xi[i] = outi[i];
    }
  }
};

// the first-level DFT of length P (P = 2, 4, 8, 16 with constant twiddles;
// 24 = 3 x 8 and 32 = 4 x 8 with the shared table)
template <int P, int N>
KFBI_HD void dft_first(float* xr, float* xi, const cf2* tw2) {
  if constexpr (P == 24) {
    DftT<3, 8>::run(xr, xi, tw2, 2 * N / P);
  } else if constexpr (P == 32) {
    DftT<4, 8>::run(xr, xi, tw2, 2 * N / P);
  } else {
    Dft<P>::run(xr, xi);
  }
}

// Tile geometry: N rows (transform index), W = 32 columns, row stride RS;
// 8 warps, P points per thread in the first level.
template <int N_, int RS_>
struct Geo {
  static constexpr int N = N_, RS = RS_, W = 32, T = 8;
  static constexpr int L = N / 2;
  static constexpr int P = L / T;
  static constexpr int NG = P / 2 > 0 ? P / 2 : 1;  // split-pair groups of k1
  static constexpr int GPT = (NG + T - 1) / T;      // groups per thread
  static_assert(N >= 32 && L % T == 0, "tile too short for the register DST");
};

// shared tables: sinv[j] = sin(pi j / N) (j < N), tw2[j] = e^{i pi j / N} (j < 2N)
template <class G>
struct State {
  float zr[G::P], zi[G::P];            // first level
  float Ar[G::GPT][8], Ai[G::GPT][8];  // second level, k1 = first of the group
  float Br[G::GPT][8], Bi[G::GPT][8];  // second level, k1 = second of the group
  float v[G::P];                       // scan segment
};

// phase A1: pre-fold, radix-P DFT over q, twiddle (reads the tile)
template <class G>
KFBI_HD void phase_a1(State<G>& st, const float* s, const float* sinv, const cf2* tw2, int a, int c) {
  constexpr int N = G::N, RS = G::RS, T = G::T, P = G::P;
#pragma unroll
  for (int q = 0; q < P; ++q) {
    const int m = a + T * q, j = 2 * m;
    const float x0 = s[j * RS + c], x1 = s[(j + 1) * RS + c];
    const float r0 = m > 0 ? s[(N - j) * RS + c] : 0.0f, r1 = s[(N - j - 1) * RS + c];
    const cf2 sn = reinterpret_cast<const cf2*>(sinv)[m];  // sin(pi j/N), sin(pi (j+1)/N)
    st.zr[q] = m > 0 ? sn.x * (x0 + r0) + 0.5f * (x0 - r0) : 0.0f;
    st.zi[q] = sn.y * (x1 + r1) + 0.5f * (x1 - r1);
  }
  dft_first<P, N>(st.zr, st.zi, tw2);
#pragma unroll
  for (int k1 = 1; k1 < P; ++k1) {
    const cf2 w = tw2[4 * a * k1];  // e^{2 pi i a k1 / L}
    const float t = st.zr[k1] * w.x - st.zi[k1] * w.y;
    st.zi[k1] = st.zr[k1] * w.y + st.zi[k1] * w.x;
    st.zr[k1] = t;
  }
}

// phase A2: first-level results to the exchange buffer (after a barrier)
template <class G>
KFBI_HD void phase_a2(const State<G>& st, cf2* ex, int a, int c) {
  constexpr int T = G::T, P = G::P, W = G::W;
#pragma unroll
  for (int k1 = 0; k1 < P; ++k1) ex[(k1 * T + a) * W + c] = cf2{st.zr[k1], st.zi[k1]};
}

template <class G>
KFBI_HD void group_k1(int g, int& kA, int& kB) {
  kA = g == 0 ? 0 : g;
  kB = g == 0 ? G::P / 2 : G::P - g;
}

// phase C: radix-8 DFTs over a for the thread's k1 groups (reads the exchange)
template <class G>
KFBI_HD void phase_c(State<G>& st, const cf2* ex, int a, int c) {
  constexpr int T = G::T, W = G::W;
#pragma unroll
  for (int gi = 0; gi < G::GPT; ++gi) {
    const int g = a + T * gi;
    if (g >= G::NG) continue;
    int kA, kB;
    group_k1<G>(g, kA, kB);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const cf2 pa = ex[(kA * T + u) * W + c];
      st.Ar[gi][u] = pa.x;
      st.Ai[gi][u] = pa.y;
      if (G::P > 1) {
        const cf2 pb = ex[(kB * T + u) * W + c];
        st.Br[gi][u] = pb.x;
        st.Bi[gi][u] = pb.y;
      }
    }
    Dft<8>::run(st.Ar[gi], st.Ai[gi]);
    Dft<8>::run(st.Br[gi], st.Bi[gi]);
  }
}

// Y_k from A = Z_k, B = Z_{L-k}, w = e^{2 pi i k/N}: I_k to row 2k (even
// output), R_k to row 2k+1 (scan input); post(j, value) maps an even output
template <class G, class Post>
KFBI_HD void split_store(float* s, const cf2* tw2, int k, float Ar, float Ai, float Br, float Bi, int c,
                         const Post& post) {
  constexpr int RS = G::RS;
  const cf2 w = tw2[2 * k];
  const float Sr = Ar + Br, Si = Ai - Bi, Dr = Ar - Br, Di = Ai + Bi;
  const float Yr = 0.5f * (Sr + w.x * Di + w.y * Dr);
  const float Yi = 0.5f * (Si - w.x * Dr + w.y * Di);
  s[(2 * k) * RS + c] = post(2 * k, Yi);
  s[(2 * k + 1) * RS + c] = Yr;
}

// phase D: real-DFT split of the owned pairs (after a barrier), writes rows
template <class G, class Post>
KFBI_HD void phase_d(const State<G>& st, float* s, const cf2* tw2, int a, int c, const Post& post) {
  constexpr int T = G::T, P = G::P, L = G::L, RS = G::RS;
#pragma unroll
  for (int gi = 0; gi < G::GPT; ++gi) {
    const int g = a + T * gi;
    if (g >= G::NG) continue;
    int kA, kB;
    group_k1<G>(g, kA, kB);
    if (g == 0) {
      // k1 = 0: k = P k2 pairs with P (8 - k2); k = 0 and k = L/2 pair with themselves
      s[c] = 0.0f;
      s[RS + c] = 0.5f * (st.Ar[gi][0] + st.Ai[gi][0]);
#pragma unroll
      for (int k2 = 1; k2 <= 4; ++k2) {
        const int k = P * k2, kk = L - k;
        split_store<G>(s, tw2, k, st.Ar[gi][k2], st.Ai[gi][k2], st.Ar[gi][(8 - k2) & 7], st.Ai[gi][(8 - k2) & 7], c,
                       post);
        if (kk != k)
          split_store<G>(s, tw2, kk, st.Ar[gi][(8 - k2) & 7], st.Ai[gi][(8 - k2) & 7], st.Ar[gi][k2], st.Ai[gi][k2],
                         c, post);
      }
      // k1 = P/2: k = P/2 + P k2 pairs with P/2 + P (7 - k2)
      if (P > 1) {
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) {
          const int k = kB + P * k2, kk = L - k;
          split_store<G>(s, tw2, k, st.Br[gi][k2], st.Bi[gi][k2], st.Br[gi][7 - k2], st.Bi[gi][7 - k2], c, post);
          split_store<G>(s, tw2, kk, st.Br[gi][7 - k2], st.Bi[gi][7 - k2], st.Br[gi][k2], st.Bi[gi][k2], c, post);
        }
      }
    } else {
      // k = kA + P k2 pairs with kB + P (7 - k2)
#pragma unroll
      for (int k2 = 0; k2 < 8; ++k2) {
        const int k = kA + P * k2;
        split_store<G>(s, tw2, k, st.Ar[gi][k2], st.Ai[gi][k2], st.Br[gi][7 - k2], st.Bi[gi][7 - k2], c, post);
        const int kk = kB + P * k2;
        split_store<G>(s, tw2, kk, st.Br[gi][k2], st.Bi[gi][k2], st.Ar[gi][7 - k2], st.Ai[gi][7 - k2], c, post);
      }
    }
  }
}

// phase E1: local inclusive scan of the warp's segment of R_k (rows 2k+1)
template <class G>
KFBI_HD void phase_e1(State<G>& st, const float* s, float* tot, int a, int c) {
  constexpr int P = G::P, RS = G::RS, W = G::W;
  float acc = 0.0f;
#pragma unroll
  for (int i = 0; i < P; ++i) {
    acc += s[(2 * (a * P + i) + 1) * RS + c];
    st.v[i] = acc;
  }
  tot[a * W + c] = acc;
}

// phase E2: add the preceding segments' totals, write the odd outputs
template <class G, class Post>
KFBI_HD void phase_e2(const State<G>& st, float* s, const float* tot, int a, int c, const Post& post) {
  constexpr int P = G::P, RS = G::RS, W = G::W;
  float off = 0.0f;
  for (int b = 0; b < a; ++b) off += tot[b * W + c];
#pragma unroll
  for (int i = 0; i < P; ++i) {
    const int j = 2 * (a * P + i) + 1;
    s[j * RS + c] = post(j, st.v[i] + off);
  }
}

struct Identity {
  KFBI_HD float operator()(int, float v) const { return v; }
};

// ---- cosine transform (DCT-I of the N + 1 rows 0..N, the Neumann box) ----
// X_p = sum_k c_k x_k cos(pi k p / N), c_0 = c_N = 1/2.  The same two-level
// FFT after the cosine pre-fold
//   y_j = (x_j + x_{N-j}) / 2 - sin(pi j / N)(x_j - x_{N-j})   (y_0 = (x_0 + x_N) / 2),
// then X_{2k} = Re Y_k (X_0 and X_N from Z_0) and the odd outputs by the scan
// X_{2k+1} = X_{2k-1} + Im Y_k (2 sin a sin b = cos(a - b) - cos(a + b)),
// started at X_1 = sum_k c_k x_k cos(pi k / N), whose terms phase A1 sums
// while it reads the rows (each thread its rows 2m, 2m + 1; warp 0 row N).

// phase A1 (cosine): pre-fold, partial X_1 to part[a][c], radix-P DFT, twiddle
template <class G>
KFBI_HD void phase_a1_cos(State<G>& st, const float* s, const float* sinv, const cf2* tw2, float* part, int a,
                          int c) {
  constexpr int N = G::N, RS = G::RS, T = G::T, P = G::P, W = G::W;
  float x1 = 0.0f;
#pragma unroll
  for (int q = 0; q < P; ++q) {
    const int m = a + T * q, j = 2 * m;
    const float x0 = s[j * RS + c], xa = s[(j + 1) * RS + c];
    const float r0 = s[(N - j) * RS + c], r1 = s[(N - j - 1) * RS + c];
    const cf2 sn = reinterpret_cast<const cf2*>(sinv)[m];  // sin(pi j/N), sin(pi (j+1)/N)
    st.zr[q] = 0.5f * (x0 + r0) - sn.x * (x0 - r0);
    st.zi[q] = 0.5f * (xa + r1) - sn.y * (xa - r1);
    x1 += (m > 0 ? tw2[j].x : 0.5f) * x0 + tw2[j + 1].x * xa;
  }
  if (a == 0) x1 -= 0.5f * s[N * RS + c];
  part[a * W + c] = x1;
  dft_first<P, N>(st.zr, st.zi, tw2);
#pragma unroll
  for (int k1 = 1; k1 < P; ++k1) {
    const cf2 w = tw2[4 * a * k1];
    const float t = st.zr[k1] * w.x - st.zi[k1] * w.y;
    st.zi[k1] = st.zr[k1] * w.y + st.zi[k1] * w.x;
    st.zr[k1] = t;
  }
}

// X_1 of every column from the partial sums (warp 0; after a barrier)
template <class G>
KFBI_HD void phase_x1(const float* part, float* x1v, int a, int c) {
  if (a != 0) return;
  float v = 0.0f;
  for (int b = 0; b < G::T; ++b) v += part[b * G::W + c];
  x1v[c] = v;
}

// Y_k from A = Z_k, B = Z_{L-k}: Re Y_k = X_{2k} to row 2k, Im Y_k (scan
// input) to row 2k+1
template <class G, class Post>
KFBI_HD void split_store_cos(float* s, const cf2* tw2, int k, float Ar, float Ai, float Br, float Bi, int c,
                             const Post& post) {
  constexpr int RS = G::RS;
  const cf2 w = tw2[2 * k];
  const float Sr = Ar + Br, Si = Ai - Bi, Dr = Ar - Br, Di = Ai + Bi;
  const float Yr = 0.5f * (Sr + w.x * Di + w.y * Dr);
  const float Yi = 0.5f * (Si - w.x * Dr + w.y * Di);
  s[(2 * k) * RS + c] = post(2 * k, Yr);
  s[(2 * k + 1) * RS + c] = Yi;
}

// phase D (cosine): real-DFT split of the owned pairs; X_0, X_N from Z_0
template <class G, class Post>
KFBI_HD void phase_d_cos(const State<G>& st, float* s, const cf2* tw2, int a, int c, const Post& post) {
  constexpr int N = G::N, T = G::T, P = G::P, L = G::L, RS = G::RS;
#pragma unroll
  for (int gi = 0; gi < G::GPT; ++gi) {
    const int g = a + T * gi;
    if (g >= G::NG) continue;
    int kA, kB;
    group_k1<G>(g, kA, kB);
    if (g == 0) {
      s[c] = post(0, st.Ar[gi][0] + st.Ai[gi][0]);
      s[N * RS + c] = post(N, st.Ar[gi][0] - st.Ai[gi][0]);
      s[RS + c] = 0.0f;
#pragma unroll
      for (int k2 = 1; k2 <= 4; ++k2) {
        const int k = P * k2, kk = L - k;
        split_store_cos<G>(s, tw2, k, st.Ar[gi][k2], st.Ai[gi][k2], st.Ar[gi][(8 - k2) & 7],
                           st.Ai[gi][(8 - k2) & 7], c, post);
        if (kk != k)
          split_store_cos<G>(s, tw2, kk, st.Ar[gi][(8 - k2) & 7], st.Ai[gi][(8 - k2) & 7], st.Ar[gi][k2],
                             st.Ai[gi][k2], c, post);
      }
      if (P > 1) {
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) {
          const int k = kB + P * k2, kk = L - k;
          split_store_cos<G>(s, tw2, k, st.Br[gi][k2], st.Bi[gi][k2], st.Br[gi][7 - k2], st.Bi[gi][7 - k2], c,
                             post);
          split_store_cos<G>(s, tw2, kk, st.Br[gi][7 - k2], st.Bi[gi][7 - k2], st.Br[gi][k2], st.Bi[gi][k2], c,
                             post);
        }
      }
    } else {
#pragma unroll
      for (int k2 = 0; k2 < 8; ++k2) {
        const int k = kA + P * k2;
        split_store_cos<G>(s, tw2, k, st.Ar[gi][k2], st.Ai[gi][k2], st.Br[gi][7 - k2], st.Bi[gi][7 - k2], c,
                           post);
        const int kk = kB + P * k2;
        split_store_cos<G>(s, tw2, kk, st.Br[gi][k2], st.Bi[gi][k2], st.Ar[gi][7 - k2], st.Ai[gi][7 - k2], c,
                           post);
      }
    }
  }
}

// phase E2 (cosine): X_1 plus the preceding segments' totals, odd outputs
template <class G, class Post>
KFBI_HD void phase_e2_cos(const State<G>& st, float* s, const float* tot, const float* x1v, int a, int c,
                          const Post& post) {
  constexpr int P = G::P, RS = G::RS, W = G::W;
  float off = x1v[c];
  for (int b = 0; b < a; ++b) off += tot[b * W + c];
#pragma unroll
  for (int i = 0; i < P; ++i) {
    const int j = 2 * (a * P + i) + 1;
    s[j * RS + c] = post(j, st.v[i] + off);
  }
}

#ifdef __CUDACC__
// The whole transform of the tile s[N][RS] (rows 1..N-1 in and out, row 0
// holds 0) by 256 threads.  ex aliases s (N * W floats), tot holds 8 * 32
// floats.  Ends with a barrier.
template <class G, class Post = Identity>
__device__ __forceinline__ void dst1_tile_reg(float* s, const float* sinv, const cf2* tw2, float* tot,
                                              const Post& post = Post()) {
  const int a = threadIdx.x >> 5, c = threadIdx.x & 31;
  State<G> st;
  cf2* ex = reinterpret_cast<cf2*>(s);
  phase_a1<G>(st, s, sinv, tw2, a, c);
  __syncthreads();
  phase_a2<G>(st, ex, a, c);
  __syncthreads();
  phase_c<G>(st, ex, a, c);
  __syncthreads();
  phase_d<G>(st, s, tw2, a, c, post);
  __syncthreads();
  phase_e1<G>(st, s, tot, a, c);
  __syncthreads();
  phase_e2<G>(st, s, tot, a, c, post);
  __syncthreads();
}

// The cosine transform of the tile s[N + 1][RS] (rows 0..N in and out) by
// 256 threads; ex aliases rows 0..N-1, tot holds 8 * 32 floats, x1v 32.
template <class G, class Post = Identity>
__device__ __forceinline__ void dct1_tile_reg(float* s, const float* sinv, const cf2* tw2, float* tot, float* x1v,
                                              const Post& post = Post()) {
  const int a = threadIdx.x >> 5, c = threadIdx.x & 31;
  State<G> st;
  cf2* ex = reinterpret_cast<cf2*>(s);
  phase_a1_cos<G>(st, s, sinv, tw2, tot, a, c);
  __syncthreads();
  phase_a2<G>(st, ex, a, c);
  __syncthreads();
  phase_x1<G>(tot, x1v, a, c);
  phase_c<G>(st, ex, a, c);
  __syncthreads();
  phase_d_cos<G>(st, s, tw2, a, c, post);
  __syncthreads();
  phase_e1<G>(st, s, tot, a, c);
  __syncthreads();
  phase_e2_cos<G>(st, s, tot, x1v, a, c, post);
  __syncthreads();
}
#endif

}  // namespace regdst
}  // namespace kfbi
