// Box solver of the corrected 5/7-point system by sine transforms
// (Sections 5.2-5.3: the correction leaves the symmetric definite matrix
// unchanged, so an FFT-based fast Poisson/Helmholtz solver applies).
//
//   v = (2/N)^d S( mu^{-1} o S r ),   S_{kp} = sin(pi k p / N),  k, p = 1..N-1,
//   mu_p = sum_a mu1[p_a] - lambda,  mu1[p] = -(4/h^2) sin^2(pi p / (2N)).
//
// Work arrays are padded to N^d with index 0 of every axis holding the zero
// Dirichlet value, so every line of the DST-I of length N-1 is a length-N row
// starting at an aligned address.  Each 1-D DST-I of length N-1 runs in shared
// memory as: sine pre-fold into a real sequence of length N, complex Stockham
// FFT of length N/2 (radix 8/4/2/3 butterflies in registers), split into the
// real DFT, and a prefix sum for the odd outputs.  A block owns a tile of W
// independent lines laid out [transform index][line] so that every butterfly
// stage is vectorised across the lines (consecutive threads touch consecutive
// words).  Passes:
//   x forward  : assembles r = alpha*src + corrections (irregular nodes) while
//                loading, transforms along x;
//   y forward  : strided rows, coalesced W-wide segments;
//   z solve    : forward DST, spectral divide, inverse DST in one pass;
//   y forward  : (the DST-I is its own inverse up to the folded scale);
//   x inverse  : transforms along x and writes the padded grid and/or a user
//                layout output  beta*v + gamma*aux.
// In 2-D the middle pass is the y solve.
#include <cuda_runtime.h>

#include <cudaTypedefs.h>

#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>

#include "dst_reg.cuh"
#include "ffloat.cuh"
#include "internal.cuh"

namespace kfbi {
namespace {

constexpr int NT = 256;

// float64 <-> T for float T on the bit patterns (a float64 conversion
// instruction costs as much as a float64 add here); identities for double
template <typename T>
__device__ __forceinline__ T to_T(double x) {
  if constexpr (sizeof(T) == 4)
    return ffl::narrow(x);
  else
    return x;
}
template <typename T>
__device__ __forceinline__ double to_double(T v) {
  if constexpr (sizeof(T) == 4)
    return ffl::widen(v);
  else
    return v;
}

// Tile geometry: N transform rows by W independent lines, row stride RS
// (W + 1 pads against bank conflicts of transposed loads; W for dense TMA
// tiles), G threads per line in the scan.
template <typename T_, int N_, int W_, int RS_>
struct Tile {
  using T = T_;
  static constexpr int N = N_, W = W_, RS = RS_;
  static constexpr int L = N / 2;
  static constexpr int G = NT / W;
  // tile, scan totals, twiddles e^{i pi j/N} (2N complex), sines (register path)
  static constexpr size_t smem_elems = (size_t)N * RS + (size_t)G * W + 4 * N + N;
};

template <typename T, int N>
struct WSel {
  static constexpr int W = sizeof(T) == 8 ? (N >= 384 ? 16 : (N < 32 ? N : 32)) : (N < 32 ? N : 32);
};

template <typename T, int N>
struct Cfg : Tile<T, N, WSel<T, N>::W, WSel<T, N>::W + 1> {};

__host__ __device__ constexpr int pick_radix(int L) {
  return (L % 8 == 0) ? 8 : (L % 4 == 0) ? 4 : (L % 2 == 0) ? 2 : (L % 3 == 0) ? 3 : 0;
}

// ---------------------------------------------------------------- butterflies
template <typename T, int R>
struct Dft;

template <typename T>
struct Dft<T, 2> {
  static __device__ __forceinline__ void run(T* xr, T* xi) {
    T ar = xr[0] + xr[1], ai = xi[0] + xi[1];
    xr[1] = xr[0] - xr[1];
    xi[1] = xi[0] - xi[1];
    xr[0] = ar;
    xi[0] = ai;
  }
};

// b_p = sum_q a_q e^{+2 pi i p q / 4}
template <typename T>
struct Dft<T, 4> {
  static __device__ __forceinline__ void run(T* xr, T* xi) {
    T t0r = xr[0] + xr[2], t0i = xi[0] + xi[2];
    T t1r = xr[0] - xr[2], t1i = xi[0] - xi[2];
    T t2r = xr[1] + xr[3], t2i = xi[1] + xi[3];
    T t3r = xr[1] - xr[3], t3i = xi[1] - xi[3];
    xr[0] = t0r + t2r;
    xi[0] = t0i + t2i;
    xr[2] = t0r - t2r;
    xi[2] = t0i - t2i;
    // b1 = t1 + i t3, b3 = t1 - i t3
    xr[1] = t1r - t3i;
    xi[1] = t1i + t3r;
    xr[3] = t1r + t3i;
    xi[3] = t1i - t3r;
  }
};

template <typename T>
struct Dft<T, 8> {
  static __device__ __forceinline__ void run(T* xr, T* xi) {
    T er[4] = {xr[0], xr[2], xr[4], xr[6]}, ei[4] = {xi[0], xi[2], xi[4], xi[6]};
    T orr[4] = {xr[1], xr[3], xr[5], xr[7]}, oi[4] = {xi[1], xi[3], xi[5], xi[7]};
    Dft<T, 4>::run(er, ei);
    Dft<T, 4>::run(orr, oi);
    const T c = (T)0.70710678118654752440;
    // w8^p O_p with w8 = e^{+i pi/4}
    T w1r = c * (orr[1] - oi[1]), w1i = c * (orr[1] + oi[1]);
    T w2r = -oi[2], w2i = orr[2];
    T w3r = -c * (orr[3] + oi[3]), w3i = c * (orr[3] - oi[3]);
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

template <typename T>
struct Dft<T, 3> {
  static __device__ __forceinline__ void run(T* xr, T* xi) {
    const T s3 = (T)0.86602540378443864676;
    T tr = xr[1] + xr[2], ti = xi[1] + xi[2];
    T ur = xr[1] - xr[2], ui = xi[1] - xi[2];
    T mr = xr[0] - (T)0.5 * tr, mi = xi[0] - (T)0.5 * ti;
    xr[0] = xr[0] + tr;
    xi[0] = xi[0] + ti;
    // b1 = m + i s3 u, b2 = m - i s3 u
    xr[1] = mr - s3 * ui;
    xi[1] = mi + s3 * ur;
    xr[2] = mr + s3 * ui;
    xi[2] = mi - s3 * ur;
  }
};

// One in-place Stockham stage of radix R on the complex sequence stored in
// rows (2m, 2m+1) of every column.  All reads precede all writes.  Ls is a
// compile-time constant so every index division is a shift or a constant.
template <typename C, int R, int Ls>
__device__ __forceinline__ void fft_stage(typename C::T* s, const typename C::T* tw) {
  using T = typename C::T;
  constexpr int L = C::L, W = C::W, RS = C::RS;
  constexpr int NB = (L / R) * W;
  constexpr int PER = NB > 0 ? (NB + NT - 1) / NT : 1;  // stages never taken for small L still compile
  T xr[PER][R], xi[PER][R];
#pragma unroll
  for (int b = 0; b < PER; ++b) {
    const int idx = threadIdx.x + b * NT;
    if (idx < NB) {
      const int c = idx % W, j = idx / W, k = j % Ls;
      const int tstep = (L / (R * Ls)) * k;
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int m = j + q * (L / R);
        T ar = s[(2 * m) * RS + c], ai = s[(2 * m + 1) * RS + c];
        if (q > 0) {
          const int e = 4 * ((tstep * q) % L);
          const T wr = tw[2 * e], wi = tw[2 * e + 1];
          const T t = ar * wr - ai * wi;
          ai = ar * wi + ai * wr;
          ar = t;
        }
        xr[b][q] = ar;
        xi[b][q] = ai;
      }
      Dft<T, R>::run(xr[b], xi[b]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < PER; ++b) {
    const int idx = threadIdx.x + b * NT;
    if (idx < NB) {
      const int c = idx % W, j = idx / W, k = j % Ls;
      const int base = (j - k) * R + k;
#pragma unroll
      for (int p = 0; p < R; ++p) {
        const int m = base + p * Ls;
        s[(2 * m) * RS + c] = xr[b][p];
        s[(2 * m + 1) * RS + c] = xi[b][p];
      }
    }
  }
  __syncthreads();
}

// the stage sequence of a length-Lrem transform, unrolled at compile time
template <typename C, int Ls, int Lrem>
struct Stages {
  static __device__ __forceinline__ void run(typename C::T* s, const typename C::T* tw) {
    constexpr int R = pick_radix(Lrem);
    fft_stage<C, R, Ls>(s, tw);
    Stages<C, Ls * R, Lrem / R>::run(s, tw);
  }
};
template <typename C, int Ls>
struct Stages<C, Ls, 1> {
  static __device__ __forceinline__ void run(typename C::T*, const typename C::T*) {}
};

// DST-I of every column of the tile s[N][RS] (rows 1..N-1 in, rows 1..N-1
// out, row 0 holds 0).  tw = e^{i pi j / N}, j = 0..2N-1 (interleaved re, im);
// tot = scan scratch [G][W].
template <typename C>
__device__ void dst1_tile(typename C::T* s, const typename C::T* tw, typename C::T* tot) {
  using T = typename C::T;
  constexpr int N = C::N, L = C::L, W = C::W, RS = C::RS, G = C::G;
  // sine pre-fold: y_j = sin(j pi/N)(x_j + x_{N-j}) + (x_j - x_{N-j})/2
  for (int idx = threadIdx.x; idx < (N / 2 + 1) * W; idx += NT) {
    const int c = idx % W, j = idx / W;
    if (j == 0) {
      s[c] = (T)0;
    } else if (j == N / 2) {
      s[j * RS + c] *= (T)2;
    } else {
      const T a = s[j * RS + c], b = s[(N - j) * RS + c];
      const T sj = tw[2 * j + 1];
      const T t1 = sj * (a + b), t2 = (T)0.5 * (a - b);
      s[j * RS + c] = t1 + t2;
      s[(N - j) * RS + c] = t1 - t2;
    }
  }
  __syncthreads();
  // complex FFT of length L = N/2 on z_m = y_{2m} + i y_{2m+1}
  Stages<C, 1, L>::run(s, tw);
  // real-DFT split: Y_k = (A + conj B)/2 - i w_k (A - conj B)/2, A = Z_k,
  // B = Z_{L-k}, w_k = e^{2 pi i k / N}; store I_k in row 2k, R_k in row 2k+1
  for (int idx = threadIdx.x; idx < (L / 2 + 1) * W; idx += NT) {
    const int c = idx % W, k = idx / W;
    if (k == 0) {
      const T a = s[c], b = s[RS + c];
      s[c] = (T)0;
      s[RS + c] = (T)0.5 * (a + b);  // F_1 = R_0 / 2
    } else {
      const int kk = L - k;
      const T Ar = s[(2 * k) * RS + c], Ai = s[(2 * k + 1) * RS + c];
      const T Br = s[(2 * kk) * RS + c], Bi = s[(2 * kk + 1) * RS + c];
      {
        const T wr = tw[2 * (2 * k)], wi = tw[2 * (2 * k) + 1];
        const T Sr = Ar + Br, Si = Ai - Bi, Dr = Ar - Br, Di = Ai + Bi;
        const T Yr = (T)0.5 * (Sr + wr * Di + wi * Dr);
        const T Yi = (T)0.5 * (Si - wr * Dr + wi * Di);
        s[(2 * k) * RS + c] = Yi;
        s[(2 * k + 1) * RS + c] = Yr;
      }
      if (kk != k) {
        const T wr = tw[2 * (2 * kk)], wi = tw[2 * (2 * kk) + 1];
        const T Sr = Br + Ar, Si = Bi - Ai, Dr = Br - Ar, Di = Bi + Ai;
        const T Yr = (T)0.5 * (Sr + wr * Di + wi * Dr);
        const T Yi = (T)0.5 * (Si - wr * Dr + wi * Di);
        s[(2 * kk) * RS + c] = Yi;
        s[(2 * kk + 1) * RS + c] = Yr;
      }
    }
  }
  __syncthreads();
  // odd outputs: F_{2k+1} = F_{2k-1} + R_k (column-wise inclusive scan)
  {
    constexpr int SEG = (L + G - 1) / G;
    const int c = threadIdx.x % W, g = threadIdx.x / W;
    const int k0 = g * SEG;
    const int k1 = (k0 + SEG < L) ? k0 + SEG : L;
    T acc = (T)0;
    for (int k = k0; k < k1; ++k) {
      acc += s[(2 * k + 1) * RS + c];
      s[(2 * k + 1) * RS + c] = acc;
    }
    tot[g * W + c] = acc;
    __syncthreads();
    T off = (T)0;
    for (int g2 = 0; g2 < g; ++g2) off += tot[g2 * W + c];
    for (int k = k0; k < k1; ++k) s[(2 * k + 1) * RS + c] += off;
    __syncthreads();
  }
}

template <typename T, int N>
__device__ __forceinline__ void load_twiddles(T* tw_s, const T* tw_g) {
  for (int i = threadIdx.x; i < 4 * N; i += NT) tw_s[i] = tw_g[i];
}

// Tile loads as asynchronous element copies (cp.async, 4 or 8 bytes): every
// copy of the tile is in flight at once instead of a few loads per thread,
// which is what keeps HBM busy when the grid does not fit in L2.
template <typename T>
__device__ __forceinline__ void copy_async(T* dst_smem, const T* src) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "element copies of 4 or 8 bytes");
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst_smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(src), "n"(sizeof(T)) : "memory");
}
__device__ __forceinline__ void copy_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// float32 tiles of 32 <= N <= 512 lines take the register-resident DST
template <typename T, int N>
constexpr bool kRegDst = sizeof(T) == 4 && N >= 32 && N <= 512;

// sines sin(pi j / N) for the register path's pre-fold (imaginary parts of tw)
template <typename T, int N>
__device__ __forceinline__ void load_sines(T* sinv, const T* tw_g) {
  if constexpr (kRegDst<T, N>)
    for (int i = threadIdx.x; i < N; i += NT) sinv[i] = tw_g[2 * i + 1];
}

// the DST-I of every column of the tile, rows 1..N-1 (post: map of the
// outputs, register path only)
template <typename C, class Post = regdst::Identity>
__device__ __forceinline__ void dst_tile(typename C::T* s, const typename C::T* tw, const typename C::T* sinv,
                                         typename C::T* tot, const Post& post = Post()) {
  if constexpr (kRegDst<typename C::T, C::N>) {
    regdst::dst1_tile_reg<regdst::Geo<C::N, C::RS>>(s, sinv, reinterpret_cast<const regdst::cf2*>(tw), tot, post);
  } else {
    dst1_tile<C>(s, tw, tot);
  }
}

// spectral divide v * scale / (mu1[j] + mu1[p] + mu1[q] - lambda) applied to
// the forward transform's outputs as they are written (register path)
struct DivPost {
  const float* mu;  // mu1 in shared memory
  float base;       // mu1[p] + mu1[q] - lambda
  float scale;
  bool zero;        // boundary column p = 0
  bool on = true;   // false: identity (the inverse transform of the same body)
  __device__ __forceinline__ float operator()(int j, float v) const {
    if (!on) return v;
    return zero ? 0.0f : v * __fdividef(scale, mu[j] + base);
  }
};

// ------------------------------------------------------------- x forward
// Tile: W consecutive lines y0..y0+W-1 of plane z; assembles
// r = alpha*src + corrections on the fly.
template <typename T, int N, int DIM>
__global__ void __launch_bounds__(NT) k_xfwd(T* __restrict__ a, const double* __restrict__ src, double alpha,
                                             const float* __restrict__ src32,
                                             const double* __restrict__ corr, const int32_t* __restrict__ irr,
                                             const int32_t* __restrict__ line_start, const T* __restrict__ tw_g,
                                             const int* __restrict__ skip) {
  using C = Cfg<T, N>;
  constexpr int W = C::W, RS = C::RS, n1 = N - 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  T* tot = s + N * RS;
  T* tw = tot + C::G * W;
  T* sinv = tw + 4 * N;
  load_twiddles<T, N>(tw, tw_g);
  load_sines<T, N>(sinv, tw_g);
  pdl_wait();
  if (skip != nullptr && *skip != 0) return;
  const int y0 = blockIdx.x * W;
  const int z = DIM == 3 ? blockIdx.y + 1 : 0;
  // the branch on src stays outside the loops: inside, the compiler
  // evaluates the (float64) scaling for every element, taken or not
  if (src != nullptr) {
    const T a_t = (T)alpha;
    for (int idx = threadIdx.x; idx < N * W; idx += NT) {
      const int x = idx % N, c = idx / N, y = y0 + c;
      T v = (T)0;
      if (x > 0 && y > 0) {
        const size_t line = DIM == 3 ? (size_t)(z - 1) * n1 + (y - 1) : (size_t)(y - 1);
        v = a_t * to_T<T>(src[line * n1 + (x - 1)]);
      }
      s[x * RS + c] = v;
    }
  } else if (src32 != nullptr) {
    for (int idx = threadIdx.x; idx < N * W; idx += NT) {
      const int x = idx % N, c = idx / N, y = y0 + c;
      T v = (T)0;
      if (x > 0 && y > 0) {
        const size_t line = DIM == 3 ? (size_t)(z - 1) * n1 + (y - 1) : (size_t)(y - 1);
        v = (T)src32[line * n1 + (x - 1)];
      }
      s[x * RS + c] = v;
    }
  } else {
    for (int idx = threadIdx.x; idx < N * W; idx += NT) s[(idx % N) * RS + idx / N] = (T)0;
  }
  __syncthreads();
  if (corr != nullptr) {
    // the line's irregular nodes (distinct x, so distinct words) shared out
    // over the NT / W threads of each column
    constexpr int G = NT / W;
    const int c = threadIdx.x % W, g = threadIdx.x / W, y = y0 + c;
    if (y > 0) {
      const int line = DIM == 3 ? (z - 1) * n1 + (y - 1) : (y - 1);
      const int i0 = line_start[line], i1 = line_start[line + 1];
      for (int i = i0 + g; i < i1; i += G) {
        const int x = irr[i] % n1 + 1;
        s[x * RS + c] += (T)corr[i];
      }
    }
  }
  __syncthreads();
  dst_tile<C>(s, tw, sinv, tot);
  pdl_launch_next();
  const size_t plane = (size_t)z * N * N;
  for (int idx = threadIdx.x; idx < N * W; idx += NT) {
    const int x = idx % N, c = idx / N;
    a[plane + (size_t)(y0 + c) * N + x] = s[x * RS + c];
  }
}

// ------------------------------------------------------------- x inverse
template <typename T, int N, int DIM>
__global__ void __launch_bounds__(NT) k_xinv(T* __restrict__ a, bool keep, double* __restrict__ out,
                                             const double* __restrict__ aux, double beta, double gamma,
                                             const T* __restrict__ tw_g, const int* __restrict__ skip,
                                             const float* __restrict__ aux32 = nullptr) {
  using C = Cfg<T, N>;
  constexpr int W = C::W, RS = C::RS, n1 = N - 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  T* tot = s + N * RS;
  T* tw = tot + C::G * W;
  T* sinv = tw + 4 * N;
  load_twiddles<T, N>(tw, tw_g);
  load_sines<T, N>(sinv, tw_g);
  pdl_wait();
  if (skip != nullptr && *skip != 0) return;
  const int y0 = blockIdx.x * W;
  const int z = DIM == 3 ? blockIdx.y + 1 : 0;
  const size_t plane = (size_t)z * N * N;
  for (int idx = threadIdx.x; idx < N * W; idx += NT) {
    const int x = idx % N, c = idx / N;
    copy_async(&s[x * RS + c], &a[plane + (size_t)(y0 + c) * N + x]);
  }
  copy_async_wait();
  __syncthreads();
  dst_tile<C>(s, tw, sinv, tot);
  pdl_launch_next();
  if (out == nullptr) {
    if (keep)
      for (int idx = threadIdx.x; idx < N * W; idx += NT) {
        const int x = idx % N, c = idx / N;
        a[plane + (size_t)(y0 + c) * N + x] = s[x * RS + c];
      }
    return;
  }
  // out = beta v + gamma aux with beta applied in T (one float64 operation
  // per element without aux, two with), or out = beta v + aux32 with aux32 a
  // padded float grid of the same layout as a (one float64 addition)
  const T b_t = (T)beta;
  for (int idx = threadIdx.x; idx < N * W; idx += NT) {
    const int x = idx % N, c = idx / N, y = y0 + c;
    const T v = s[x * RS + c];
    const size_t pidx = plane + (size_t)y * N + x;
    if (keep) a[pidx] = v;
    if (x > 0 && y > 0) {
      const size_t line = DIM == 3 ? (size_t)(z - 1) * n1 + (y - 1) : (size_t)(y - 1);
      const size_t o = line * n1 + (x - 1);
      const double bv = to_double(b_t * v);
      if (aux32 != nullptr)
        out[o] = bv + ffl::widen(aux32[pidx]);
      else
        out[o] = aux != nullptr ? fma(gamma, aux[o], bv) : bv;
    }
  }
}

// --------------------------------------------------- strided (y / z) passes
// Tile rows = transform index k (stride row_stride), columns x0..x0+W-1 of
// plane q = blockIdx.y + qoff.  SOLVE = forward DST, spectral multiply,
// inverse DST.
template <typename T, int N, bool SOLVE, int DIM>
__global__ void __launch_bounds__(NT) k_strided(T* __restrict__ a, size_t row_stride, size_t plane_stride, int qoff,
                                                const T* __restrict__ mu1, T lambda, T scale,
                                                const T* __restrict__ tw_g, const int* __restrict__ skip,
                                                const T* __restrict__ rinv = nullptr) {
  using C = Cfg<T, N>;
  constexpr int W = C::W, RS = C::RS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  T* tot = s + N * RS;
  T* tw = tot + C::G * W;
  T* sinv = tw + 4 * N;
  load_twiddles<T, N>(tw, tw_g);
  load_sines<T, N>(sinv, tw_g);
  pdl_wait();
  if (skip != nullptr && *skip != 0) return;
  const int x0 = blockIdx.x * W;
  const int q = blockIdx.y + qoff;
  T* base = a + (size_t)q * plane_stride + x0;
  for (int idx = threadIdx.x; idx < N * W; idx += NT) {
    const int c = idx % W, k = idx / W;
    copy_async(&s[k * RS + c], &base[(size_t)k * row_stride + c]);
  }
  copy_async_wait();
  __syncthreads();
  const T muq = DIM == 3 ? mu1[q] : (T)0;
  if constexpr (kRegDst<T, N>) {
    if (SOLVE) {
      const int p = x0 + (int)(threadIdx.x & 31);
      // mu1 is read from global memory here (L1-resident, N values)
      const DivPost post{mu1, mu1[p] + muq - lambda, scale, p == 0};
      dst_tile<C>(s, tw, sinv, tot, post);
    }
    dst_tile<C>(s, tw, sinv, tot);
  } else {
    dst1_tile<C>(s, tw, tot);
    if (SOLVE) {
      // the mode factor scale / mu_p from the table built for this lambda
      // (same expression, so the same value), else divided here
      const T* rq = rinv != nullptr ? rinv + (size_t)q * N * N : nullptr;
      for (int idx = threadIdx.x; idx < N * W; idx += NT) {
        const int c = idx % W, k = idx / W, p = x0 + c;
        T v = (T)0;
        if (k > 0 && p > 0)
          v = s[k * RS + c] * (rq != nullptr ? rq[(size_t)k * N + p] : (scale / (mu1[k] + mu1[p] + muq - lambda)));
        s[k * RS + c] = v;
      }
      __syncthreads();
      dst1_tile<C>(s, tw, tot);
    }
  }
  pdl_launch_next();
  for (int idx = threadIdx.x; idx < N * W; idx += NT) {
    const int c = idx % W, k = idx / W;
    base[(size_t)k * row_stride + c] = s[k * RS + c];
  }
}

// ------------------------------------------- TMA-fed strided passes (float32)
// Persistent blocks walk over [N x 32] tiles of the padded float grid.  One
// thread issues a TMA tensor load of the next tile into the other shared
// buffer (completion counted on an mbarrier) while all threads transform the
// current tile; the finished tile goes back by a TMA tensor store.  Every
// wait is bounded: on timeout the block records DEVERR_TIMEOUT and returns.
constexpr int TMA_W = 32;
// a poll of an incomplete mbarrier takes about 4 us on GB300, so 2^18 polls give up
// after about a second (a tile load completes in microseconds)
constexpr long TMA_WAIT_CAP = 1L << 18;
// resident blocks per SM: three (shared memory allows three at N = 256); at
// 80 registers neither pass spills as long as the plain pass runs its single
// transform inside the runtime-bounded loop (the compile-time bound of one
// lets the compiler schedule it into spills)
template <bool SOLVE>
constexpr int tma_blocks() {
  return 3;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void tma_load3(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void tma_store3(const CUtensorMap* map, const void* src, int x, int y, int z) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(z), "r"(smem_addr(src))
               : "memory");
}
__device__ __forceinline__ void tma_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void tma_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void tma_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

template <int N>
using TmaTile = Tile<float, N, TMA_W, TMA_W>;

// two tiles, scan totals, twiddles, sines, mu1, two mbarriers
template <int N>
constexpr size_t tma_smem_bytes() {
  return (2 * (size_t)N * TMA_W + (size_t)TmaTile<N>::G * TMA_W + 6 * (size_t)N) * sizeof(float) + 2 * sizeof(uint64_t);
}

// mode 0: tiles [y][x-chunk] of plane z = q; mode 1: tiles [z][x-chunk] of row y = q
template <int N, bool SOLVE>
__global__ void __launch_bounds__(NT, tma_blocks<SOLVE>()) k_strided_tma(const __grid_constant__ CUtensorMap map, int mode,
                                                    const float* __restrict__ mu1, float lambda, float scale,
                                                    const float* __restrict__ tw_g, int* __restrict__ err,
                                                    int reps, const int* __restrict__ skip) {
  using C = TmaTile<N>;
  constexpr int W = TMA_W, NX = N / TMA_W;
  constexpr int ntiles = NX * (N - 1);
  constexpr uint32_t bytes = (uint32_t)(N * W * sizeof(float));
  extern __shared__ __align__(128) unsigned char smem_tma[];
  float* buf0 = reinterpret_cast<float*>(smem_tma);
  float* buf1 = buf0 + N * W;
  float* tot = buf1 + N * W;
  float* tw = tot + C::G * W;
  float* sinv = tw + 4 * N;
  float* mus = sinv + N;
  uint64_t* bar = reinterpret_cast<uint64_t*>(mus + N);
  for (int i = threadIdx.x; i < 4 * N; i += NT) tw[i] = tw_g[i];
  for (int i = threadIdx.x; i < N; i += NT) {
    sinv[i] = tw_g[2 * i + 1];
    mus[i] = mu1[i];
  }
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  pdl_wait();
  // an iteration enqueued ahead of the convergence test: nothing to do (the
  // flag is tested before any copy is issued)
  if (skip != nullptr && *skip != 0) return;
  pdl_launch_next();
  __syncthreads();
  auto coords = [&](int t, int& x, int& y, int& z) {
    const int q = t / NX + 1;
    x = (t % NX) * W;
    y = mode == 0 ? 0 : q;
    z = mode == 0 ? q : 0;
  };
  int t = blockIdx.x;
  if (t < ntiles && threadIdx.x == 0) {
    int x, y, z;
    coords(t, x, y, z);
    mbar_expect_tx(&bar[0], bytes);
    tma_load3(buf0, &map, &bar[0], x, y, z);
  }
  for (int i = 0; t < ntiles; t += gridDim.x, ++i) {
    const int b = i & 1;
    float* s = b ? buf1 : buf0;
    float* s_next = b ? buf0 : buf1;
    const int tn = t + gridDim.x;
    if (threadIdx.x == 0 && tn < ntiles) {
      tma_wait_read_all();  // the store of the previous tile has left s_next
      int x, y, z;
      coords(tn, x, y, z);
      mbar_expect_tx(&bar[b ^ 1], bytes);
      tma_load3(s_next, &map, &bar[b ^ 1], x, y, z);
    }
    bool ok = false;
    for (long it = 0; it < TMA_WAIT_CAP; ++it)
      if (mbar_try_wait(&bar[b], (uint32_t)((i >> 1) & 1))) {
        ok = true;
        break;
      }
    if (!ok) {
      if (threadIdx.x == 0) {
        atomicOr(err, DEVERR_TIMEOUT);
        // the copies this block issued finish before its shared memory goes:
        // stores by their bulk group, the pending load by its barrier
        tma_wait_all();
        if (tn < ntiles)
          for (long it = 0; it < TMA_WAIT_CAP; ++it)
            if (mbar_try_wait(&bar[b ^ 1], (uint32_t)(((i + 1) >> 1) & 1))) break;
      }
      return;
    }
    {
      // forward DST with the spectral divide applied to its outputs, then the
      // inverse DST by the same (single inlined) body
      const int q = t / NX + 1, p = (t % NX) * W + (int)(threadIdx.x & 31);
      DivPost post{mus, mus[p] + mus[q] - lambda, scale, p == 0, SOLVE};
#pragma unroll 1
      for (int rep = 0; rep < (SOLVE ? 2 : reps); ++rep) {
        regdst::dst1_tile_reg<regdst::Geo<N, W>>(s, sinv, reinterpret_cast<const regdst::cf2*>(tw), tot, post);
        post.on = false;
      }
    }
    fence_async_shared();
    __syncthreads();
    if (threadIdx.x == 0) {
      int x, y, z;
      coords(t, x, y, z);
      tma_store3(&map, s, x, y, z);
      tma_commit();
    }
  }
  if (threadIdx.x == 0) tma_wait_all();
}

// ------------------------------- fused x and y passes (thread-block clusters)
// One z-plane of the padded float32 grid is transformed along x and then y
// by a cluster of N / 32 blocks (N <= 256) that exchange the plane through
// distributed shared memory, so the plane crosses global memory once per
// direction instead of twice.  Block r of the cluster owns the 32 y-lines
// y = 32 r + c (tile A: rows x, columns c) for the x transform and the 32
// x-modes kx = 32 r + c (tile B: rows y, columns c) for the y transform.
// Between the two, block r reads from every block q the 32 x 32 piece
// A_q[32 r .. 32 r + 31][0 .. 31] (rows of 32 consecutive words in the
// owner's shared memory) and writes it transposed into B rows 32 q ..
// 32 q + 31; the row stride 33 keeps both sides free of bank conflicts.  A
// cluster barrier after the first transform makes every A complete before it
// is read; a second one after the exchange keeps each block's shared memory
// alive until its peers have read it.
namespace cg = cooperative_groups;

template <int N>
constexpr size_t xy_smem_bytes() {
  using C = Cfg<float, N>;
  return (2 * (size_t)N * C::RS + (size_t)C::G * C::W + 5 * (size_t)N) * sizeof(float);
}

// dst[(32 q + lane) RS + j] = src_q[(y0 + j) RS + lane] for every block q of
// the cluster and j < 32: the transposed 32 x 32 pieces.  Warp w moves rows
// j = w + 8 i; the distributed-shared-memory loads of four blocks are issued
// together (16 in flight per thread) before their stores.
template <int N>
__device__ __forceinline__ void xy_exchange(const cg::cluster_group& cluster, float* src, float* dst, int y0) {
  using C = Cfg<float, N>;
  constexpr int W = C::W, RS = C::RS, CL = N / W, R = W / (NT / 32), QB = CL < 4 ? CL : 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll 1
  for (int q0 = 0; q0 < CL; q0 += QB) {
    float v[QB][R];
#pragma unroll
    for (int k = 0; k < QB; ++k) {
      const float* ps = cluster.map_shared_rank(src, q0 + k);
#pragma unroll
      for (int i = 0; i < R; ++i) v[k][i] = ps[(y0 + warp + (NT / 32) * i) * RS + lane];
    }
#pragma unroll
    for (int k = 0; k < QB; ++k)
#pragma unroll
      for (int i = 0; i < R; ++i) dst[((q0 + k) * W + lane) * RS + warp + (NT / 32) * i] = v[k][i];
  }
}

// forward: r = alpha src + corrections (as k_xfwd), x DST, exchange, y DST
template <int N>
__global__ void __launch_bounds__(NT) k_xy_fwd(float* __restrict__ a, const double* __restrict__ src, double alpha,
                                               const float* __restrict__ src32, const double* __restrict__ corr,
                                               const int32_t* __restrict__ irr, const int32_t* __restrict__ line_start,
                                               const float* __restrict__ tw_g, const int* __restrict__ skip) {
  using C = Cfg<float, N>;
  constexpr int W = C::W, RS = C::RS, n1 = N - 1, CL = N / W;
  static_assert(W == 32 && N % W == 0 && CL <= 8, "one cluster of at most 8 blocks per plane");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sA = reinterpret_cast<float*>(smem_raw);
  float* sB = sA + N * RS;
  float* tot = sB + N * RS;
  float* tw = tot + C::G * W;
  float* sinv = tw + 4 * N;
  cg::cluster_group cluster = cg::this_cluster();
  // the flag is set before this launch by the stream's previous kernels, so
  // every block of a cluster sees the same value
  const bool skipped = skip != nullptr && *skip != 0;
  load_twiddles<float, N>(tw, tw_g);
  load_sines<float, N>(sinv, tw_g);
  if (skipped) return;
  const int r = (int)cluster.block_rank();
  const int y0 = r * W;
  const int z = blockIdx.y + 1;
  if (src != nullptr) {
    const float a_t = (float)alpha;
    for (int idx = threadIdx.x; idx < N * W; idx += NT) {
      const int x = idx % N, c = idx / N, y = y0 + c;
      float v = 0.0f;
      if (x > 0 && y > 0) v = a_t * ffl::narrow(src[((size_t)(z - 1) * n1 + (y - 1)) * n1 + (x - 1)]);
      sA[x * RS + c] = v;
    }
  } else if (src32 != nullptr) {
    for (int idx = threadIdx.x; idx < N * W; idx += NT) {
      const int x = idx % N, c = idx / N, y = y0 + c;
      float v = 0.0f;
      if (x > 0 && y > 0) v = src32[((size_t)(z - 1) * n1 + (y - 1)) * n1 + (x - 1)];
      sA[x * RS + c] = v;
    }
  } else {
    for (int idx = threadIdx.x; idx < N * W; idx += NT) sA[(idx % N) * RS + idx / N] = 0.0f;
  }
  __syncthreads();
  if (corr != nullptr) {
    constexpr int G = NT / W;
    const int c = threadIdx.x % W, g = threadIdx.x / W, y = y0 + c;
    if (y > 0) {
      const int line = (z - 1) * n1 + (y - 1);
      const int i0 = line_start[line], i1 = line_start[line + 1];
      for (int i = i0 + g; i < i1; i += G) sA[(irr[i] % n1 + 1) * RS + c] += (float)corr[i];
    }
  }
  __syncthreads();
  dst_tile<C>(sA, tw, sinv, tot);
  cluster.sync();
  xy_exchange<N>(cluster, sA, sB, y0);
  cluster.sync();
  dst_tile<C>(sB, tw, sinv, tot);
  const size_t plane = (size_t)z * N * N;
  for (int idx = threadIdx.x; idx < N * W; idx += NT) {
    const int c = idx % W, y = idx / W;
    a[plane + (size_t)y * N + y0 + c] = sB[y * RS + c];
  }
}

// inverse: y DST, exchange, x DST, output as k_xinv
template <int N>
__global__ void __launch_bounds__(NT) k_xy_inv(float* __restrict__ a, bool keep, double* __restrict__ out,
                                               const double* __restrict__ aux, double beta, double gamma,
                                               const float* __restrict__ tw_g, const int* __restrict__ skip) {
  using C = Cfg<float, N>;
  constexpr int W = C::W, RS = C::RS, n1 = N - 1, CL = N / W;
  static_assert(W == 32 && N % W == 0 && CL <= 8, "one cluster of at most 8 blocks per plane");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sA = reinterpret_cast<float*>(smem_raw);
  float* sB = sA + N * RS;
  float* tot = sB + N * RS;
  float* tw = tot + C::G * W;
  float* sinv = tw + 4 * N;
  cg::cluster_group cluster = cg::this_cluster();
  const bool skipped = skip != nullptr && *skip != 0;
  load_twiddles<float, N>(tw, tw_g);
  load_sines<float, N>(sinv, tw_g);
  if (skipped) return;
  const int r = (int)cluster.block_rank();
  const int y0 = r * W;
  const int z = blockIdx.y + 1;
  const size_t plane = (size_t)z * N * N;
  for (int idx = threadIdx.x; idx < N * W; idx += NT) {
    const int c = idx % W, y = idx / W;
    copy_async(&sB[y * RS + c], &a[plane + (size_t)y * N + y0 + c]);
  }
  copy_async_wait();
  __syncthreads();
  dst_tile<C>(sB, tw, sinv, tot);
  cluster.sync();
  xy_exchange<N>(cluster, sB, sA, y0);
  cluster.sync();
  dst_tile<C>(sA, tw, sinv, tot);
  if (out == nullptr) {
    if (keep)
      for (int idx = threadIdx.x; idx < N * W; idx += NT) {
        const int x = idx % N, c = idx / N;
        a[plane + (size_t)(y0 + c) * N + x] = sA[x * RS + c];
      }
    return;
  }
  const float b_t = (float)beta;
  for (int idx = threadIdx.x; idx < N * W; idx += NT) {
    const int x = idx % N, c = idx / N, y = y0 + c;
    const float v = sA[x * RS + c];
    if (keep) a[plane + (size_t)y * N + x] = v;
    if (x > 0 && y > 0) {
      const size_t o = ((size_t)(z - 1) * n1 + (y - 1)) * n1 + (x - 1);
      const double bv = ffl::widen(b_t * v);
      out[o] = aux != nullptr ? fma(gamma, aux[o], bv) : bv;
    }
  }
}

template <typename K, typename... Args>
cudaError_t launch_cluster(K kernel, int cl, dim3 grid, size_t smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(NT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// opt each kernel into its dynamic shared-memory size once per process
template <typename K>
int prep(K kernel, size_t smem) {
  static const void* done[256];
  static int ndone = 0;
  const void* key = (const void*)kernel;
  for (int i = 0; i < ndone; ++i)
    if (done[i] == key) return KFBI_OK;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) {
    set_error("cudaFuncSetAttribute failed: %s", cudaGetErrorString(e));
    return KFBI_ERR_CUDA;
  }
  if (ndone < 256) done[ndone++] = key;
  return KFBI_OK;
}

// one strided 3-D pass (mode 0: along y, mode 1: along z); float32 grids of
// 32 <= N <= 256 go through the TMA-fed persistent kernel
template <typename T, int N>
int launch_strided3(kfbi_handle* h, int mode, bool solve, T* work, const T* mu1, T lam, T scale, const T* tw,
                    const T* rinv = nullptr) {
  using C = Cfg<T, N>;
  cudaStream_t st = h->stream;
  int rc;
  if constexpr (sizeof(T) == 4 && N >= TMA_W && N <= 256) {
    // the handle's second float grid has its own tensor maps
    const bool second = (const void*)work == (const void*)h->w.grid32b;
    if (h->tma && (!second || h->tma_b)) {
      constexpr size_t smem = tma_smem_bytes<N>();
      const CUtensorMap& map =
          mode == 0 ? (second ? h->tmap_y32b : h->tmap_y32) : (second ? h->tmap_z32b : h->tmap_z32);
      const int tiles = (N / TMA_W) * (N - 1);
      const int nb = (solve ? tma_blocks<true>() : tma_blocks<false>()) * h->sms;
      const int grid = tiles < nb ? tiles : nb;
      cudaError_t e;
      if (solve) {
        if ((rc = prep(k_strided_tma<N, true>, smem))) return rc;
        e = launch_pdl(k_strided_tma<N, true>, dim3(grid), dim3(NT), smem, st, map, mode, mu1, lam, scale, tw,
                       h->w.err, 2, (const int*)h->skip);
      } else {
        if ((rc = prep(k_strided_tma<N, false>, smem))) return rc;
        e = launch_pdl(k_strided_tma<N, false>, dim3(grid), dim3(NT), smem, st, map, mode, mu1, lam, scale, tw,
                       h->w.err, 1, (const int*)h->skip);
      }
      return e == cudaSuccess ? KFBI_OK : launch_failed("TMA strided pass");
    }
  }
  const size_t smem = C::smem_elems * sizeof(T);
  const size_t NN = (size_t)N * N;
  dim3 grid(N / C::W, N - 1);
  if constexpr (sizeof(T) == 4) {
    cudaError_t e;
    if (solve) {
      if ((rc = prep(k_strided<T, N, true, 3>, smem))) return rc;
      e = launch_pdl(k_strided<T, N, true, 3>, grid, dim3(NT), smem, st, work, (size_t)(mode == 0 ? N : NN),
                     (size_t)(mode == 0 ? NN : N), 1, mu1, lam, scale, tw, (const int*)h->skip, rinv);
    } else {
      if ((rc = prep(k_strided<T, N, false, 3>, smem))) return rc;
      e = launch_pdl(k_strided<T, N, false, 3>, grid, dim3(NT), smem, st, work, (size_t)(mode == 0 ? N : NN),
                     (size_t)(mode == 0 ? NN : N), 1, mu1, lam, scale, tw, (const int*)h->skip, (const T*)nullptr);
    }
    return e == cudaSuccess ? KFBI_OK : launch_failed("strided pass");
  }
  if (solve) {
    if ((rc = prep(k_strided<T, N, true, 3>, smem))) return rc;
    k_strided<T, N, true, 3><<<grid, NT, smem, st>>>(work, mode == 0 ? N : NN, mode == 0 ? NN : N, 1, mu1, lam,
                                                     scale, tw, h->skip, rinv);
  } else {
    if ((rc = prep(k_strided<T, N, false, 3>, smem))) return rc;
    k_strided<T, N, false, 3><<<grid, NT, smem, st>>>(work, mode == 0 ? N : NN, mode == 0 ? NN : N, 1, mu1, lam,
                                                      scale, tw, h->skip);
  }
  return KFBI_OK;
}

// scale / mu_p over the mode grid (q, k, p) of the float64 middle pass,
// mu_p = (mu1[k] + mu1[p]) + mu1[q] (3-D) - lambda, in the pass's own order;
// n modes per axis, mode 0 absent (sine modes) or present (cosine modes)
__global__ void k_rinv(const double* __restrict__ mu1, double lambda, double scale, int n, int dim, bool mode0,
                       double* __restrict__ out, int64_t total) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(i % n), k = (int)((i / n) % n), q = (int)(i / ((int64_t)n * n));
    const double muq = dim == 3 ? mu1[q] : 0.0;
    const bool on = mode0 || (k > 0 && p > 0 && (dim == 2 || q > 0));
    out[i] = on ? scale / (mu1[k] + mu1[p] + muq - lambda) : 0.0;
  }
}

// the float64 solve's mode factors for this lambda: built once per lambda
// in a table of N^dim values that the handle owns (none for float32, nor for
// handles that must not allocate)
template <typename T, int N>
const T* mode_factors(kfbi_handle* h, double lambda, double scale) {
  if constexpr (sizeof(T) != 8) {
    return nullptr;
  } else {
    if (!h->rinv_ok) return nullptr;
    const bool cosine = h->grid.bc == KFBI_BOX_NEUMANN;
    const int n = cosine ? N + 1 : N;
    const int64_t total = h->grid.dim == 3 ? (int64_t)n * n * n : (int64_t)n * n;
    if (h->rinv64 == nullptr) {
      if (dalloc(h, &h->rinv64, (size_t)total) != KFBI_OK) {
        cudaGetLastError();
        h->rinv_ok = false;
        return nullptr;
      }
      h->rinv_lambda = std::nan("");
    }
    if (!(h->rinv_lambda == lambda)) {
      const int nb = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
      k_rinv<<<nb, 256, 0, h->stream>>>(h->t.mu, lambda, scale, n, h->grid.dim, cosine, h->rinv64, total);
      KFBI_COUNT(1);
      h->rinv_lambda = lambda;
    }
    return h->rinv64;
  }
}

template <typename T, int N>
int run_solve(kfbi_handle* h, const SolveArgs& sa, T* work, const T* mu1, const T* tw) {
  using C = Cfg<T, N>;
  constexpr int W = C::W;
  const size_t smem = C::smem_elems * sizeof(T);
  const int dim = h->grid.dim;
  cudaStream_t st = h->stream;
  const Tables& t = h->t;
  const T lam = (T)sa.lambda;
  const T scale = (T)(dim == 3 ? (2.0 / N) * (2.0 / N) * (2.0 / N) : (2.0 / N) * (2.0 / N));
  int rc;
  if (dim == 3) {
    dim3 grid(N / W, N - 1);
    if constexpr (sizeof(T) == 4 && N >= 32 && N <= 256) {
      // fused x-y passes: three passes per solve (xy forward, z solve, xy inverse)
      if (h->xy_fused) {
        constexpr size_t sxy = xy_smem_bytes<N>();
        if ((rc = prep(k_xy_fwd<N>, sxy))) return rc;
        if ((rc = prep(k_xy_inv<N>, sxy))) return rc;
        cudaError_t e = launch_cluster(k_xy_fwd<N>, N / 32, grid, sxy, st, work, sa.src, sa.alpha, sa.src32, sa.corr,
                                       (const int32_t*)t.irr, (const int32_t*)t.line_start, tw, h->skip);
        if (e == cudaSuccess) {
          if ((rc = launch_strided3<T, N>(h, 1, true, work, mu1, lam, scale, tw))) return rc;
          e = launch_cluster(k_xy_inv<N>, N / 32, grid, sxy, st, work, sa.keep || sa.out_user == nullptr,
                             sa.out_user, sa.aux, sa.beta, sa.gamma, tw, h->skip);
          if (e != cudaSuccess) {
            set_error("cluster launch of the fused x-y inverse pass failed: %s", cudaGetErrorString(e));
            return KFBI_ERR_CUDA;
          }
          KFBI_CHECK_LAUNCH_N(3);
          return KFBI_OK;
        }
        // no cluster of this size fits: the five-pass path from now on
        cudaGetLastError();
        h->xy_fused = false;
      }
    }
    const T* rinv = mode_factors<T, N>(h, sa.lambda, (double)scale);
    if ((rc = prep(k_xfwd<T, N, 3>, smem))) return rc;
    if ((rc = prep(k_xinv<T, N, 3>, smem))) return rc;
    if constexpr (sizeof(T) == 4) {
      // float32: the five passes chained by programmatic dependent launch
      if (launch_pdl(k_xfwd<T, N, 3>, grid, dim3(NT), smem, st, work, sa.src, sa.alpha, sa.src32, sa.corr,
                     (const int32_t*)t.irr, (const int32_t*)t.line_start, tw, (const int*)h->skip) != cudaSuccess)
        return launch_failed("x forward pass");
    } else {
      k_xfwd<T, N, 3><<<grid, NT, smem, st>>>(work, sa.src, sa.alpha, sa.src32, sa.corr, t.irr, t.line_start, tw,
                                               h->skip);
    }
    if ((rc = launch_strided3<T, N>(h, 0, false, work, mu1, lam, scale, tw))) return rc;
    if ((rc = launch_strided3<T, N>(h, 1, true, work, mu1, lam, scale, tw, rinv))) return rc;
    if ((rc = launch_strided3<T, N>(h, 0, false, work, mu1, lam, scale, tw))) return rc;
    if constexpr (sizeof(T) == 4) {
      if (launch_pdl(k_xinv<T, N, 3>, grid, dim3(NT), smem, st, work, sa.keep || sa.out_user == nullptr, sa.out_user,
                     (const double*)sa.aux, sa.beta, sa.gamma, tw, (const int*)h->skip, sa.aux32) != cudaSuccess)
        return launch_failed("x inverse pass");
    } else {
      k_xinv<T, N, 3><<<grid, NT, smem, st>>>(work, sa.keep || sa.out_user == nullptr, sa.out_user, sa.aux, sa.beta,
                                               sa.gamma, tw, h->skip, sa.aux32);
    }
  } else {
    dim3 grid(N / W, 1);
    const T* rinv = mode_factors<T, N>(h, sa.lambda, (double)scale);
    if ((rc = prep(k_xfwd<T, N, 2>, smem))) return rc;
    k_xfwd<T, N, 2><<<grid, NT, smem, st>>>(work, sa.src, sa.alpha, sa.src32, sa.corr, t.irr, t.line_start, tw,
                                             h->skip);
    if ((rc = prep(k_strided<T, N, true, 2>, smem))) return rc;
    k_strided<T, N, true, 2><<<grid, NT, smem, st>>>(work, N, 0, 0, mu1, lam, scale, tw, h->skip, rinv);
    if ((rc = prep(k_xinv<T, N, 2>, smem))) return rc;
    k_xinv<T, N, 2><<<grid, NT, smem, st>>>(work, sa.keep || sa.out_user == nullptr, sa.out_user, sa.aux, sa.beta,
                                             sa.gamma, tw, h->skip, sa.aux32);
  }
  KFBI_CHECK_LAUNCH_N(dim == 3 ? 5 : 3);
  return KFBI_OK;
}

// one pass of the solver on the padded work grid (timing of single kernels)
template <typename T, int N>
int run_pass(kfbi_handle* h, int pass, double lambda, T* work, const T* mu1, const T* tw) {
  using C = Cfg<T, N>;
  constexpr int W = C::W;
  const size_t smem = C::smem_elems * sizeof(T);
  const int dim = h->grid.dim;
  cudaStream_t st = h->stream;
  const Tables& t = h->t;
  const T lam = (T)lambda;
  const T scale = (T)(dim == 3 ? (2.0 / N) * (2.0 / N) * (2.0 / N) : (2.0 / N) * (2.0 / N));
  const size_t NN = (size_t)N * N;
  dim3 grid(N / W, dim == 3 ? N - 1 : 1);
  int rc;
  if (dim == 3) {
    if (pass == 0) {
      if ((rc = prep(k_xfwd<T, N, 3>, smem))) return rc;
      k_xfwd<T, N, 3><<<grid, NT, smem, st>>>(work, nullptr, 1.0, nullptr, nullptr, t.irr, t.line_start, tw, nullptr);
    } else if (pass == 1) {
      if ((rc = launch_strided3<T, N>(h, 0, false, work, mu1, lam, scale, tw))) return rc;
    } else if (pass == 2) {
      const T* rinv = mode_factors<T, N>(h, lambda, (double)scale);
      if ((rc = launch_strided3<T, N>(h, 1, true, work, mu1, lam, scale, tw, rinv))) return rc;
    } else if (pass == 3) {
      if ((rc = prep(k_xinv<T, N, 3>, smem))) return rc;
      k_xinv<T, N, 3><<<grid, NT, smem, st>>>(work, true, nullptr, nullptr, 1.0, 0.0, tw, nullptr);
    } else {
      // 4 / 5: the fused x-y forward / inverse pass
      if constexpr (sizeof(T) == 4 && N >= 32 && N <= 256) {
        if (h->xy_fused) {
          constexpr size_t sxy = xy_smem_bytes<N>();
          cudaError_t e;
          if (pass == 4) {
            if ((rc = prep(k_xy_fwd<N>, sxy))) return rc;
            e = launch_cluster(k_xy_fwd<N>, N / 32, grid, sxy, st, work, (const double*)nullptr, 1.0,
                               (const float*)nullptr, (const double*)nullptr, (const int32_t*)t.irr,
                               (const int32_t*)t.line_start, tw, (const int*)nullptr);
          } else {
            if ((rc = prep(k_xy_inv<N>, sxy))) return rc;
            e = launch_cluster(k_xy_inv<N>, N / 32, grid, sxy, st, work, true, (double*)nullptr,
                               (const double*)nullptr, 1.0, 0.0, tw, (const int*)nullptr);
          }
          if (e != cudaSuccess) {
            set_error("cluster launch failed: %s", cudaGetErrorString(e));
            return KFBI_ERR_CUDA;
          }
          KFBI_CHECK_LAUNCH();
          return KFBI_OK;
        }
      }
      set_error("no fused x-y pass for this grid and precision");
      return KFBI_ERR_ARG;
    }
    (void)NN;
  } else {
    if (pass == 0) {
      if ((rc = prep(k_xfwd<T, N, 2>, smem))) return rc;
      k_xfwd<T, N, 2><<<grid, NT, smem, st>>>(work, nullptr, 1.0, nullptr, nullptr, t.irr, t.line_start, tw, nullptr);
    } else if (pass == 1 || pass == 2) {
      const T* rinv = mode_factors<T, N>(h, lambda, (double)scale);
      if ((rc = prep(k_strided<T, N, true, 2>, smem))) return rc;
      k_strided<T, N, true, 2><<<grid, NT, smem, st>>>(work, N, 0, 0, mu1, lam, scale, tw, nullptr, rinv);
    } else {
      if ((rc = prep(k_xinv<T, N, 2>, smem))) return rc;
      k_xinv<T, N, 2><<<grid, NT, smem, st>>>(work, true, nullptr, nullptr, 1.0, 0.0, tw, nullptr);
    }
  }
  KFBI_CHECK_LAUNCH();
  return KFBI_OK;
}

// ------------------------------------------ coupled anisotropic solve pass
// Middle pass of the coupled box solve (3-D: along z, 2-D: along y) on the
// two padded work grids a (intracellular) and b (extracellular): forward
// DST of both tiles, the per-mode 2 x 2 solve of Eq. pde1 with diagonal
// conductivities (Section 5.2, Eq. FDE),
//   [A_i - kappa, kappa; kappa, A_e - kappa] (v_i, v_e) = (r_i, r_e),
//   A_c = sum_a d_c,a mu1(p_a),
// scaled by (2/N)^d, then the inverse DST of both tiles.  The solve takes
// its three factors per mode (v_i = f0 r_i + f1 r_e, v_e = f1 r_i + f2 r_e)
// from a table built once per kappa in float64 (k_cpl_factors).
template <typename T, int N, int DIM>
__global__ void __launch_bounds__(NT) k_strided_coupled(T* __restrict__ a, T* __restrict__ b, size_t row_stride,
                                                        size_t plane_stride, int qoff, const T* __restrict__ cf,
                                                        size_t cf_stride, const T* __restrict__ tw_g,
                                                        const int* __restrict__ skip) {
  using C = Cfg<T, N>;
  constexpr int W = C::W, RS = C::RS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sa = reinterpret_cast<T*>(smem_raw);
  T* sb = sa + N * RS;
  T* tot = sb + N * RS;
  T* tw = tot + C::G * W;
  T* sinv = tw + 4 * N;
  const bool skipped = skip != nullptr && *skip != 0;
  load_twiddles<T, N>(tw, tw_g);
  load_sines<T, N>(sinv, tw_g);
  if (skipped) return;
  const int x0 = blockIdx.x * W;
  const int q = blockIdx.y + qoff;
  T* ba = a + (size_t)q * plane_stride + x0;
  T* bb = b + (size_t)q * plane_stride + x0;
  for (int idx = threadIdx.x; idx < N * W; idx += NT) {
    const int c = idx % W, k = idx / W;
    copy_async(&sa[k * RS + c], &ba[(size_t)k * row_stride + c]);
    copy_async(&sb[k * RS + c], &bb[(size_t)k * row_stride + c]);
  }
  copy_async_wait();
  __syncthreads();
  dst_tile<C>(sa, tw, sinv, tot);
  dst_tile<C>(sb, tw, sinv, tot);
  // table row of this plane: modes (q, k, p), p fastest
  const T* f0 = cf + (size_t)q * N * N + x0;
  for (int idx = threadIdx.x; idx < N * W; idx += NT) {
    const int c = idx % W, k = idx / W;
    const size_t o = (size_t)k * N + c;
    const T g0 = f0[o], g1 = f0[o + cf_stride], g2 = f0[o + 2 * cf_stride];
    const T ri = sa[k * RS + c], re = sb[k * RS + c];
    sa[k * RS + c] = g0 * ri + g1 * re;
    sb[k * RS + c] = g1 * ri + g2 * re;
  }
  __syncthreads();
  dst_tile<C>(sa, tw, sinv, tot);
  dst_tile<C>(sb, tw, sinv, tot);
  for (int idx = threadIdx.x; idx < N * W; idx += NT) {
    const int c = idx % W, k = idx / W;
    ba[(size_t)k * row_stride + c] = sa[k * RS + c];
    bb[(size_t)k * row_stride + c] = sb[k * RS + c];
  }
}

// factors of the per-mode 2 x 2 solve over the mode grid (q, k, p) of the
// middle pass (3-D: y = q, z = k; 2-D: y = k, q = 0), x = p:
//   [A_i - kappa, kappa; kappa, A_e - kappa]^{-1} scale
//     = (scale / det) [A_e - kappa, -kappa; -kappa, A_i - kappa],
//   A_c = sum_a d_c,a mu1(p_a), det = (A_i - kappa)(A_e - kappa) - kappa^2,
// computed in float64 and stored as T (0 for the absent sine modes)
template <typename T>
__global__ void k_cpl_factors(const double* __restrict__ mu1, Coupling cp, int N, int dim, T* __restrict__ cf,
                              int64_t total) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(i % N), k = (int)((i / N) % N), q = (int)(i / ((int64_t)N * N));
    double g0 = 0.0, g1 = 0.0, g2 = 0.0;
    if (k > 0 && p > 0 && (dim == 2 || q > 0)) {
      const double mx = mu1[p], my = dim == 3 ? mu1[q] : mu1[k], mz = dim == 3 ? mu1[k] : 0.0;
      const double ai = cp.di[0] * mx + cp.di[1] * my + cp.di[2] * mz - cp.kappa;
      const double ae = cp.de[0] * mx + cp.de[1] * my + cp.de[2] * mz - cp.kappa;
      const double sc = cp.scale / (ai * ae - cp.kappa * cp.kappa);
      g0 = ae * sc;
      g1 = -cp.kappa * sc;
      g2 = ai * sc;
    }
    cf[i] = (T)g0;
    cf[i + total] = (T)g1;
    cf[i + 2 * total] = (T)g2;
  }
}

// the handle's factor table of element type T for this kappa (built when
// kappa changes)
template <typename T>
const T* coupled_factors(kfbi_handle* h, const Coupling& cp, int N, int64_t total) {
  T** tab;
  double* kap;
  if constexpr (sizeof(T) == 8) {
    tab = &h->cpl64;
    kap = &h->cpl64_kappa;
  } else {
    tab = &h->cpl32;
    kap = &h->cpl32_kappa;
  }
  if (*tab == nullptr) {
    if (dalloc(h, tab, (size_t)(3 * total)) != KFBI_OK) return nullptr;
    *kap = std::nan("");
  }
  if (!(*kap == cp.kappa)) {
    const int nb = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
    k_cpl_factors<T><<<nb, 256, 0, h->stream>>>(h->t.mu, cp, N, h->grid.dim, *tab, total);
    KFBI_COUNT(1);
    *kap = cp.kappa;
  }
  return *tab;
}

// the coupled box solve on two padded grids of element type T: x forward
// (sources and corrections), y, the coupled z solve, y, x inverse (outputs).
// The y passes of both fields use the plain strided kernel (the tensor maps
// describe only the handle's first float grid).
template <typename T, int N>
int run_solve_coupled(kfbi_handle* h, const SolveArgs& si, const SolveArgs& se, const Coupling& cp0, T* wa, T* wb,
                      const T* mu1T, const T* tw) {
  using C = Cfg<T, N>;
  constexpr int W = C::W;
  const size_t smem = C::smem_elems * sizeof(T);
  const size_t smem2 = (2 * (size_t)N * C::RS + (size_t)C::G * W + 5 * (size_t)N) * sizeof(T);
  const int dim = h->grid.dim;
  cudaStream_t st = h->stream;
  const Tables& t = h->t;
  Coupling cp = cp0;
  cp.scale = dim == 3 ? (2.0 / N) * (2.0 / N) * (2.0 / N) : (2.0 / N) * (2.0 / N);
  int rc;
  const dim3 grid(N / W, dim == 3 ? N - 1 : 1);
  const int64_t total = dim == 3 ? (int64_t)N * N * N : (int64_t)N * N;
  const T* cf = coupled_factors<T>(h, cp, N, total);
  if (cf == nullptr) {
    set_error("allocation of the coupled solve's factor table failed");
    return KFBI_ERR_OOM;
  }
  if (dim == 3) {
    if ((rc = prep(k_xfwd<T, N, 3>, smem))) return rc;
    if ((rc = prep(k_strided_coupled<T, N, 3>, smem2))) return rc;
    if ((rc = prep(k_xinv<T, N, 3>, smem))) return rc;
    if ((rc = prep(k_strided<T, N, false, 3>, smem))) return rc;
    k_xfwd<T, N, 3><<<grid, NT, smem, st>>>(wa, si.src, si.alpha, si.src32, si.corr, t.irr, t.line_start, tw, h->skip);
    k_xfwd<T, N, 3><<<grid, NT, smem, st>>>(wb, se.src, se.alpha, se.src32, se.corr, t.irr, t.line_start, tw, h->skip);
    const size_t NN = (size_t)N * N;
    for (T* w : {wa, wb})
      k_strided<T, N, false, 3><<<grid, NT, smem, st>>>(w, N, NN, 1, mu1T, (T)0, (T)1, tw, h->skip);
    k_strided_coupled<T, N, 3><<<grid, NT, smem2, st>>>(wa, wb, NN, N, 1, cf, (size_t)total, tw, h->skip);
    for (T* w : {wa, wb})
      k_strided<T, N, false, 3><<<grid, NT, smem, st>>>(w, N, NN, 1, mu1T, (T)0, (T)1, tw, h->skip);
    k_xinv<T, N, 3><<<grid, NT, smem, st>>>(wa, si.keep || si.out_user == nullptr, si.out_user, si.aux, si.beta,
                                             si.gamma, tw, h->skip);
    k_xinv<T, N, 3><<<grid, NT, smem, st>>>(wb, se.keep || se.out_user == nullptr, se.out_user, se.aux, se.beta,
                                             se.gamma, tw, h->skip);
  } else {
    if ((rc = prep(k_xfwd<T, N, 2>, smem))) return rc;
    if ((rc = prep(k_strided_coupled<T, N, 2>, smem2))) return rc;
    if ((rc = prep(k_xinv<T, N, 2>, smem))) return rc;
    k_xfwd<T, N, 2><<<grid, NT, smem, st>>>(wa, si.src, si.alpha, si.src32, si.corr, t.irr, t.line_start, tw, h->skip);
    k_xfwd<T, N, 2><<<grid, NT, smem, st>>>(wb, se.src, se.alpha, se.src32, se.corr, t.irr, t.line_start, tw, h->skip);
    k_strided_coupled<T, N, 2><<<grid, NT, smem2, st>>>(wa, wb, N, 0, 0, cf, (size_t)total, tw, h->skip);
    k_xinv<T, N, 2><<<grid, NT, smem, st>>>(wa, si.keep || si.out_user == nullptr, si.out_user, si.aux, si.beta,
                                             si.gamma, tw, h->skip);
    k_xinv<T, N, 2><<<grid, NT, smem, st>>>(wb, se.keep || se.out_user == nullptr, se.out_user, se.aux, se.beta,
                                             se.gamma, tw, h->skip);
  }
  KFBI_CHECK_LAUNCH_N(dim == 3 ? 9 : 5);
  return KFBI_OK;
}

template <typename T>
int dispatch(kfbi_handle* h, const SolveArgs& sa, T* work, const T* mu1, const T* tw) {
  switch (h->grid.N) {
    case 8: return run_solve<T, 8>(h, sa, work, mu1, tw);
    case 16: return run_solve<T, 16>(h, sa, work, mu1, tw);
    case 32: return run_solve<T, 32>(h, sa, work, mu1, tw);
    case 64: return run_solve<T, 64>(h, sa, work, mu1, tw);
    case 128: return run_solve<T, 128>(h, sa, work, mu1, tw);
    case 256: return run_solve<T, 256>(h, sa, work, mu1, tw);
    case 384: return run_solve<T, 384>(h, sa, work, mu1, tw);
    case 512: return run_solve<T, 512>(h, sa, work, mu1, tw);
    default:
      set_error("unsupported grid size N=%d", h->grid.N);
      return KFBI_ERR_ARG;
  }
}

template <typename T>
int dispatch_pass(kfbi_handle* h, int pass, double lambda, T* work, const T* mu1, const T* tw) {
  switch (h->grid.N) {
    case 8: return run_pass<T, 8>(h, pass, lambda, work, mu1, tw);
    case 16: return run_pass<T, 16>(h, pass, lambda, work, mu1, tw);
    case 32: return run_pass<T, 32>(h, pass, lambda, work, mu1, tw);
    case 64: return run_pass<T, 64>(h, pass, lambda, work, mu1, tw);
    case 128: return run_pass<T, 128>(h, pass, lambda, work, mu1, tw);
    case 256: return run_pass<T, 256>(h, pass, lambda, work, mu1, tw);
    case 384: return run_pass<T, 384>(h, pass, lambda, work, mu1, tw);
    case 512: return run_pass<T, 512>(h, pass, lambda, work, mu1, tw);
    default:
      set_error("unsupported grid size N=%d", h->grid.N);
      return KFBI_ERR_ARG;
  }
}

// ------------------------------------------------------ Neumann box (DCT-I)
// The box Green's function of Section 4 with zero normal derivative on the
// box boundary: all (N+1)^d nodes are unknowns, the boundary rows use the
// mirrored ghost value, and the cosine modes diagonalise the operator,
//   v = (2/N)^d C( mu^{-1} o C r ),  C_{kp} = c_k cos(pi k p / N),
//   c_0 = c_N = 1/2, c_k = 1 otherwise, k, p = 0..N,
// with the same mu_p as the sine solve (p = 0..N).  Work and user grids share
// the layout (N+1)^d, x fastest.  A tile holds N+1 transform rows by W lines.

template <typename C>
constexpr size_t dct_smem_elems() {
  // tile, scan totals, twiddles, X_1 per column, sines (register path)
  return (size_t)(C::N + 1) * C::RS + (size_t)C::G * C::W + 4 * (size_t)C::N + C::W + C::N;
}

// DCT-I X_p = sum_k c_k x_k cos(pi k p / N) of every column of the tile
// s[N+1][RS] in place.  The same length-N/2 complex FFT as the sine
// transform, after the cosine pre-fold
//   y_0 = (x_0 + x_N)/2,  y_j = (x_j + x_{N-j})/2 - sin(pi j/N)(x_j - x_{N-j}),
// gives Y_k = sum_j y_j e^{2 pi i j k / N} with X_{2k} = Re Y_k and
// X_{2k+1} = X_{2k-1} + Im Y_k (from 2 sin a sin b = cos(a-b) - cos(a+b)),
// started by X_1 = sum_k c_k x_k cos(pi k / N), summed directly.
// x1 = scratch [W].
template <typename C>
__device__ void dct1_tile(typename C::T* s, const typename C::T* tw, typename C::T* tot, typename C::T* x1) {
  using T = typename C::T;
  constexpr int N = C::N, L = C::L, W = C::W, RS = C::RS, G = C::G;
  {
    constexpr int SEG = (N + 1 + G - 1) / G;
    const int c = threadIdx.x % W, g = threadIdx.x / W;
    const int j0 = g * SEG;
    const int j1 = (j0 + SEG < N + 1) ? j0 + SEG : N + 1;
    T acc = (T)0;
    for (int j = j0; j < j1; ++j) {
      T cw = tw[2 * j];
      if (j == 0 || j == N) cw *= (T)0.5;
      acc += cw * s[j * RS + c];
    }
    tot[g * W + c] = acc;
    __syncthreads();
    if (g == 0) {
      T sum = (T)0;
      for (int g2 = 0; g2 < G; ++g2) sum += tot[g2 * W + c];
      x1[c] = sum;
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < (N / 2 + 1) * W; idx += NT) {
    const int c = idx % W, j = idx / W;
    if (j == 0) {
      s[c] = (T)0.5 * (s[c] + s[N * RS + c]);
    } else if (j < N / 2) {
      const T a = s[j * RS + c], b = s[(N - j) * RS + c];
      const T m = (T)0.5 * (a + b), d = tw[2 * j + 1] * (a - b);
      s[j * RS + c] = m - d;
      s[(N - j) * RS + c] = m + d;
    }
  }
  __syncthreads();
  Stages<C, 1, L>::run(s, tw);
  // split into the real DFT: X_0, X_N from Z_0; X_{2k} in row 2k and the
  // increments Im Y_k in row 2k+1
  for (int idx = threadIdx.x; idx < (L / 2 + 1) * W; idx += NT) {
    const int c = idx % W, k = idx / W;
    if (k == 0) {
      const T a = s[c], b = s[RS + c];
      s[c] = a + b;
      s[N * RS + c] = a - b;
      s[RS + c] = (T)0;
    } else {
      const int kk = L - k;
      const T Ar = s[(2 * k) * RS + c], Ai = s[(2 * k + 1) * RS + c];
      const T Br = s[(2 * kk) * RS + c], Bi = s[(2 * kk + 1) * RS + c];
      {
        const T wr = tw[2 * (2 * k)], wi = tw[2 * (2 * k) + 1];
        const T Sr = Ar + Br, Si = Ai - Bi, Dr = Ar - Br, Di = Ai + Bi;
        s[(2 * k) * RS + c] = (T)0.5 * (Sr + wr * Di + wi * Dr);
        s[(2 * k + 1) * RS + c] = (T)0.5 * (Si - wr * Dr + wi * Di);
      }
      if (kk != k) {
        const T wr = tw[2 * (2 * kk)], wi = tw[2 * (2 * kk) + 1];
        const T Sr = Br + Ar, Si = Bi - Ai, Dr = Br - Ar, Di = Bi + Ai;
        s[(2 * kk) * RS + c] = (T)0.5 * (Sr + wr * Di + wi * Dr);
        s[(2 * kk + 1) * RS + c] = (T)0.5 * (Si - wr * Dr + wi * Di);
      }
    }
  }
  __syncthreads();
  // odd outputs: column-wise inclusive scan of the increments, plus X_1
  {
    constexpr int SEG = (L + G - 1) / G;
    const int c = threadIdx.x % W, g = threadIdx.x / W;
    const int k0 = g * SEG;
    const int k1 = (k0 + SEG < L) ? k0 + SEG : L;
    T acc = (T)0;
    for (int k = k0; k < k1; ++k) {
      acc += s[(2 * k + 1) * RS + c];
      s[(2 * k + 1) * RS + c] = acc;
    }
    tot[g * W + c] = acc;
    __syncthreads();
    T off = x1[c];
    for (int g2 = 0; g2 < g; ++g2) off += tot[g2 * W + c];
    for (int k = k0; k < k1; ++k) s[(2 * k + 1) * RS + c] += off;
    __syncthreads();
  }
}

// the cosine transform of every column of the tile, rows 0..N: the
// register-resident path for float32 tiles of 32 <= N <= 512 lines, the
// shared-memory FFT otherwise
template <typename C>
__device__ __forceinline__ void dct_tile(typename C::T* s, const typename C::T* tw, const typename C::T* sinv,
                                         typename C::T* tot, typename C::T* x1) {
  if constexpr (kRegDst<typename C::T, C::N>) {
    regdst::dct1_tile_reg<regdst::Geo<C::N, C::RS>>(s, sinv, reinterpret_cast<const regdst::cf2*>(tw), tot, x1);
  } else {
    dct1_tile<C>(s, tw, tot, x1);
  }
}

// x forward on the Neumann layout: W lines y0..y0+W-1 (y <= N) of plane z,
// r = alpha*src + corrections assembled while loading.  The irregular nodes
// (all interior) are listed per interior x-line in the interior numbering.
template <typename T, int N, int DIM>
__global__ void __launch_bounds__(NT) k_nxfwd(T* __restrict__ a, const double* __restrict__ src, double alpha,
                                              const float* __restrict__ src32,
                                              const double* __restrict__ corr, const int32_t* __restrict__ irr,
                                              const int32_t* __restrict__ line_start, const T* __restrict__ tw_g,
                                              const int* __restrict__ skip) {
  using C = Cfg<T, N>;
  constexpr int W = C::W, RS = C::RS, P = N + 1, n1 = N - 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  T* tot = s + P * RS;
  T* tw = tot + C::G * W;
  T* x1 = tw + 4 * N;
  T* sinv = x1 + W;
  const bool skipped = skip != nullptr && *skip != 0;
  load_twiddles<T, N>(tw, tw_g);
  load_sines<T, N>(sinv, tw_g);
  if (skipped) return;
  const int y0 = blockIdx.x * W;
  const int z = DIM == 3 ? blockIdx.y : 0;
  const size_t plane = (size_t)z * P * P;
  for (int idx = threadIdx.x; idx < P * W; idx += NT) {
    const int x = idx % P, c = idx / P, y = y0 + c;
    T v = (T)0;
    if (y <= N) {
      if (src != nullptr) v = (T)alpha * to_T<T>(src[plane + (size_t)y * P + x]);
      else if (src32 != nullptr) v = (T)src32[plane + (size_t)y * P + x];
    }
    s[x * RS + c] = v;
  }
  __syncthreads();
  if (corr != nullptr) {
    constexpr int G = NT / W;
    const int c = threadIdx.x % W, g = threadIdx.x / W, y = y0 + c;
    if (y >= 1 && y <= n1 && (DIM == 2 || (z >= 1 && z <= n1))) {
      const int line = DIM == 3 ? (z - 1) * n1 + (y - 1) : (y - 1);
      const int i0 = line_start[line], i1 = line_start[line + 1];
      for (int i = i0 + g; i < i1; i += G) {
        const int x = irr[i] % n1 + 1;
        s[x * RS + c] += (T)corr[i];
      }
    }
  }
  __syncthreads();
  dct_tile<C>(s, tw, sinv, tot, x1);
  for (int idx = threadIdx.x; idx < P * W; idx += NT) {
    const int x = idx % P, c = idx / P, y = y0 + c;
    if (y <= N) a[plane + (size_t)y * P + x] = s[x * RS + c];
  }
}

// x inverse on the Neumann layout: the work grid keeps v (keep) and/or
// out = beta v + gamma aux
template <typename T, int N, int DIM>
__global__ void __launch_bounds__(NT) k_nxinv(T* __restrict__ a, bool keep, double* __restrict__ out,
                                              const double* __restrict__ aux, double beta, double gamma,
                                              const T* __restrict__ tw_g, const int* __restrict__ skip) {
  using C = Cfg<T, N>;
  constexpr int W = C::W, RS = C::RS, P = N + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  T* tot = s + P * RS;
  T* tw = tot + C::G * W;
  T* x1 = tw + 4 * N;
  T* sinv = x1 + W;
  if (skip != nullptr && *skip != 0) return;
  load_twiddles<T, N>(tw, tw_g);
  load_sines<T, N>(sinv, tw_g);
  const int y0 = blockIdx.x * W;
  const int z = DIM == 3 ? blockIdx.y : 0;
  const size_t plane = (size_t)z * P * P;
  for (int idx = threadIdx.x; idx < P * W; idx += NT) {
    const int x = idx % P, c = idx / P, y = y0 + c;
    if (y <= N) copy_async(&s[x * RS + c], &a[plane + (size_t)y * P + x]);
    else s[x * RS + c] = (T)0;
  }
  copy_async_wait();
  __syncthreads();
  dct_tile<C>(s, tw, sinv, tot, x1);
  for (int idx = threadIdx.x; idx < P * W; idx += NT) {
    const int x = idx % P, c = idx / P, y = y0 + c;
    if (y > N) continue;
    const size_t o = plane + (size_t)y * P + x;
    const T v = s[x * RS + c];
    if (keep) a[o] = v;
    if (out != nullptr) {
      const double bv = to_double((T)beta * v);
      out[o] = aux != nullptr ? fma(gamma, aux[o], bv) : bv;
    }
  }
}

// strided (y / z) pass on the Neumann layout: rows k = 0..N at row_stride,
// columns x0..x0+W-1 (x <= N) of plane q.  SOLVE: forward DCT, multiply by
// scale / (mu1[k] + mu1[p] + mu1[q] - lambda), inverse DCT.
template <typename T, int N, bool SOLVE, int DIM>
__global__ void __launch_bounds__(NT) k_nstrided(T* __restrict__ a, size_t row_stride, size_t plane_stride,
                                                 const T* __restrict__ mu1, T lambda, T scale,
                                                 const T* __restrict__ tw_g, const int* __restrict__ skip,
                                                 const T* __restrict__ rinv = nullptr) {
  using C = Cfg<T, N>;
  constexpr int W = C::W, RS = C::RS, P = N + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  T* tot = s + P * RS;
  T* tw = tot + C::G * W;
  T* x1 = tw + 4 * N;
  T* sinv = x1 + W;
  const bool skipped = skip != nullptr && *skip != 0;
  load_twiddles<T, N>(tw, tw_g);
  load_sines<T, N>(sinv, tw_g);
  if (skipped) return;
  const int x0 = blockIdx.x * W;
  const int q = blockIdx.y;
  T* base = a + (size_t)q * plane_stride + x0;
  for (int idx = threadIdx.x; idx < P * W; idx += NT) {
    const int c = idx % W, k = idx / W;
    if (x0 + c <= N) copy_async(&s[k * RS + c], &base[(size_t)k * row_stride + c]);
    else s[k * RS + c] = (T)0;
  }
  copy_async_wait();
  __syncthreads();
  dct_tile<C>(s, tw, sinv, tot, x1);
  if (SOLVE) {
    const T muq = DIM == 3 ? mu1[q] : (T)0;
    const T* rq = rinv != nullptr ? rinv + (size_t)q * P * P : nullptr;
    for (int idx = threadIdx.x; idx < P * W; idx += NT) {
      const int c = idx % W, k = idx / W, p = x0 + c;
      if (p <= N)
        s[k * RS + c] *= rq != nullptr ? rq[(size_t)k * P + p] : scale / (mu1[k] + mu1[p] + muq - lambda);
    }
    __syncthreads();
    dct_tile<C>(s, tw, sinv, tot, x1);
  }
  for (int idx = threadIdx.x; idx < P * W; idx += NT) {
    const int c = idx % W, k = idx / W;
    if (x0 + c <= N) base[(size_t)k * row_stride + c] = s[k * RS + c];
  }
}

template <typename T, int N>
int run_solve_neumann(kfbi_handle* h, const SolveArgs& sa, T* work, const T* mu1, const T* tw) {
  using C = Cfg<T, N>;
  constexpr int W = C::W, P = N + 1;
  const size_t smem = dct_smem_elems<C>() * sizeof(T);
  const int dim = h->grid.dim;
  cudaStream_t st = h->stream;
  const Tables& t = h->t;
  const T scale = (T)(dim == 3 ? (2.0 / N) * (2.0 / N) * (2.0 / N) : (2.0 / N) * (2.0 / N));
  const T lam = (T)sa.lambda;
  const dim3 grid((P + W - 1) / W, dim == 3 ? P : 1);
  const size_t PP = (size_t)P * P;
  const T* rinv = mode_factors<T, N>(h, sa.lambda, (double)scale);
  int rc;
  if (dim == 3) {
    if ((rc = prep(k_nxfwd<T, N, 3>, smem))) return rc;
    if ((rc = prep(k_nstrided<T, N, false, 3>, smem))) return rc;
    if ((rc = prep(k_nstrided<T, N, true, 3>, smem))) return rc;
    if ((rc = prep(k_nxinv<T, N, 3>, smem))) return rc;
    k_nxfwd<T, N, 3><<<grid, NT, smem, st>>>(work, sa.src, sa.alpha, sa.src32, sa.corr, t.irr, t.line_start, tw,
                                                h->skip);
    k_nstrided<T, N, false, 3><<<grid, NT, smem, st>>>(work, P, PP, mu1, lam, scale, tw, h->skip);
    k_nstrided<T, N, true, 3><<<grid, NT, smem, st>>>(work, PP, P, mu1, lam, scale, tw, h->skip, rinv);
    k_nstrided<T, N, false, 3><<<grid, NT, smem, st>>>(work, P, PP, mu1, lam, scale, tw, h->skip);
    k_nxinv<T, N, 3><<<grid, NT, smem, st>>>(work, sa.keep || sa.out_user == nullptr, sa.out_user, sa.aux, sa.beta,
                                              sa.gamma, tw, h->skip);
    KFBI_CHECK_LAUNCH_N(5);
  } else {
    if ((rc = prep(k_nxfwd<T, N, 2>, smem))) return rc;
    if ((rc = prep(k_nstrided<T, N, true, 2>, smem))) return rc;
    if ((rc = prep(k_nxinv<T, N, 2>, smem))) return rc;
    k_nxfwd<T, N, 2><<<grid, NT, smem, st>>>(work, sa.src, sa.alpha, sa.src32, sa.corr, t.irr, t.line_start, tw,
                                                h->skip);
    k_nstrided<T, N, true, 2><<<grid, NT, smem, st>>>(work, P, 0, mu1, lam, scale, tw, h->skip, rinv);
    k_nxinv<T, N, 2><<<grid, NT, smem, st>>>(work, sa.keep || sa.out_user == nullptr, sa.out_user, sa.aux, sa.beta,
                                              sa.gamma, tw, h->skip);
    KFBI_CHECK_LAUNCH_N(3);
  }
  return KFBI_OK;
}

template <typename T>
int box_solve_neumann(kfbi_handle* h, const SolveArgs& sa, T* work, const T* mu1, const T* tw) {
  if (!(sa.lambda > 0.0)) {
    set_error("the Neumann box needs lambda > 0 (no Green's function of the Poisson operator exists)");
    return KFBI_ERR_ARG;
  }
  switch (h->grid.N) {
    case 8: return run_solve_neumann<T, 8>(h, sa, work, mu1, tw);
    case 16: return run_solve_neumann<T, 16>(h, sa, work, mu1, tw);
    case 32: return run_solve_neumann<T, 32>(h, sa, work, mu1, tw);
    case 64: return run_solve_neumann<T, 64>(h, sa, work, mu1, tw);
    case 128: return run_solve_neumann<T, 128>(h, sa, work, mu1, tw);
    case 256: return run_solve_neumann<T, 256>(h, sa, work, mu1, tw);
    case 384: return run_solve_neumann<T, 384>(h, sa, work, mu1, tw);
    case 512: return run_solve_neumann<T, 512>(h, sa, work, mu1, tw);
    default:
      set_error("unsupported grid size N=%d", h->grid.N);
      return KFBI_ERR_ARG;
  }
}

}  // namespace

// TMA descriptors of the padded float32 grid for the strided passes (3-D,
// 32 <= N <= 256): boxes of 32 x-values by N rows along y or along z.
int make_tma_maps(kfbi_handle* h) {
  h->tma = false;
  {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
      h->sms = sms;
    cudaGetLastError();
  }
  const int N = h->grid.N;
  if (h->grid.dim != 3 || N < TMA_W || N > 256) return KFBI_OK;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || fn == nullptr) {
    cudaGetLastError();
    return KFBI_OK;  // no tensor maps: the strided passes keep their plain loads
  }
  auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  const cuuint64_t dims[3] = {(cuuint64_t)N, (cuuint64_t)N, (cuuint64_t)N};
  const cuuint64_t strides[2] = {(cuuint64_t)N * sizeof(float), (cuuint64_t)N * N * sizeof(float)};
  const cuuint32_t estr[3] = {1, 1, 1};
  const cuuint32_t box_y[3] = {(cuuint32_t)TMA_W, (cuuint32_t)N, 1};
  const cuuint32_t box_z[3] = {(cuuint32_t)TMA_W, 1, (cuuint32_t)N};
  CUresult r1 = encode(&h->tmap_y32, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, h->w.grid32, dims, strides, box_y, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  CUresult r2 = encode(&h->tmap_z32, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, h->w.grid32, dims, strides, box_z, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r1 != CUDA_SUCCESS || r2 != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d, %d)", (int)r1, (int)r2);
    return KFBI_ERR_CUDA;
  }
  h->tma = true;
  if (h->w.grid32b != nullptr) {
    r1 = encode(&h->tmap_y32b, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, h->w.grid32b, dims, strides, box_y, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    r2 = encode(&h->tmap_z32b, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, h->w.grid32b, dims, strides, box_z, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    h->tma_b = r1 == CUDA_SUCCESS && r2 == CUDA_SUCCESS;
  }
  // fused x-y passes need cluster launches (a cluster of N/32 blocks per
  // plane).  They pay off only for small planes: measured per float32 solve
  // (CUDA events, back-to-back) 18.8 against 24.4 us at 64^3, 48.4 against
  // 47.7 us at 128^3 and 211 against 172 us at 256^3, where the separate
  // passes are bound by the transforms' instruction issue with the grid in
  // L2, and the fused blocks add two cluster barriers and the exchange.
  int dev = 0, cl = 0;
  cudaGetDevice(&dev);
  if (N <= 64 && cudaDeviceGetAttribute(&cl, cudaDevAttrClusterLaunch, dev) == cudaSuccess && cl) h->xy_fused = true;
  cudaGetLastError();
  return KFBI_OK;
}

int transform_pass(kfbi_handle* h, int precision, int pass, double lambda) {
  if (precision == KFBI_FP64) return dispatch_pass<double>(h, pass, lambda, h->w.grid64, h->t.mu, h->t.tw64);
  return dispatch_pass<float>(h, pass, lambda, h->w.grid32, h->t.mu32, h->t.tw32);
}

int dst_supported(int N) {
  return N == 8 || N == 16 || N == 32 || N == 64 || N == 128 || N == 256 || N == 384 || N == 512;
}

int box_solve64(kfbi_handle* h, const SolveArgs& a, double* work) {
  if (h->grid.bc == KFBI_BOX_NEUMANN) return box_solve_neumann<double>(h, a, work, h->t.mu, h->t.tw64);
  return dispatch<double>(h, a, work, h->t.mu, h->t.tw64);
}

int box_solve32(kfbi_handle* h, const SolveArgs& a, float* work) {
  if (h->grid.bc == KFBI_BOX_NEUMANN) return box_solve_neumann<float>(h, a, work, h->t.mu32, h->t.tw32);
  return dispatch<float>(h, a, work, h->t.mu32, h->t.tw32);
}

namespace {
template <typename T>
int dispatch_coupled(kfbi_handle* h, const SolveArgs& si, const SolveArgs& se, const Coupling& cp, T* wa, T* wb,
                     const T* mu1T, const T* tw) {
  switch (h->grid.N) {
    case 16: return run_solve_coupled<T, 16>(h, si, se, cp, wa, wb, mu1T, tw);
    case 32: return run_solve_coupled<T, 32>(h, si, se, cp, wa, wb, mu1T, tw);
    case 64: return run_solve_coupled<T, 64>(h, si, se, cp, wa, wb, mu1T, tw);
    case 128: return run_solve_coupled<T, 128>(h, si, se, cp, wa, wb, mu1T, tw);
    case 256: return run_solve_coupled<T, 256>(h, si, se, cp, wa, wb, mu1T, tw);
    case 384: return run_solve_coupled<T, 384>(h, si, se, cp, wa, wb, mu1T, tw);
    case 512: return run_solve_coupled<T, 512>(h, si, se, cp, wa, wb, mu1T, tw);
    default:
      set_error("unsupported grid size N=%d for the coupled solve", h->grid.N);
      return KFBI_ERR_ARG;
  }
}
}  // namespace

int box_solve_coupled64(kfbi_handle* h, const SolveArgs& si, const SolveArgs& se, const Coupling& cp, double* wa,
                        double* wb) {
  return dispatch_coupled<double>(h, si, se, cp, wa, wb, h->t.mu, h->t.tw64);
}

int box_solve_coupled32(kfbi_handle* h, const SolveArgs& si, const SolveArgs& se, const Coupling& cp, float* wa,
                        float* wb) {
  return dispatch_coupled<float>(h, si, se, cp, wa, wb, h->t.mu32, h->t.tw32);
}

namespace {
// an mbarrier that nothing ever completes, polled with the transform
// kernels' bounded wait: the poll cap must end the wait and raise the flag
__global__ void k_selftest_wait(long cap, int* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  bool ok = false;
  for (long it = 0; it < cap; ++it)
    if (mbar_try_wait(&bar, 0u)) {
      ok = true;
      break;
    }
  if (!ok && threadIdx.x == 0) atomicOr(err, DEVERR_TIMEOUT);
}
}  // namespace

}  // namespace kfbi

extern "C" int kfbi_selftest_bounded_wait(int polls, int* timed_out, double* ms) {
  using namespace kfbi;
  if (polls < 1 || polls > (1 << 20) || !timed_out) {
    set_error("polls must be in 1 .. 2^20");
    return KFBI_ERR_ARG;
  }
  int* err = nullptr;
  KFBI_CUDA(cudaMalloc(&err, sizeof(int)));
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaMemset(err, 0, sizeof(int));
  cudaEventRecord(a);
  k_selftest_wait<<<1, 32>>>((long)polls, err);
  cudaEventRecord(b);
  const cudaError_t e = cudaEventSynchronize(b);
  int herr = 0;
  if (e == cudaSuccess) cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
  float t = 0.0f;
  cudaEventElapsedTime(&t, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(err);
  if (e != cudaSuccess) {
    set_error("self-test launch failed: %s", cudaGetErrorString(e));
    return KFBI_ERR_CUDA;
  }
  *timed_out = (herr & DEVERR_TIMEOUT) ? 1 : 0;
  if (ms) *ms = t;
  KFBI_COUNT(1);
  return KFBI_OK;
}
