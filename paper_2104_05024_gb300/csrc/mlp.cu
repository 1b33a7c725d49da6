// Point-wise MLP of the learned density warm start (not in the paper): 9
// features per interface node -- the history projection psi_F, its residual
// r_F and the right-hand side g^n, each divided by its root mean square over
// the nodes, then the node and its unit normal -- through 4 hidden layers of
// width 128 with SiLU to one output o; the initial density is
// psi_L = psi_F + 2 gamma r_F + rms(r_F) (s_out o + m_out).  bfloat16 weights
// and activations, float32 accumulation on the tensor cores (wmma bf16
// 16x16x16 fragments), float32 master weights with Adam.  The network only
// supplies GMRES's initial guess; the solver tolerance still fixes the
// converged density.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <mma.h>

#include <cmath>
#include <vector>

#include "internal.cuh"

using bf16 = __nv_bfloat16;

namespace kfbi {
namespace {

constexpr int NIN = 9, KIN = 16, WID = 128, NL = 5;  // 4 hidden + output
constexpr int TILE = 64;

struct Offsets {
  size_t w[NL], b[NL], total;
  Offsets() {
    const int in[NL] = {NIN, WID, WID, WID, WID};
    const int out[NL] = {WID, WID, WID, WID, 1};
    size_t o = 0;
    for (int l = 0; l < NL; ++l) {
      w[l] = o;
      o += (size_t)in[l] * out[l];
      b[l] = o;
      o += out[l];
    }
    total = o;
  }
};

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + expf(-z)); }
__device__ __forceinline__ float dsilu_f(float z) {
  const float s = 1.0f / (1.0f + expf(-z));
  return s * (1.0f + z * (1.0f - s));
}

// C[M x N] (=, or += by atomics for split-K) A[M x K] B[K x N]; bf16 operands,
// float32 accumulation.  A row-major: A[m lda + k]; col-major: A[k lda + m].
// B row-major: B[k ldb + n]; col-major: B[n ldb + k].  M, N, K multiples of 16.
template <typename LA, typename LB, bool ATOMIC>
__global__ void __launch_bounds__(128) k_gemm(const bf16* __restrict__ A, int lda, const bf16* __restrict__ B, int ldb,
                                              float* __restrict__ C, int ldc, int M, int N, int K, int kchunk) {
  using namespace nvcuda;
  const int warp = threadIdx.x >> 5, wy = warp >> 1, wx = warp & 1;
  const int m0 = blockIdx.y * TILE + wy * 32, n0 = blockIdx.x * TILE + wx * 32;
  const int k0 = blockIdx.z * kchunk;
  const int k1 = min(K, k0 + kchunk);
  wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) wmma::fill_fragment(acc[i][j], 0.0f);
  const bool a_row = std::is_same<LA, wmma::row_major>::value;
  const bool b_row = std::is_same<LB, wmma::row_major>::value;
  for (int k = k0; k < k1; k += 16) {
    wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, LA> fa[2];
    wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, LB> fb[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int m = m0 + i * 16;
      if (m < M) wmma::load_matrix_sync(fa[i], a_row ? A + (size_t)m * lda + k : A + (size_t)k * lda + m, lda);
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int n = n0 + j * 16;
      if (n < N) wmma::load_matrix_sync(fb[j], b_row ? B + (size_t)k * ldb + n : B + (size_t)n * ldb + k, ldb);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j)
        if (m0 + i * 16 < M && n0 + j * 16 < N) wmma::mma_sync(acc[i][j], fa[i], fb[j], acc[i][j]);
  }
  __shared__ float stage[4][16 * 16];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int m = m0 + i * 16, n = n0 + j * 16;
      if (m >= M || n >= N) continue;
      if (!ATOMIC) {
        wmma::store_matrix_sync(C + (size_t)m * ldc + n, acc[i][j], ldc, wmma::mem_row_major);
      } else {
        wmma::store_matrix_sync(stage[warp], acc[i][j], 16, wmma::mem_row_major);
        __syncwarp();
        for (int e = threadIdx.x & 31; e < 256; e += 32)
          atomicAdd(C + (size_t)(m + e / 16) * ldc + n + (e % 16), stage[warp][e]);
        __syncwarp();
      }
    }
}

// normalised bfloat16 features [Bp][16] from raw float32 features [B][9]
__global__ void k_feat_raw(const float* __restrict__ F, int B, int Bp, const float* __restrict__ norm, bf16* X) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Bp * KIN) return;
  const int b = i / KIN, c = i % KIN;
  float v = 0.0f;
  if (b < B && c < NIN) v = (F[(size_t)b * NIN + c] - norm[c]) / norm[NIN + c];
  X[i] = __float2bfloat16_rn(v);
}

// raw input row of node b from the solver state: psi_F, r_F and g^n each
// scaled by the inverse root mean square rsqrt(sq[k] / B) (sq = their sums
// of squares over the B nodes), then the node and its unit normal
__device__ __forceinline__ void raw_features(const double* __restrict__ psiF, const double* __restrict__ rF,
                                             const double* __restrict__ g, const double* __restrict__ sq,
                                             const double* __restrict__ nodes, const double* __restrict__ normals,
                                             int B, int b, float* f) {
  const double s0 = rsqrt(fmax(sq[0] / B, 1e-300)), s1 = rsqrt(fmax(sq[1] / B, 1e-300)),
               s2 = rsqrt(fmax(sq[2] / B, 1e-300));
  f[0] = (float)(psiF[b] * s0);
  f[1] = (float)(rF[b] * s1);
  f[2] = (float)(g[b] * s2);
  for (int k = 0; k < 3; ++k) {
    f[3 + k] = (float)nodes[(size_t)b * 3 + k];
    f[6 + k] = (float)normals[(size_t)b * 3 + k];
  }
}

// normalised bfloat16 network input rows [Bp][16] from the solver state
__global__ void k_feat_proj(const double* __restrict__ psiF, const double* __restrict__ rF,
                            const double* __restrict__ g, const double* __restrict__ sq,
                            const double* __restrict__ nodes, const double* __restrict__ normals, int B, int Bp,
                            const float* __restrict__ norm, bf16* X) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= Bp) return;
  float f[NIN];
  if (b < B) raw_features(psiF, rF, g, sq, nodes, normals, B, b, f);
  for (int c = 0; c < KIN; ++c) {
    float v = 0.0f;
    if (b < B && c < NIN) v = (f[c] - norm[c]) / norm[NIN + c];
    X[(size_t)b * KIN + c] = __float2bfloat16_rn(v);
  }
}

// training rows of one solve: raw features F[b][9] (the rows the network
// reads at inference) and the target T[b] = (psi - psi_F - 2 gamma r_F) /
// rms(r_F), the correction of the projection start in units of rms(r_F)
__global__ void k_train_rows(const double* __restrict__ psi, const double* __restrict__ psiF,
                             const double* __restrict__ rF, const double* __restrict__ g,
                             const double* __restrict__ sq, const double* __restrict__ nodes,
                             const double* __restrict__ normals, int B, double two_gamma, float* __restrict__ F,
                             float* __restrict__ T) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  float f[NIN];
  raw_features(psiF, rF, g, sq, nodes, normals, B, b, f);
  for (int c = 0; c < NIN; ++c) F[(size_t)b * NIN + c] = f[c];
  const double s1 = rsqrt(fmax(sq[1] / B, 1e-300));
  T[b] = (float)((psi[b] - psiF[b] - two_gamma * rF[b]) * s1);
}

// normalisation moments of the training rows, one block per column (the 9
// features of F [n][9], then the targets T [n]): mean and sample standard
// deviation in float64, two passes (mean first, then the squared deviations);
// a spread below 1e-12 (features) or 1e-30 (target) becomes 1.  out[c] =
// mean, out[10 + c] = std.
__global__ void __launch_bounds__(256) k_moments(const float* __restrict__ F, const float* __restrict__ T, int n,
                                                 double* __restrict__ out) {
  const int c = blockIdx.x;
  __shared__ double red[256];
  auto value = [&](int i) -> double { return c < NIN ? (double)F[(size_t)i * NIN + c] : (double)T[i]; };
  auto block_sum = [&](double v) -> double {
    red[threadIdx.x] = v;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
      if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
      __syncthreads();
    }
    const double t = red[0];
    __syncthreads();
    return t;
  };
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += value(i);
  const double mean = block_sum(acc) / n;
  acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double d = value(i) - mean;
    acc += d * d;
  }
  const double var = n > 1 ? block_sum(acc) / (n - 1) : 0.0;
  if (threadIdx.x == 0) {
    const double sd = sqrt(var);
    out[c] = mean;
    out[10 + c] = sd > (c < NIN ? 1e-12 : 1e-30) ? sd : 1.0;
  }
}

__global__ void k_bias_act(float* __restrict__ Z, const float* __restrict__ bias, bf16* __restrict__ A, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float z = Z[i] + bias[i % WID];
  Z[i] = z;
  A[i] = __float2bfloat16_rn(silu_f(z));
}

// o_b = sum_j A3[b][j] w4[j] + b4 (one warp per row)
__global__ void k_out(const bf16* __restrict__ A, const bf16* __restrict__ w4, const float* __restrict__ b4, float* o,
                      int Bp) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= Bp) return;
  float acc = 0.0f;
  for (int j = lane; j < WID; j += 32) acc += __bfloat162float(A[(size_t)row * WID + j]) * __bfloat162float(w4[j]);
  for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
  if (lane == 0) o[row] = acc + b4[0];
}

// output-layer delta d4 = (o - t)/B and the loss partial sums; the raw
// targets T are normalised first, t = (T - m_out) / s_out (norm[18], norm[19])
__global__ void k_delta_out(const float* __restrict__ o, const float* __restrict__ T, const float* __restrict__ norm,
                            int B, int Bp, float* d4, float* loss) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  float r = 0.0f;
  if (b < B) r = o[b] - (T[b] - norm[2 * NIN]) / norm[2 * NIN + 1];
  if (b < Bp) d4[b] = r / (float)B;
  float sq = r * r;
  for (int s = 16; s > 0; s >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, s);
  if ((threadIdx.x & 31) == 0 && sq != 0.0f) atomicAdd(loss, sq);
}

// gradients of the output layer and delta of the last hidden layer
__global__ void k_back_out(const float* __restrict__ d4, const bf16* __restrict__ A3, const float* __restrict__ Z3,
                           const bf16* __restrict__ w4, float* gw4, float* gb4, float* d, bf16* db, int Bp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Bp * WID) return;
  const int b = i / WID, j = i % WID;
  const float dq = __bfloat162float(__float2bfloat16_rn(d4[b]));
  atomicAdd(gw4 + j, dq * __bfloat162float(A3[i]));
  if (j == 0 && d4[b] != 0.0f) atomicAdd(gb4, d4[b]);
  const float v = dq * __bfloat162float(w4[j]) * dsilu_f(Z3[i]);
  d[i] = v;
  db[i] = __float2bfloat16_rn(v);
}

__global__ void k_dsilu(const float* __restrict__ da, const float* __restrict__ Z, float* d, bf16* db, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float v = da[i] * dsilu_f(Z[i]);
  d[i] = v;
  db[i] = __float2bfloat16_rn(v);
}

// bias gradient: column sums of d [Bp][128]
__global__ void k_colsum(const float* __restrict__ d, int Bp, float* g) {
  const int j = threadIdx.x % WID;
  float acc = 0.0f;
  for (int b = blockIdx.x * (blockDim.x / WID) + threadIdx.x / WID; b < Bp; b += gridDim.x * (blockDim.x / WID))
    acc += d[(size_t)b * WID + j];
  atomicAdd(g + j, acc);
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int n, float lr, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

// bfloat16 weight copies (W0 padded from 9 to 16 input columns)
__global__ void k_refresh(const float* __restrict__ p, Offsets off, bf16* W0, bf16* W1, bf16* W2, bf16* W3, bf16* w4) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < WID * KIN) {
    const int r = i / KIN, c = i % KIN;
    W0[i] = __float2bfloat16_rn(c < NIN ? p[off.w[0] + (size_t)r * NIN + c] : 0.0f);
  }
  if (i < WID * WID) {
    W1[i] = __float2bfloat16_rn(p[off.w[1] + i]);
    W2[i] = __float2bfloat16_rn(p[off.w[2] + i]);
    W3[i] = __float2bfloat16_rn(p[off.w[3] + i]);
  }
  if (i < WID) w4[i] = __float2bfloat16_rn(p[off.w[4] + i]);
}

// W0 gradient: columns 0..8 of the padded [128][16] product
__global__ void k_unpad_w0(const float* __restrict__ g16, float* gw0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < WID * NIN) gw0[i] += g16[(i / NIN) * KIN + i % NIN];
}

// psi_L = psi_F + 2 gamma r_F + rms(r_F) * (s_out o + m_out), the network
// output denormalised in float32
__global__ void k_predict(const double* __restrict__ psiF, const double* __restrict__ rF,
                          const double* __restrict__ sq, double two_gamma, const float* __restrict__ o,
                          const float* __restrict__ norm, double* out, int B) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B) {
    const double sr = sqrt(sq[1] / B);
    out[b] = psiF[b] + two_gamma * rF[b] + sr * (double)(norm[2 * NIN + 1] * o[b] + norm[2 * NIN]);
  }
}

// Inference of the whole network in one persistent kernel (the training
// path keeps the layer-by-layer kernels, whose activations the backward pass
// needs).  The bfloat16 weights are staged in shared memory once per block;
// per tile of 64 rows each layer runs on the tensor cores from the tile's
// activations in shared memory, the float32 products go to a shared staging
// tile, and the epilogue adds the bias, applies SiLU and rounds to bfloat16
// in place; the output layer is one warp dot product per row.  Same
// operations and summation order per element as the layer-by-layer path.
constexpr int IR = 64;                      // rows per tile
constexpr int LDW = WID + 8, LDX = KIN + 8;  // padded bf16 leading dimensions
constexpr int LDS = WID + 4;                 // padded float32 staging
constexpr size_t INFER_SMEM = (size_t)3 * WID * LDW * 2 + (size_t)WID * LDX * 2 + (size_t)IR * LDW * 2 +
                              (size_t)IR * LDX * 2 + (size_t)IR * LDS * 4 + (size_t)4 * WID * 4 + (size_t)WID * 4;

__global__ void __launch_bounds__(256, 1) k_mlp_infer(const bf16* __restrict__ X, int Bp, const bf16* __restrict__ W0,
                                                      const bf16* __restrict__ W1, const bf16* __restrict__ W2,
                                                      const bf16* __restrict__ W3, const bf16* __restrict__ w4,
                                                      const float* __restrict__ p, Offsets off, float* __restrict__ o) {
  using namespace nvcuda;
  extern __shared__ __align__(128) unsigned char sm_infer[];
  bf16* sW = reinterpret_cast<bf16*>(sm_infer);  // 3 x [WID][LDW], B[n][k]
  bf16* sW0 = sW + 3 * WID * LDW;                 // [WID][LDX]
  bf16* sA = sW0 + WID * LDX;                     // [IR][LDW]
  bf16* sX = sA + IR * LDW;                       // [IR][LDX]
  float* sZ = reinterpret_cast<float*>(sX + IR * LDX);  // [IR][LDS]
  float* sB = sZ + IR * LDS;                      // [4][WID]
  float* sw4 = sB + 4 * WID;                      // [WID]
  const int tid = threadIdx.x;
  const bf16* Wg[3] = {W1, W2, W3};
  for (int l = 0; l < 3; ++l)
    for (int i = tid; i < WID * WID / 8; i += blockDim.x) {
      const int n = i / (WID / 8), q = i % (WID / 8);
      *reinterpret_cast<uint4*>(sW + (size_t)l * WID * LDW + n * LDW + 8 * q) =
          *reinterpret_cast<const uint4*>(Wg[l] + (size_t)n * WID + 8 * q);
    }
  for (int i = tid; i < WID * KIN / 8; i += blockDim.x) {
    const int n = i / (KIN / 8), q = i % (KIN / 8);
    *reinterpret_cast<uint4*>(sW0 + n * LDX + 8 * q) = *reinterpret_cast<const uint4*>(W0 + (size_t)n * KIN + 8 * q);
  }
  for (int i = tid; i < 4 * WID; i += blockDim.x) sB[i] = p[off.b[i / WID] + i % WID];
  for (int i = tid; i < WID; i += blockDim.x) sw4[i] = __bfloat162float(w4[i]);
  const float b4 = p[off.b[4]];
  const int warp = tid >> 5, lane = tid & 31;
  const int rb = warp & 3, cb = (warp >> 2) * 4;  // 16-row block, four 16-column blocks
  for (int tile = blockIdx.x; tile < Bp / IR; tile += gridDim.x) {
    for (int i = tid; i < IR * KIN / 8; i += blockDim.x) {
      const int r = i / (KIN / 8), q = i % (KIN / 8);
      *reinterpret_cast<uint4*>(sX + r * LDX + 8 * q) =
          *reinterpret_cast<const uint4*>(X + ((size_t)tile * IR + r) * KIN + 8 * q);
    }
    __syncthreads();
    for (int l = 0; l < 4; ++l) {
      const bf16* Ain = l == 0 ? sX : sA;
      const int lda = l == 0 ? LDX : LDW, ldb = lda, K = l == 0 ? KIN : WID;
      const bf16* Bw = l == 0 ? sW0 : sW + (size_t)(l - 1) * WID * LDW;
      wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) wmma::fill_fragment(acc[j], 0.0f);
      for (int k0 = 0; k0 < K; k0 += 16) {
        wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, wmma::row_major> fa;
        wmma::load_matrix_sync(fa, Ain + rb * 16 * lda + k0, lda);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, wmma::col_major> fb;
          wmma::load_matrix_sync(fb, Bw + (cb + j) * 16 * ldb + k0, ldb);
          wmma::mma_sync(acc[j], fa, fb, acc[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j)
        wmma::store_matrix_sync(sZ + rb * 16 * LDS + (cb + j) * 16, acc[j], LDS, wmma::mem_row_major);
      __syncthreads();  // every warp has read its inputs and written its products
      for (int i = tid; i < IR * WID; i += blockDim.x) {
        const int r = i / WID, c = i % WID;
        sA[r * LDW + c] = __float2bfloat16_rn(silu_f(sZ[r * LDS + c] + sB[l * WID + c]));
      }
      __syncthreads();
    }
    for (int r = warp; r < IR; r += (int)(blockDim.x >> 5)) {
      float acc = 0.0f;
      for (int j = lane; j < WID; j += 32) acc += __bfloat162float(sA[r * LDW + j]) * sw4[j];
      for (int sft = 16; sft > 0; sft >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, sft);
      if (lane == 0) o[(size_t)tile * IR + r] = acc + b4;
    }
    __syncthreads();  // the next tile overwrites sX and sA
  }
}

}  // namespace
}  // namespace kfbi

struct kfbi_mlp {
  kfbi::Offsets off;
  int bmax = 0, bpmax = 0;
  cudaStream_t stream = nullptr;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr, *norm = nullptr;
  bf16 *W0 = nullptr, *W[3] = {nullptr, nullptr, nullptr}, *w4 = nullptr;
  bf16* X = nullptr;
  bf16* A[4] = {nullptr, nullptr, nullptr, nullptr};
  float* Z[4] = {nullptr, nullptr, nullptr, nullptr};
  float *o = nullptr, *d4 = nullptr, *d = nullptr, *da = nullptr, *g16 = nullptr, *loss = nullptr;
  bf16* db = nullptr;
  float* dump_d = nullptr;   // kfbi_mlp_layers: per-layer deltas go here (else null)
  float* dump_d4 = nullptr;
  int step = 0;
  std::vector<void*> allocs;
};

namespace kfbi {
namespace {

template <typename T>
int malloc_mlp(kfbi_mlp* m, T** p, size_t n) {
  if (cudaMalloc((void**)p, sizeof(T) * (n ? n : 1)) != cudaSuccess) {
    set_error("cudaMalloc failed for the MLP workspace");
    return KFBI_ERR_OOM;
  }
  m->allocs.push_back((void*)*p);
  return KFBI_OK;
}

int blocks(size_t n, int bs) { return (int)((n + bs - 1) / bs); }

// forward over rows already placed in m->X; leaves o, Z, A
int mlp_forward_rows(kfbi_mlp* m, int Bp) {
  using namespace nvcuda;
  cudaStream_t st = m->stream;
  const dim3 g(WID / TILE, Bp / TILE, 1);
  k_gemm<wmma::row_major, wmma::col_major, false><<<g, 128, 0, st>>>(m->X, KIN, m->W0, KIN, m->Z[0], WID, Bp, WID, KIN, KIN);
  k_bias_act<<<blocks((size_t)Bp * WID, 256), 256, 0, st>>>(m->Z[0], m->p + m->off.b[0], m->A[0], Bp * WID);
  for (int l = 1; l < 4; ++l) {
    k_gemm<wmma::row_major, wmma::col_major, false><<<g, 128, 0, st>>>(m->A[l - 1], WID, m->W[l - 1], WID, m->Z[l], WID,
                                                                       Bp, WID, WID, WID);
    k_bias_act<<<blocks((size_t)Bp * WID, 256), 256, 0, st>>>(m->Z[l], m->p + m->off.b[l], m->A[l], Bp * WID);
  }
  k_out<<<blocks((size_t)Bp * 32, 256), 256, 0, st>>>(m->A[3], m->w4, m->p + m->off.b[4], m->o, Bp);
  KFBI_CHECK_LAUNCH_N(9);
  return KFBI_OK;
}

// inference over rows already placed in m->X (Bp a multiple of 64): m->o
int mlp_infer_rows(kfbi_mlp* m, int Bp) {
  static bool opted = false;
  if (!opted) {
    if (cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)INFER_SMEM) !=
        cudaSuccess) {
      set_error("cudaFuncSetAttribute failed for the inference kernel");
      return KFBI_ERR_CUDA;
    }
    opted = true;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int tiles = Bp / IR;
  const int grid = tiles < sms ? tiles : sms;
  k_mlp_infer<<<grid, 256, INFER_SMEM, m->stream>>>(m->X, Bp, m->W0, m->W[0], m->W[1], m->W[2], m->w4, m->p, m->off,
                                                    m->o);
  KFBI_CHECK_LAUNCH();
  return KFBI_OK;
}

int mlp_prepare_raw(kfbi_mlp* m, const float* F, int B, int* Bp) {
  if (B < 1 || B > m->bmax) {
    set_error("batch %d outside 1..%d", B, m->bmax);
    return KFBI_ERR_ARG;
  }
  *Bp = (B + TILE - 1) / TILE * TILE;
  k_feat_raw<<<blocks((size_t)*Bp * KIN, 256), 256, 0, m->stream>>>(F, B, *Bp, m->norm, m->X);
  KFBI_CHECK_LAUNCH();
  return KFBI_OK;
}

// gradients of 0.5 mean (o - t)^2 into m->g (rows already forwarded)
int mlp_backward(kfbi_mlp* m, const float* t, int B, int Bp) {
  using namespace nvcuda;
  cudaStream_t st = m->stream;
  const Offsets& off = m->off;
  KFBI_CUDA(cudaMemsetAsync(m->g, 0, sizeof(float) * off.total, st));
  KFBI_CUDA(cudaMemsetAsync(m->loss, 0, sizeof(float), st));
  KFBI_CUDA(cudaMemsetAsync(m->g16, 0, sizeof(float) * WID * KIN, st));
  k_delta_out<<<blocks(Bp, 256), 256, 0, st>>>(m->o, t, m->norm, B, Bp, m->d4, m->loss);
  k_back_out<<<blocks((size_t)Bp * WID, 256), 256, 0, st>>>(m->d4, m->A[3], m->Z[3], m->w4, m->g + off.w[4],
                                                            m->g + off.b[4], m->d, m->db, Bp);
  int launched = 2;
  if (m->dump_d4) KFBI_CUDA(cudaMemcpyAsync(m->dump_d4, m->d4, sizeof(float) * B, cudaMemcpyDeviceToDevice, st));
  const int kch = 1024;
  for (int l = 3; l >= 0; --l) {
    if (m->dump_d)
      KFBI_CUDA(cudaMemcpyAsync(m->dump_d + (size_t)(3 - l) * B * WID, m->d, sizeof(float) * B * WID,
                                cudaMemcpyDeviceToDevice, st));
    // weight gradient d^T A_{l-1} (split over rows, float32 atomics)
    const dim3 gg(l == 0 ? 1 : WID / TILE, WID / TILE, (Bp + kch - 1) / kch);
    if (l > 0) {
      k_gemm<wmma::col_major, wmma::row_major, true><<<gg, 128, 0, st>>>(m->db, WID, m->A[l - 1], WID, m->g + off.w[l],
                                                                         WID, WID, WID, Bp, kch);
    } else {
      k_gemm<wmma::col_major, wmma::row_major, true><<<gg, 128, 0, st>>>(m->db, WID, m->X, KIN, m->g16, KIN, WID, KIN,
                                                                         Bp, kch);
      k_unpad_w0<<<blocks(WID * NIN, 256), 256, 0, st>>>(m->g16, m->g + off.w[0]);
      ++launched;
    }
    k_colsum<<<64, 256, 0, st>>>(m->d, Bp, m->g + off.b[l]);
    launched += 2;
    if (l > 0) {
      const dim3 g2(WID / TILE, Bp / TILE, 1);
      k_gemm<wmma::row_major, wmma::row_major, false><<<g2, 128, 0, st>>>(m->db, WID, m->W[l - 1], WID, m->da, WID, Bp,
                                                                          WID, WID, WID);
      k_dsilu<<<blocks((size_t)Bp * WID, 256), 256, 0, st>>>(m->da, m->Z[l - 1], m->d, m->db, Bp * WID);
      launched += 2;
    }
  }
  KFBI_CHECK_LAUNCH_N(launched);
  return KFBI_OK;
}

int mlp_refresh(kfbi_mlp* m) {
  k_refresh<<<blocks(WID * WID, 256), 256, 0, m->stream>>>(m->p, m->off, m->W0, m->W[0], m->W[1], m->W[2], m->w4);
  KFBI_CHECK_LAUNCH();
  return KFBI_OK;
}

}  // namespace

// warm start used by bidomain_step: psi_L from the projection psi_F, its
// residual r_F and g (sq = their sums of squares) through the network
int mlp_warmstart(kfbi_mlp* m, cudaStream_t st, const double* psiF, const double* rF, const double* g,
                  const double* sq, const double* nodes, const double* normals, int M, double two_gamma,
                  double* out) {
  if (M > m->bmax) {
    set_error("warm start: %d nodes exceed the network's batch capacity %d", M, m->bmax);
    return KFBI_ERR_ARG;
  }
  cudaStream_t saved = m->stream;
  m->stream = st;
  const int Bp = (M + TILE - 1) / TILE * TILE;
  k_feat_proj<<<blocks(Bp, 128), 128, 0, st>>>(psiF, rF, g, sq, nodes, normals, M, Bp, m->norm, m->X);
  KFBI_CHECK_LAUNCH();
  int rc = mlp_infer_rows(m, Bp);
  if (rc == KFBI_OK) {
    k_predict<<<blocks(M, 256), 256, 0, st>>>(psiF, rF, sq, two_gamma, m->o, m->norm, out, M);
    KFBI_CHECK_LAUNCH();
  }
  m->stream = saved;
  return rc;
}

int launch_train_rows(cudaStream_t st, const double* psi, const double* psiF, const double* rF, const double* g,
                      const double* sq, const double* nodes, const double* normals, int M, double two_gamma, float* F,
                      float* T) {
  k_train_rows<<<blocks(M, 256), 256, 0, st>>>(psi, psiF, rF, g, sq, nodes, normals, M, two_gamma, F, T);
  KFBI_CHECK_LAUNCH();
  return KFBI_OK;
}

}  // namespace kfbi

using namespace kfbi;

extern "C" {

int kfbi_mlp_fit_norm(const float* F_dev, const float* T_dev, int n, void* stream, float* norm_host) {
  if (!F_dev || !T_dev || !norm_host || n < 1) {
    set_error("null argument or no rows");
    return KFBI_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  double* out = nullptr;
  KFBI_CUDA(cudaMalloc((void**)&out, sizeof(double) * 20));
  k_moments<<<NIN + 1, 256, 0, st>>>(F_dev, T_dev, n, out);
  double h[20];
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(out);
  if (e != cudaSuccess) {
    set_error("normalisation moments failed: %s", cudaGetErrorString(e));
    return KFBI_ERR_CUDA;
  }
  KFBI_COUNT(1);
  for (int c = 0; c < NIN; ++c) {
    norm_host[c] = (float)h[c];
    norm_host[NIN + c] = (float)h[10 + c];
  }
  norm_host[2 * NIN] = (float)h[NIN];
  norm_host[2 * NIN + 1] = (float)h[10 + NIN];
  return KFBI_OK;
}

int kfbi_mlp_create(const float* params_host, const float* norm_host, int max_batch, void* stream, kfbi_mlp** out) {
  if (!params_host || !norm_host || !out || max_batch < 1) {
    set_error("null argument or empty batch");
    return KFBI_ERR_ARG;
  }
  kfbi_mlp* m = new kfbi_mlp();
  m->stream = (cudaStream_t)stream;
  m->bmax = max_batch;
  m->bpmax = (max_batch + TILE - 1) / TILE * TILE;
  const size_t P = m->off.total, Bp = m->bpmax;
  int rc = 0;
  auto fail = [&](int code) {
    kfbi_mlp_destroy(m);
    return code;
  };
  if ((rc = malloc_mlp(m, &m->p, P)) || (rc = malloc_mlp(m, &m->g, P)) || (rc = malloc_mlp(m, &m->m, P)) ||
      (rc = malloc_mlp(m, &m->v, P)) || (rc = malloc_mlp(m, &m->norm, 2 * NIN + 2)) ||
      (rc = malloc_mlp(m, &m->W0, WID * KIN)) || (rc = malloc_mlp(m, &m->w4, WID)) ||
      (rc = malloc_mlp(m, &m->X, Bp * KIN)) || (rc = malloc_mlp(m, &m->o, Bp)) || (rc = malloc_mlp(m, &m->d4, Bp)) ||
      (rc = malloc_mlp(m, &m->d, Bp * WID)) || (rc = malloc_mlp(m, &m->da, Bp * WID)) ||
      (rc = malloc_mlp(m, &m->db, Bp * WID)) || (rc = malloc_mlp(m, &m->g16, WID * KIN)) ||
      (rc = malloc_mlp(m, &m->loss, 1)))
    return fail(rc);
  for (int l = 0; l < 3; ++l)
    if ((rc = malloc_mlp(m, &m->W[l], WID * WID))) return fail(rc);
  for (int l = 0; l < 4; ++l)
    if ((rc = malloc_mlp(m, &m->A[l], Bp * WID)) || (rc = malloc_mlp(m, &m->Z[l], Bp * WID))) return fail(rc);
  cudaStream_t st = m->stream;
  if (cudaMemcpyAsync(m->p, params_host, sizeof(float) * P, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(m->norm, norm_host, sizeof(float) * (2 * NIN + 2), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(m->m, 0, sizeof(float) * P, st) != cudaSuccess ||
      cudaMemsetAsync(m->v, 0, sizeof(float) * P, st) != cudaSuccess) {
    set_error("MLP upload failed");
    return fail(KFBI_ERR_CUDA);
  }
  if ((rc = mlp_refresh(m))) return fail(rc);
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    set_error("MLP setup failed");
    return fail(KFBI_ERR_CUDA);
  }
  *out = m;
  return KFBI_OK;
}

void kfbi_mlp_destroy(kfbi_mlp* m) {
  if (!m) return;
  cudaStreamSynchronize(m->stream);
  for (void* p : m->allocs) cudaFree(p);
  delete m;
}

int kfbi_mlp_num_params(void) { return (int)Offsets().total; }

int kfbi_mlp_get(kfbi_mlp* m, float* params_host) {
  if (!m || !params_host) {
    set_error("null argument");
    return KFBI_ERR_ARG;
  }
  KFBI_CUDA(cudaMemcpyAsync(params_host, m->p, sizeof(float) * m->off.total, cudaMemcpyDeviceToHost, m->stream));
  KFBI_CUDA(cudaStreamSynchronize(m->stream));
  return KFBI_OK;
}

int kfbi_mlp_forward(kfbi_mlp* m, const float* F_dev, int B, float* o_dev) {
  if (!m || !F_dev || !o_dev) {
    set_error("null argument");
    return KFBI_ERR_ARG;
  }
  int Bp, rc;
  if ((rc = mlp_prepare_raw(m, F_dev, B, &Bp))) return rc;
  if ((rc = mlp_infer_rows(m, Bp))) return rc;
  KFBI_CUDA(cudaMemcpyAsync(o_dev, m->o, sizeof(float) * B, cudaMemcpyDeviceToDevice, m->stream));
  return KFBI_OK;
}

int kfbi_mlp_grad(kfbi_mlp* m, const float* F_dev, const float* t_dev, int B, float* loss_host, float* grad_host) {
  if (!m || !F_dev || !t_dev) {
    set_error("null argument");
    return KFBI_ERR_ARG;
  }
  int Bp, rc;
  if ((rc = mlp_prepare_raw(m, F_dev, B, &Bp))) return rc;
  if ((rc = mlp_forward_rows(m, Bp))) return rc;
  if ((rc = mlp_backward(m, t_dev, B, Bp))) return rc;
  float l = 0.0f;
  KFBI_CUDA(cudaMemcpyAsync(&l, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
  if (grad_host)
    KFBI_CUDA(cudaMemcpyAsync(grad_host, m->g, sizeof(float) * m->off.total, cudaMemcpyDeviceToHost, m->stream));
  KFBI_CUDA(cudaStreamSynchronize(m->stream));
  if (loss_host) *loss_host = 0.5f * l / (float)B;
  return KFBI_OK;
}

int kfbi_mlp_layers(kfbi_mlp* m, const float* F_dev, const float* T_dev, int B, float* z_dev, float* o_dev,
                    float* d_dev, float* d4_dev) {
  if (!m || !F_dev) {
    set_error("null argument");
    return KFBI_ERR_ARG;
  }
  int Bp, rc;
  if ((rc = mlp_prepare_raw(m, F_dev, B, &Bp))) return rc;
  if ((rc = mlp_forward_rows(m, Bp))) return rc;
  cudaStream_t st = m->stream;
  if (z_dev)
    for (int l = 0; l < 4; ++l)
      KFBI_CUDA(cudaMemcpyAsync(z_dev + (size_t)l * B * WID, m->Z[l], sizeof(float) * B * WID,
                                cudaMemcpyDeviceToDevice, st));
  if (o_dev) KFBI_CUDA(cudaMemcpyAsync(o_dev, m->o, sizeof(float) * B, cudaMemcpyDeviceToDevice, st));
  if (T_dev) {
    m->dump_d = d_dev;
    m->dump_d4 = d4_dev;
    rc = mlp_backward(m, T_dev, B, Bp);
    m->dump_d = m->dump_d4 = nullptr;
    if (rc) return rc;
  }
  KFBI_CUDA(cudaStreamSynchronize(st));
  return KFBI_OK;
}

int kfbi_mlp_train_step(kfbi_mlp* m, const float* F_dev, const float* t_dev, int B, float lr, float* loss_host) {
  int rc = kfbi_mlp_grad(m, F_dev, t_dev, B, loss_host, nullptr);
  if (rc) return rc;
  ++m->step;
  const float c1 = 1.0f - powf(0.9f, (float)m->step), c2 = 1.0f - powf(0.999f, (float)m->step);
  k_adam<<<blocks(m->off.total, 256), 256, 0, m->stream>>>(m->p, m->g, m->m, m->v, (int)m->off.total, lr, c1, c2);
  KFBI_CHECK_LAUNCH();
  return mlp_refresh(m);
}

}  // extern "C"
