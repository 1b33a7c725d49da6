// Hot-path kernels other than the transforms:
//  - irregular-node correction (Section 5.3, Eq. correct) as a gather over
//    each irregular node's crossing arms of precomputed density rows;
//  - periodic-spline moments of the density (2-D boundary representation);
//  - interface limits dv^+/dn (Section 5.4) as a 6/10-point gather from the
//    padded solution grid plus the node's own jump row;
//  - Krylov vector kernels (dot products, updates, Givens rotations);
//  - FitzHugh-Nagumo forward/backward Euler half steps (Sections 3, 7);
//  - extracellular potential with zero mean over Omega.
#include <cuda_runtime.h>

#include "ffloat.cuh"
#include "internal.cuh"

namespace kfbi {
namespace {

constexpr int RED_BLOCKS = 152;  // one partial sum per SM for the dot products
// blocks of the Arnoldi kernels (one row per thread up to 155,648 rows); the
// partial-sum buffer holds ARN_BLOCKS x (MAX_RESTART + 2) values
constexpr int ARN_BLOCKS = KFBI_ARN_BLOCKS;

// corr_i = sum over the node's CSR row of w_k x[pid_k] (the row is its arms'
// crossing rows concatenated, built at setup: two dependent loads per entry)
__global__ void k_correction(Tables t, const double* __restrict__ x, double* __restrict__ corr,
                             const int* __restrict__ skip) {
  pdl_wait();
  pdl_launch_next();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.n_irr || (skip != nullptr && *skip)) return;
  const int k0 = t.cr_ptr[i], k1 = t.cr_ptr[i + 1];
  double acc = 0.0;
  for (int k = k0; k < k1; ++k) acc += t.cr_w[k] * x[t.cr_pid[k]];
  corr[i] = acc;
}

// x = [psi; m] with m_i = sum_j gcol[(i - j) mod M] psi_j
__global__ void k_spline(const double* __restrict__ gcol, const double* __restrict__ psi, double* __restrict__ x, int M) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  double acc = 0.0;
  for (int j = 0; j < M; ++j) {
    int k = i - j;
    if (k < 0) k += M;
    acc += gcol[k] * psi[j];
  }
  x[i] = psi[i];
  x[M + i] = acc;
}

// out_i = base_i + sgn * (sum_j wn_ij v(p_j) + sum_k dw_ik x[dpid_ik])
template <typename T>
__global__ void k_limit(Tables t, GridParams gr, const T* __restrict__ grid, const double* __restrict__ x,
                        const double* __restrict__ base, double sgn, double* __restrict__ out,
                        const int* __restrict__ skip) {
  pdl_wait();
  pdl_launch_next();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.M || (skip != nullptr && *skip)) return;
  const int d = gr.dim, P = work_n(gr);
  const int64_t sx = 1, sy = P, sz = (int64_t)P * P;
  const int64_t c = t.n_base[i];
  const int s0 = t.n_sign[(size_t)i * d], s1 = t.n_sign[(size_t)i * d + 1];
  const double* wn = t.n_wn + (size_t)i * t.P;
  double acc = wn[0] * (double)grid[c] + wn[1] * (double)grid[c - sx] + wn[2] * (double)grid[c + sx] +
               wn[3] * (double)grid[c - sy] + wn[4] * (double)grid[c + sy];
  if (d == 2) {
    acc += wn[5] * (double)grid[c + s0 * sx + s1 * sy];
  } else {
    const int s2 = t.n_sign[(size_t)i * d + 2];
    acc += wn[5] * (double)grid[c - sz] + wn[6] * (double)grid[c + sz];
    acc += wn[7] * (double)grid[c + s0 * sx + s1 * sy];
    acc += wn[8] * (double)grid[c + s0 * sx + s2 * sz];
    acc += wn[9] * (double)grid[c + s1 * sy + s2 * sz];
  }
  if (x != nullptr) {
    const size_t o = (size_t)i * (PATCH_MAX + 1);
    const int K = t.n_dcnt[i];
    for (int k = 0; k < K; ++k) acc += t.n_dw[o + k] * x[t.n_dpid[o + k]];
  }
  out[i] = (base != nullptr ? base[i] : 0.0) + sgn * acc;
}

// same limit from a field-layout grid
__global__ void k_limit_user(Tables t, GridParams gr, const double* __restrict__ u, const double* __restrict__ x,
                             const double* __restrict__ base, double sgn, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.M) return;
  const int d = gr.dim, n1 = field_n(gr), k0 = field_first(gr);
  const int* c = t.n_center + (size_t)i * d;
  const int8_t* sg = t.n_sign + (size_t)i * d;
  const double* wn = t.n_wn + (size_t)i * t.P;
  const int cx = c[0], cy = c[1], cz = d == 3 ? c[2] : 1;
  auto at = [&](int dx, int dy, int dz) -> double {
    const int64_t f = (int64_t)(cx + dx - k0) + (int64_t)(cy + dy - k0) * n1 +
                      (d == 3 ? (int64_t)(cz + dz - k0) * n1 * n1 : 0);
    return u[f];
  };
  double acc = wn[0] * at(0, 0, 0) + wn[1] * at(-1, 0, 0) + wn[2] * at(1, 0, 0) + wn[3] * at(0, -1, 0) +
               wn[4] * at(0, 1, 0);
  if (d == 2) {
    acc += wn[5] * at(sg[0], sg[1], 0);
  } else {
    acc += wn[5] * at(0, 0, -1) + wn[6] * at(0, 0, 1);
    acc += wn[7] * at(sg[0], sg[1], 0) + wn[8] * at(sg[0], 0, sg[2]) + wn[9] * at(0, sg[1], sg[2]);
  }
  if (x != nullptr) {
    const size_t o = (size_t)i * (PATCH_MAX + 1);
    const int K = t.n_dcnt[i];
    for (int k = 0; k < K; ++k) acc += t.n_dw[o + k] * x[t.n_dpid[o + k]];
  }
  out[i] = (base != nullptr ? base[i] : 0.0) + sgn * acc;
}

// res = alpha*src - (L_h u) on the user layout, L_h the 5/7-point operator
// with zero Dirichlet data (float64 residual of the refined box solve)
// r = alpha*src - L_h u on the user layout; one block row per (y, z) grid line
// so no index needs a 64-bit division.
__global__ void k_residual(GridParams gr, const double* __restrict__ src, double alpha, const double* __restrict__ u,
                           double lambda, double* __restrict__ res) {
  const int n1 = gr.N - 1;
  const double ih2 = 1.0 / (gr.h * gr.h);
  const double diag = -2.0 * gr.dim * ih2 - lambda;
  const int y = blockIdx.x, z = blockIdx.y;
  const int64_t s = (int64_t)n1 * n1;
  const int64_t base = (int64_t)z * s + (int64_t)y * n1;
  for (int x = threadIdx.x; x < n1; x += blockDim.x) {
    const int64_t f = base + x;
    const double uc = u[f];
    double nb = (x > 0 ? u[f - 1] : 0.0) + (x < n1 - 1 ? u[f + 1] : 0.0);
    nb += (y > 0 ? u[f - n1] : 0.0) + (y < n1 - 1 ? u[f + n1] : 0.0);
    if (gr.dim == 3) nb += (z > 0 ? u[f - s] : 0.0) + (z < n1 - 1 ? u[f + s] : 0.0);
    const double Lu = nb * ih2 + diag * uc;
    res[f] = (src != nullptr ? alpha * src[f] : 0.0) - Lu;
  }
}

// error-free transformations: Knuth's TwoSum (s + e = a + b exactly) and the
// product error by a fused multiply-add (p + e = a b exactly)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = a * b;
  e = fmaf(a, b, -p);
}

// a float64 source value as a float pair, split on its bits (a float64
// conversion costs as much as a float64 add here); sources beyond the float
// range or not finite become infinities or NaN
__device__ __forceinline__ void src_pair(double sv, float& sh, float& sl) {
  ffl::ff p;
  if (ffl::split(sv, p)) {
    sh = p.h;
    sl = p.l;
  } else {
    sh = ffl::narrow(sv);
    sl = 0.0f;
  }
}

// r = -L_h u for u given exactly by the padded float32 grid of a float32
// solve (index 0 of each axis holds the zero boundary value), in float-float
// arithmetic: the float64 pipe is 1/64 of the float32 rate here, and the
// 6-point sum of float32 values, ih2 and the diagonal kept as float pairs
// give L_h u to about 1e-14 of its terms, ample for a refinement residual
// that is 1e-7 of them.  One block row per (y, z) line.
__global__ void k_residual_ff(GridParams gr, const float* __restrict__ u32, float ih2_hi, float ih2_lo, float dg_hi,
                              float dg_lo, const double* __restrict__ src, float al_hi, float al_lo,
                              float* __restrict__ res) {
  const int N = gr.N, n1 = N - 1;
  const int y = blockIdx.x, z = blockIdx.y;
  const size_t NN = (size_t)N * N;
  const size_t pbase = gr.dim == 3 ? (size_t)(z + 1) * NN + (size_t)(y + 1) * N : (size_t)(y + 1) * N;
  const size_t ubase = gr.dim == 3 ? ((size_t)z * n1 + y) * n1 : (size_t)y * n1;
  for (int x = threadIdx.x; x < n1; x += blockDim.x) {
    const size_t p = pbase + x + 1;
    const float uc = u32[p];
    float s = u32[p - 1], e = 0.0f, t;
    two_sum(s, x < n1 - 1 ? u32[p + 1] : 0.0f, s, t);
    e += t;
    two_sum(s, u32[p - N], s, t);
    e += t;
    two_sum(s, y < n1 - 1 ? u32[p + N] : 0.0f, s, t);
    e += t;
    if (gr.dim == 3) {
      two_sum(s, u32[p - NN], s, t);
      e += t;
      two_sum(s, z < n1 - 1 ? u32[p + NN] : 0.0f, s, t);
      e += t;
    }
    float p1, e1, p2, e2, hsum, e3;
    two_prod(ih2_hi, s, p1, e1);
    e1 += ih2_hi * e + ih2_lo * s;
    two_prod(dg_hi, uc, p2, e2);
    e2 += dg_lo * uc;
    two_sum(p1, p2, hsum, e3);
    float lo = e1 + e2 + e3;
    if (src != nullptr) {
      // + alpha * src, src split into a float pair on its bits
      const double sv = src[ubase + x];
      float sh, sl;
      src_pair(sv, sh, sl);
      float q, eq, h2, e4;
      two_prod(al_hi, sh, q, eq);
      eq += al_hi * sl + al_lo * sh;
      two_sum(q, -hsum, h2, e4);
      res[ubase + x] = h2 + (e4 + eq - lo);
    } else {
      res[ubase + x] = -(hsum + lo);
    }
  }
}

// at the irregular nodes, where the correction makes r a small difference of
// large terms: r = corr - L_h u in float64, from the float64 copy of u, or
// (u == nullptr) from the padded float grid u32 that holds u exactly
__global__ void k_residual_irr(GridParams gr, Tables t, const double* __restrict__ corr, const double* __restrict__ u,
                               double lambda, const double* __restrict__ src, double alpha, float* __restrict__ res,
                               const float* __restrict__ u32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.n_irr) return;
  const int N = gr.N, n1 = N - 1;
  const double ih2 = 1.0 / (gr.h * gr.h);
  const double diag = -2.0 * gr.dim * ih2 - lambda;
  const int64_t f = t.irr[i];
  const int64_t s = (int64_t)n1 * n1;
  const int x = (int)(f % n1), y = (int)((f / n1) % n1), z = gr.dim == 3 ? (int)(f / s) : 0;
  double uc, nb;
  if (u != nullptr) {
    uc = u[f];
    nb = (x > 0 ? u[f - 1] : 0.0) + (x < n1 - 1 ? u[f + 1] : 0.0);
    nb += (y > 0 ? u[f - n1] : 0.0) + (y < n1 - 1 ? u[f + n1] : 0.0);
    if (gr.dim == 3) nb += (z > 0 ? u[f - s] : 0.0) + (z < n1 - 1 ? u[f + s] : 0.0);
  } else {
    // padded index of (x, y, z): index 0 of each axis is the zero boundary
    const size_t NN = (size_t)N * N;
    const size_t p = gr.dim == 3 ? ((size_t)(z + 1) * N + (y + 1)) * N + (x + 1) : (size_t)(y + 1) * N + (x + 1);
    uc = ffl::widen(u32[p]);
    nb = ffl::widen(u32[p - 1]) + (x < n1 - 1 ? ffl::widen(u32[p + 1]) : 0.0);
    nb += ffl::widen(u32[p - N]) + (y < n1 - 1 ? ffl::widen(u32[p + N]) : 0.0);
    if (gr.dim == 3) nb += ffl::widen(u32[p - NN]) + (z < n1 - 1 ? ffl::widen(u32[p + NN]) : 0.0);
  }
  const double a = src != nullptr ? alpha * src[f] : 0.0;
  res[f] = (float)(a + corr[i] - (nb * ih2 + diag * uc));
}

// the float-float residual on the Neumann box's field layout: u32 is the
// float32 work grid itself (all (N+1)^d nodes), a neighbour beyond the box
// its mirror image
__global__ void k_residual_ff_neumann(GridParams gr, const float* __restrict__ u32, float ih2_hi, float ih2_lo,
                                      float dg_hi, float dg_lo, const double* __restrict__ src, float al_hi,
                                      float al_lo, float* __restrict__ res) {
  const int P = gr.N + 1;
  const int y = blockIdx.x, z = blockIdx.y;
  const int64_t PP = (int64_t)P * P;
  const int64_t base = (int64_t)z * PP + (int64_t)y * P;
  const int64_t ym = y > 0 ? -P : P, yp = y < P - 1 ? P : -P;
  const int64_t zm = z > 0 ? -PP : PP, zp = z < P - 1 ? PP : -PP;
  for (int x = threadIdx.x; x < P; x += blockDim.x) {
    const int64_t f = base + x;
    const float uc = u32[f];
    float sm = u32[f + (x > 0 ? -1 : 1)], e = 0.0f, t;
    two_sum(sm, u32[f + (x < P - 1 ? 1 : -1)], sm, t);
    e += t;
    two_sum(sm, u32[f + ym], sm, t);
    e += t;
    two_sum(sm, u32[f + yp], sm, t);
    e += t;
    if (gr.dim == 3) {
      two_sum(sm, u32[f + zm], sm, t);
      e += t;
      two_sum(sm, u32[f + zp], sm, t);
      e += t;
    }
    float p1, e1, p2, e2, hsum, e3;
    two_prod(ih2_hi, sm, p1, e1);
    e1 += ih2_hi * e + ih2_lo * sm;
    two_prod(dg_hi, uc, p2, e2);
    e2 += dg_lo * uc;
    two_sum(p1, p2, hsum, e3);
    const float lo = e1 + e2 + e3;
    if (src != nullptr) {
      const double sv = src[f];
      float sh, sl;
      src_pair(sv, sh, sl);
      float q, eq, h2, e4;
      two_prod(al_hi, sh, q, eq);
      eq += al_hi * sl + al_lo * sh;
      two_sum(q, -hsum, h2, e4);
      res[f] = h2 + (e4 + eq - lo);
    } else {
      res[f] = -(hsum + lo);
    }
  }
}

// the irregular nodes of the Neumann box in float64 (interior nodes: no
// mirrored neighbour)
__global__ void k_residual_irr_neumann(GridParams gr, Tables t, const double* __restrict__ corr,
                                       const double* __restrict__ u, double lambda, const double* __restrict__ src,
                                       double alpha, float* __restrict__ res) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.n_irr) return;
  const int P = gr.N + 1;
  const double ih2 = 1.0 / (gr.h * gr.h);
  const double diag = -2.0 * gr.dim * ih2 - lambda;
  const int64_t f = t.irr_user[i];
  const int64_t PP = (int64_t)P * P;
  double nb = u[f - 1] + u[f + 1] + u[f - P] + u[f + P];
  if (gr.dim == 3) nb += u[f - PP] + u[f + PP];
  const double a = src != nullptr ? alpha * src[f] : 0.0;
  res[f] = (float)(a + corr[i] - (nb * ih2 + diag * u[f]));
}

__global__ void k_scatter_add(Tables t, const double* __restrict__ corr, double* __restrict__ g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < t.n_irr) g[t.irr_user[i]] += corr[i];
}

// r = alpha*src - L_h u on the Neumann box's field layout (all (N+1)^d
// nodes; a neighbour beyond the box is the mirror image across it)
__global__ void k_residual_neumann(GridParams gr, const double* __restrict__ src, double alpha,
                                   const double* __restrict__ u, double lambda, double* __restrict__ res) {
  const int P = gr.N + 1;
  const double ih2 = 1.0 / (gr.h * gr.h);
  const double diag = -2.0 * gr.dim * ih2 - lambda;
  const int y = blockIdx.x, z = blockIdx.y;
  const int64_t s = (int64_t)P * P;
  const int64_t base = (int64_t)z * s + (int64_t)y * P;
  const int64_t ym = y > 0 ? -P : P, yp = y < P - 1 ? P : -P;
  const int64_t zm = z > 0 ? -s : s, zp = z < P - 1 ? s : -s;
  for (int x = threadIdx.x; x < P; x += blockDim.x) {
    const int64_t f = base + x;
    const double uc = u[f];
    double nb = u[f + (x > 0 ? -1 : 1)] + u[f + (x < P - 1 ? 1 : -1)];
    nb += u[f + ym] + u[f + yp];
    if (gr.dim == 3) nb += u[f + zm] + u[f + zp];
    const double Lu = nb * ih2 + diag * uc;
    res[f] = (src != nullptr ? alpha * src[f] : 0.0) - Lu;
  }
}

__global__ void k_add_scalar(double* __restrict__ out, const double* __restrict__ slot, double c, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += c * slot[0];
}

__global__ void k_stim_source(const double* __restrict__ V, double lambda, const double* __restrict__ I, double c,
                              double* __restrict__ f, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    f[i] = (V != nullptr ? -lambda * V[i] : 0.0) + c * I[i];
}

__global__ void k_phi_e(const double* __restrict__ V, const double* __restrict__ S, double si, double se,
                        double* __restrict__ ue, int64_t n) {
  const double inv = 1.0 / (si + se);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    ue[i] = (S[i] - si * V[i]) * inv;
}

__global__ void k_sub_mean(double* __restrict__ ue, const double* __restrict__ sum, double inv_count, int64_t n) {
  const double mean = sum[0] * inv_count;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    ue[i] -= mean;
}

__global__ void k_lincomb(double* __restrict__ y, double a, const double* __restrict__ x, double b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

__global__ void k_scatter(Tables t, const double* __restrict__ corr, double* __restrict__ g, int64_t total) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < total; f += (int64_t)gridDim.x * blockDim.x)
    g[f] = 0.0;
}
__global__ void k_scatter2(Tables t, const double* __restrict__ corr, double* __restrict__ g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < t.n_irr) g[t.irr_user[i]] = corr[i];
}

__global__ void k_pad_to_user(GridParams gr, const double* __restrict__ p, double* __restrict__ u, int64_t total) {
  const int N = gr.N, n1 = N - 1;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < total; f += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(f % n1) + 1, y = (int)((f / n1) % n1) + 1;
    const int z = gr.dim == 3 ? (int)(f / ((int64_t)n1 * n1)) + 1 : 0;
    u[f] = p[((int64_t)z * N + y) * N + x];
  }
}

// ---------------------------------------------------------------- Krylov
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// partial[k][b] = sum over block b's slice of V_k . w
__global__ void k_dots_partial(const double* __restrict__ V, int ld, const double* __restrict__ w, int n,
                               double* __restrict__ partial) {
  const int k = blockIdx.y;
  const double* v = V + (size_t)k * ld;
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) acc += v[i] * w[i];
  __shared__ double ws[32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
    s = warp_sum(s);
    if (threadIdx.x == 0) partial[(size_t)k * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void k_dots_final(const double* __restrict__ partial, int nb, int nvec, double* __restrict__ out) {
  const int k = blockIdx.x;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += partial[(size_t)k * nb + b];
  __shared__ double ws[32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
    s = warp_sum(s);
    if (threadIdx.x == 0) out[k] = s;
  }
}

// w += sign * sum_k coef[k] V_k
__global__ void k_update(double* __restrict__ w, const double* __restrict__ V, int nvec, int ld,
                         const double* __restrict__ coef, double sign, int n) {
  __shared__ double cs[MAX_RESTART + 2];
  for (int k = threadIdx.x; k < nvec; k += blockDim.x) cs[k] = coef[k];
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int k = 0; k < nvec; ++k) acc += cs[k] * V[(size_t)k * ld + i];
    w[i] += sign * acc;
  }
}

__global__ void k_axpby(double* __restrict__ y, double a, const double* __restrict__ x, double b, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = a * x[i] + b * y[i];
}

__global__ void k_scale_norm(double* __restrict__ v, const double* __restrict__ w, const double* __restrict__ nrm2, int n,
                             const int* __restrict__ skip) {
  pdl_wait();
  pdl_launch_next();
  if (skip != nullptr && *skip) return;
  const double s = sqrt(nrm2[0]);
  const double inv = s > 0.0 ? 1.0 / s : 0.0;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = w[i] * inv;
}

// small-vector layout (doubles): H column-major [(m+1) x m] at 0, cs at HS,
// sn at HS+m, g at HS+2m, hcol at HS+3m+1, nrm2 at HS+4m+2, result at HS+4m+3
struct SmallLayout {
  int m;
  __host__ __device__ int H() const { return 0; }
  __host__ __device__ int cs() const { return (m + 1) * m; }
  __host__ __device__ int sn() const { return cs() + m; }
  __host__ __device__ int g() const { return sn() + m; }
  __host__ __device__ int hcol() const { return g() + m + 1; }
  __host__ __device__ int nrm2() const { return hcol() + m + 2; }
  __host__ __device__ int res() const { return nrm2() + 2; }
  __host__ __device__ int y() const { return res() + 2; }
  __host__ __device__ int total() const { return y() + m + 2; }
};

// column j of H from hcol and sqrt(nrm2); apply rotations; new rotation; |g_{j+1}|
__device__ void givens_column(double* s, int m, int j) {
  SmallLayout L{m};
  double* H = s + L.H();
  double* cs = s + L.cs();
  double* sn = s + L.sn();
  double* g = s + L.g();
  const double* hc = s + L.hcol();
  double col[MAX_RESTART + 2];
  for (int i = 0; i <= j; ++i) col[i] = hc[i];
  col[j + 1] = sqrt(s[L.nrm2()]);
  for (int i = 0; i < j; ++i) {
    const double t = cs[i] * col[i] + sn[i] * col[i + 1];
    col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
    col[i] = t;
  }
  const double den = hypot(col[j], col[j + 1]);
  cs[j] = col[j] / den;
  sn[j] = col[j + 1] / den;
  col[j] = den;
  col[j + 1] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  for (int i = 0; i <= j + 1; ++i) H[(size_t)j * (m + 1) + i] = col[i];
  s[L.res()] = fabs(g[j + 1]);
}

__global__ void k_givens(double* s, int m, int j) { givens_column(s, m, j); }

// ---------------------------------------------- fused Arnoldi step (CGS2)
// One Krylov step after w = A v_j takes four launches: h = V^T w; w -= V h
// with y = V^T w; w -= V y with ||w||^2, H(:, j) = h + y and the Givens
// update; v_{j+1} = w / ||w||.  Each thread owns a grid-stride set of rows;
// the last block to finish (a ticket counter, reset by that block) reduces
// the per-block partial sums in a fixed order, so results do not depend on
// block scheduling.  skip (optional): a device flag; when set, the kernel
// does nothing (an iteration enqueued ahead of the convergence test).

// true in every thread of the block that finishes last
__device__ __forceinline__ bool arn_last_block(unsigned* counter) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  return last;
}

// out[k] = sum_b partial[k][b] for k < nv, one warp per k; each lane keeps
// four independent L2 loads in flight (the partials were written by other
// blocks just before, so every load is a round trip to L2), in a fixed order
__device__ __forceinline__ void arn_reduce(const double* partial, int nb, int nv, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = warp; k < nv; k += nw) {
    const double* pk = partial + (size_t)k * nb;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int b = lane;
    for (; b + 96 < nb; b += 128) {
      const double x0 = __ldcg(&pk[b]), x1 = __ldcg(&pk[b + 32]), x2 = __ldcg(&pk[b + 64]), x3 = __ldcg(&pk[b + 96]);
      a0 += x0;
      a1 += x1;
      a2 += x2;
      a3 += x3;
    }
    for (; b < nb; b += 32) a0 += __ldcg(&pk[b]);
    double acc = (a0 + a1) + (a2 + a3);
    acc = warp_sum(acc);
    if (lane == 0) out[k] = acc;
  }
}

constexpr int ARN_CH = 8;  // basis vectors per register chunk

// Sums of eight per-lane values over the warp with nine float64 additions
// per lane instead of forty (float64 issue is scarce on this part): each
// halving step keeps half of the values and adds the partner lane's copy of
// them, so that after offsets 16, 8 and 4 lane l holds vector (l >> 2) & 7
// summed over the lanes that differ in bits 2-4; offsets 2 and 1 finish the
// sum.  The lanes with (l & 3) == 0 return the totals.
__device__ __forceinline__ double warp_sum8(double (&v)[ARN_CH]) {
  const int lane = threadIdx.x & 31;
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const double send = b4 ? v[i] : v[i + 4], keep = b4 ? v[i + 4] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const double send = b3 ? v[i] : v[i + 2], keep = b3 ? v[i + 2] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  {
    const double send = b2 ? v[0] : v[1], keep = b2 ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  double t = v[0];
  t += __shfl_xor_sync(0xffffffffu, t, 2);
  t += __shfl_xor_sync(0xffffffffu, t, 1);
  return t;
}

// w_i -= sum_{k < nv} cs[k] V_k[i] over a grid-stride set of rows; each
// chunk's loads are independent, so a thread has ARN_CH of them in flight
__device__ __forceinline__ void arn_update(double* __restrict__ w, const double* __restrict__ V, int ld, int n, int nv,
                                           const double* cs, double* sq) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int k0 = 0; k0 < nv; k0 += ARN_CH) {
      double x[ARN_CH];
#pragma unroll
      for (int u = 0; u < ARN_CH; ++u) x[u] = k0 + u < nv ? V[(size_t)(k0 + u) * ld + i] : 0.0;
#pragma unroll
      for (int u = 0; u < ARN_CH; ++u)
        if (k0 + u < nv) acc += cs[k0 + u] * x[u];
    }
    const double wi = w[i] - acc;
    w[i] = wi;
    if (sq != nullptr) *sq += wi * wi;
  }
}

// [UPDATE: w -= sum_k coef[k] V_k;]  out[k] = V_k . w  (k < nv)
template <bool UPDATE>
__global__ void __launch_bounds__(256) k_arn_gs(double* __restrict__ w, const double* __restrict__ V, int ld, int n,
                                                int nv, const double* __restrict__ coef, double* __restrict__ partial,
                                                unsigned* __restrict__ counter, double* __restrict__ out,
                                                const int* __restrict__ skip) {
  pdl_wait();
  pdl_launch_next();
  if (skip != nullptr && *skip) return;
  __shared__ double cs[MAX_RESTART + 2];
  __shared__ double red[8][MAX_RESTART + 2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (UPDATE) {
    for (int k = threadIdx.x; k < nv; k += blockDim.x) cs[k] = coef[k];
    __syncthreads();
    arn_update(w, V, ld, n, nv, cs, nullptr);
  }
  // each thread reads back only the rows it updated itself
  for (int k0 = 0; k0 < nv; k0 += ARN_CH) {
    double d[ARN_CH];
#pragma unroll
    for (int u = 0; u < ARN_CH; ++u) d[u] = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      const double wi = w[i];
#pragma unroll
      for (int u = 0; u < ARN_CH; ++u)
        if (k0 + u < nv) d[u] += V[(size_t)(k0 + u) * ld + i] * wi;
    }
    const double t = warp_sum8(d);
    const int u = lane >> 2;
    if ((lane & 3) == 0 && k0 + u < nv) red[warp][k0 + u] = t;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nv; k += blockDim.x) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q][k];
    partial[(size_t)k * gridDim.x + blockIdx.x] = t;
  }
  if (!arn_last_block(counter)) return;
  arn_reduce(partial, gridDim.x, nv, out);
  if (threadIdx.x == 0) *counter = 0u;
}

// w -= sum_k y[k] V_k; ||w||^2; hcol += y; Givens update of column j; the
// residual estimate |g_{j+1}| and the stop flag (estimate / gnorm <= tol, or
// not finite: the host's test, in the same float64 operations)
__global__ void __launch_bounds__(256) k_arn_close(double* __restrict__ w, const double* __restrict__ V, int ld, int n,
                                                   int nv, double* __restrict__ s, int m, int j,
                                                   double* __restrict__ partial, unsigned* __restrict__ counter,
                                                   double gnorm, double tol, int* stop, const int* skip) {
  pdl_wait();
  pdl_launch_next();
  if (skip != nullptr && *skip) return;
  SmallLayout L{m};
  __shared__ double cs[MAX_RESTART + 2];
  __shared__ double ws[32];
  for (int k = threadIdx.x; k < nv; k += blockDim.x) cs[k] = s[L.y() + k];
  __syncthreads();
  double sq = 0.0;
  arn_update(w, V, ld, n, nv, cs, &sq);
  sq = warp_sum(sq);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
  }
  if (!arn_last_block(counter)) return;
  if (threadIdx.x < 32) arn_reduce(partial, gridDim.x, 1, s + L.nrm2());
  for (int k = threadIdx.x; k < nv; k += blockDim.x) s[L.hcol() + k] += cs[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    givens_column(s, m, j);
    const double rel = s[L.res()] / gnorm;
    const int done = !(rel > tol) || !isfinite(rel);
    s[L.res() + 1] = done ? 1.0 : 0.0;
    *stop = done;
    *counter = 0u;
  }
}

// Normal equations of the density-history projection in one launch:
// G[u][v] = h_u . h_v (u, v < K), b[u] = h_u . g, gg = g . g, with h_u the
// rows of H (leading dimension ld).  Per-thread sums over a grid-stride set
// of rows, warp and block reductions, and the last block's fixed-order sum
// of the per-block partials.
template <int K>
__global__ void __launch_bounds__(256) k_gram(const double* __restrict__ H, int ld, const double* __restrict__ g, int n,
                                              double* __restrict__ partial, unsigned* __restrict__ counter,
                                              double* __restrict__ G, double* __restrict__ b, double* __restrict__ gg) {
  constexpr int NP = K * (K + 1) / 2 + K + 1;
  double acc[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) acc[p] = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double x[K + 1];
#pragma unroll
    for (int u = 0; u < K; ++u) x[u] = H[(size_t)u * ld + i];
    x[K] = g[i];
    int p = 0;
#pragma unroll
    for (int u = 0; u < K; ++u)
#pragma unroll
      for (int v = u; v <= K; ++v) acc[p++] += x[u] * x[v];
    acc[p] += x[K] * x[K];
  }
  __shared__ double red[8][NP];
  __shared__ double fin[NP];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const double t = warp_sum(acc[p]);
    if (lane == 0) red[warp][p] = t;
  }
  __syncthreads();
  for (int p = threadIdx.x; p < NP; p += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][p];
    partial[(size_t)p * gridDim.x + blockIdx.x] = t;
  }
  if (!arn_last_block(counter)) return;
  arn_reduce(partial, gridDim.x, NP, fin);
  __syncthreads();
  if (threadIdx.x == 0) {
    int p = 0;
    for (int u = 0; u < K; ++u) {
      for (int v = u; v < K; ++v) {
        G[u * K + v] = fin[p];
        G[v * K + u] = fin[p];
        ++p;
      }
      b[u] = fin[p++];
    }
    *gg = fin[p];
    *counter = 0u;
  }
}

// y = R^{-1} g for the leading k x k block
__global__ void k_backsolve(double* s, int m, int k) {
  SmallLayout L{m};
  const double* H = s + L.H();
  const double* g = s + L.g();
  double* y = s + L.y();
  for (int i = k - 1; i >= 0; --i) {
    double a = g[i];
    for (int c = i + 1; c < k; ++c) a -= H[(size_t)c * (m + 1) + i] * y[c];
    y[i] = a / H[(size_t)i * (m + 1) + i];
  }
}

__global__ void k_init_arnoldi(double* s, int m) {
  SmallLayout L{m};
  const int i = threadIdx.x;
  if (i <= m) s[L.g() + i] = i == 0 ? sqrt(s[L.nrm2()]) : 0.0;
}

__global__ void k_add_small(double* s, int m, int n) {
  // hcol += second-pass coefficients stored right after it (CGS2)
  SmallLayout L{m};
  const int i = threadIdx.x;
  if (i < n) s[L.hcol() + i] += s[L.y() + i];
}

// ------------------------------------------------------------- reaction
// FP64 work is scarce on this part (2 FMA per SM per clock): the pointwise
// kernels keep float64 for what must be float64, write the cubic of the
// ionic current in Horner form with the constants folded (one fused
// multiply-add per power), and take branch decisions on integer bits.
//
// Forward-Euler half step: with a = k H / Cm,
//   V1 = V + a (V (V - theta)(1 - V) - q)
//      = ((-a V + a (1 + theta)) V - a theta) V + (V - a q),
//   q1 = (1 - k zeta) q + k alpha V.
__global__ void k_react_fe(kfbi_fhn p, double k, double* __restrict__ V, double* __restrict__ w, int64_t n) {
  const double a = k * p.H / p.Cm, ka = k * p.alpha, kz1 = 1.0 - k * p.zeta;
  const double p1 = a * (1.0 + p.theta), p0 = -a * p.theta;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = V[i], q = w[i];
    const double t = fma(fma(-a, v, p1), v, p0);
    V[i] = fma(t, v, fma(-a, q, v));
    w[i] = fma(ka, v, kz1 * q);
  }
}

// |x| < bound (bound > 0) on the bits: no float64 instruction; false for NaN
__device__ __forceinline__ bool abs_below(double x, double bound) {
  return (__double_as_longlong(x) & 0x7fffffffffffffffLL) < __double_as_longlong(bound);
}

// Backward-Euler half step: w is eliminated (w1 = (w0 + k alpha v) / (1 + k
// zeta)) and Newton solves the cubic in v,
//   F(v) = v - v0 - c (v (v - theta)(1 - v) - w1(v))
//        = ((c v - c (1 + theta)) v + (1 + c theta + c k alpha / den)) v + (c w0 / den - v0),
// c = k H / Cm, den = 1 + k zeta.  Float32 Newton steps first bring v to
// float32 resolution (error e0 <~ 1e-7 |v|); one more step then uses the
// residual F(v_f) evaluated in float-float arithmetic (v0 and w0 split into
// float pairs on their bits, about 48 significant bits, F to ~1e-14 of the
// sum S of its terms' sizes) with the float32 derivative (a quasi-Newton
// step: error <~ 1e-7 e0 + C e0^2 + 1e-14 S / |F'|), and w1 is formed as a
// float pair too.  The state meets float64 arithmetic in three additions only
// (v1 = v_f - dv as the sum of three exactly widened floats, w1 from its
// pair).  Converged: the float32 phase converged, the float-float step dv is
// below 1e-5 and small enough that the step's second-order error |F'' / 2F'|
// dv^2 stays below 1e-13, and S < 8 |F'| (away from a fold of the cubic,
// where the pairs' error and the float32 derivative's, divided by F', grow);
// otherwise plain float64 Newton steps continue from v_f until a step is
// below 1e-10 (also for inputs outside the pairs' range or not finite).
struct BeConsts {
  double c, e2, e1, cid, kid, inv_den;  // float64 fallback
  float cf, rf, thf, kaf, idf, th1;     // float32 Newton
  float c3f, e2f, e1f;                  // |c|, |e2|, |e1|: sizes of the residual's terms
  float e2x2;                           // 2 e2 (second derivative 6 c v + 2 e2)
  ffl::ff cP, e2P, e1P, cidP, kaP, idP; // float-float residual and w1
  // the next step's forward-Euler half step (see k_react_fe), when fused
  double fa, fp1, fp0, fka, fkz1;
};

struct VW {
  double v, w;
};

// float64 Newton steps from v (from v0 when start_f32 is false) for the
// nodes the float-pair step does not take, v0 = 2 (a + b) - c with MID, else
// c: kept out of line so that none of its float64 work is hoisted into the
// common path
template <bool MID>
__device__ __noinline__ VW be_newton64(const BeConsts& K, double a, double b, double c, double q0, bool start_f32,
                                       double v, int* err) {
  const double v0 = MID ? 2.0 * (a + b) - c : c;
  if (!start_f32) v = v0;
  const double a0 = fma(K.cid, q0, -v0);
  bool ok = false;
  for (int it = 0; it < 50; ++it) {
    const double F = fma(fma(fma(K.c, v, K.e2), v, K.e1), v, a0);
    const double dF = fma(fma(3.0 * K.c, v, 2.0 * K.e2), v, K.e1);
    const double dv = F / dF;
    v -= dv;
    if (abs_below(dv, 1e-10)) {
      ok = true;
      break;
    }
  }
  if (!ok) atomicOr(err, DEVERR_NEWTON);
  return VW{v, fma(K.kid, v, q0 * K.inv_den)};
}

// MID: v0 is the implicit-midpoint assembly 2 (v_V + v_B) - V of the
// float32 forms, formed here on float pairs from the three float64 fields
// (the midpoint value itself is never stored; it enters only this step).
// FE: the forward-Euler half step that opens the next Strang step follows in
// the same pass (the same float64 operations as k_react_fe), so that V and w
// cross memory once for both half steps and the forward step's float64 work
// overlaps the backward step's float32 work.
template <bool MID, bool FE>
__global__ void k_react_be(BeConsts K, double* __restrict__ V, double* __restrict__ w, const double* __restrict__ vV,
                           const double* __restrict__ vB, int64_t n, int* err) {
  using namespace ffl;
  // the next node's inputs are loaded before the current node is computed
  // (the Newton work between a node's loads and its stores is long)
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double nV = 0.0, nq = 0.0, na = 0.0, nb = 0.0;
  if (i < n) {
    nV = V[i];
    nq = w[i];
    if constexpr (MID) {
      na = vV[i];
      nb = vB[i];
    }
  }
  for (; i < n; i += stride) {
    const double Vi = nV, q0 = nq, a = na, b = nb;
    if (i + stride < n) {
      nV = V[i + stride];
      nq = w[i + stride];
      if constexpr (MID) {
        na = vV[i + stride];
        nb = vB[i + stride];
      }
    }
    ff v0p, q0p;
    bool pairs = split(q0, q0p);
    if constexpr (MID) {
      ff ap{0.0f, 0.0f}, bp{0.0f, 0.0f}, cp{0.0f, 0.0f};
      pairs = split(a, ap) & split(b, bp) & split(Vi, cp) & pairs;
      const ff sum = add(ap, bp);
      v0p = add(add(sum, sum), neg(cp));
    } else {
      pairs = split(Vi, v0p) & pairs;
    }
    double v = 0.0;
    VW res{0.0, 0.0};
    bool done = false, from_f32 = false;
    if (pairs) {
      const float v0f = v0p.h, q0f = q0p.h;
      float vf = v0f;
      for (int it = 0; it < 12; ++it) {
        const float q1 = (q0f + K.kaf * vf) * K.idf;
        const float Fv = vf - v0f - K.cf * (vf * (vf - K.thf) * (1.0f - vf) - q1);
        const float dF = 1.0f - K.cf * ((-3.0f * vf + K.th1) * vf - K.thf - K.rf);
        const float dv = __fdividef(Fv, dF);  // a Newton step needs no correctly rounded quotient
        vf -= dv;
        if (fabsf(dv) <= 1e-6f * fmaxf(1.0f, fabsf(vf))) break;
      }
      const float q1 = (q0f + K.kaf * vf) * K.idf;
      const bool f32_ok = fabsf(vf - v0f - K.cf * (vf * (vf - K.thf) * (1.0f - vf) - q1)) <= 1e-5f;
      // F(v_f) = ((c v_f + e2) v_f + e1) v_f + (c w0 / den - v0) on float pairs
      const ff a0 = add(mul(K.cidP, q0p), neg(v0p));
      const ff F = add(mul(add(mul(add(mul(K.cP, vf), K.e2P), vf), K.e1P), vf), a0);
      const float dFf = 1.0f - K.cf * ((-3.0f * vf + K.th1) * vf - K.thf - K.rf);
      const ff dv = mul(F, __fdividef(1.0f, dFf));
      // the float pairs carry F to ~1e-14 of the sum of its terms' sizes S;
      // near a fold of the cubic (F' small against S) that error, divided by
      // F', is too large, and float64 steps take over
      const float av = fabsf(vf);
      const float S = ((K.c3f * av + K.e2f) * av + K.e1f) * av + fabsf(a0.h);
      // the quasi-Newton step leaves about (F'' / 2 F') dv^2: below 1e-13
      const float d2F = 6.0f * K.cf * vf + K.e2x2;
      if (f32_ok && fabsf(dv.h) < 1e-5f && S < 8.0f * fabsf(dFf) &&
          dv.h * dv.h * fabsf(d2F) < 2e-13f * fabsf(dFf)) {
        const ff v1 = add(ff{vf, 0.0f}, neg(dv));
        res.v = widen(v1.h) + widen(v1.l);
        // w1 = (w0 + k alpha v1) / den with v1 ~ v_f - dv.h (dv.l k alpha is below 1e-19)
        const ff W = mul(add(q0p, mul(K.kaP, ff{vf, -dv.h})), K.idP);
        res.w = widen(W.h) + widen(W.l);
        done = true;
      } else if (isfinite(vf)) {
        v = widen(vf);
        from_f32 = true;
      }
    }
    // float64 Newton steps (rare: near folds of the cubic, unconverged
    // float32 phases, inputs outside the pairs' range), from v_f when the
    // float32 phase left a finite value, else from v0
    if (!done) res = be_newton64<MID>(K, a, b, Vi, q0, from_f32, v, err);
    if constexpr (FE) {
      const double t = fma(fma(-K.fa, res.v, K.fp1), res.v, K.fp0);
      const double v2 = fma(t, res.v, fma(-K.fa, res.w, res.v));
      res.w = fma(K.fka, res.v, K.fkz1 * res.w);
      res.v = v2;
    }
    V[i] = res.v;
    w[i] = res.w;
  }
}

// sum of V over inside nodes -> partial sums
__global__ void k_masked_sum(const double* __restrict__ V, const uint8_t* __restrict__ inside, int64_t n,
                             double* __restrict__ partial) {
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (inside[i]) acc += V[i];
  __shared__ double ws[32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
    s = warp_sum(s);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
  }
}

__global__ void k_ue(const double* __restrict__ V, const double* __restrict__ sum, double inv_count, double si,
                     double se, double* __restrict__ ue, int64_t n) {
  const double mean = sum[0] * inv_count;
  const double f = si / (si + se);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    ue[i] = f * (mean - V[i]);
}

int grid_blocks(int64_t n, int bs) {
  int64_t b = (n + bs - 1) / bs;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

int small_size(int m) { return SmallLayout{m}.total(); }
int small_res(int m) { return SmallLayout{m}.res(); }
int small_g(int m) { return SmallLayout{m}.g(); }
int small_hcol(int m) { return SmallLayout{m}.hcol(); }
int small_nrm2(int m) { return SmallLayout{m}.nrm2(); }
int small_y(int m) { return SmallLayout{m}.y(); }

int launch_correction(kfbi_handle* h, const double* x, double* corr) { return launch_correction_t(h, h->t, x, corr); }

int launch_correction_t(kfbi_handle* h, const Tables& t, const double* x, double* corr) {
  if (t.n_irr == 0) return KFBI_OK;
  if (launch_pdl(k_correction, dim3((t.n_irr + 127) / 128), dim3(128), 0, h->stream, t, x, corr,
                 (const int*)h->skip) != cudaSuccess)
    return launch_failed("correction");
  KFBI_CHECK_LAUNCH();
  return KFBI_OK;
}

int launch_spline(kfbi_handle* h, const double* psi, double* x) {
  const int M = h->t.M;
  k_spline<<<(M + 127) / 128, 128, 0, h->stream>>>(h->t.spline_G, psi, x, M);
  KFBI_CHECK_LAUNCH();
  return KFBI_OK;
}

int launch_limit64(kfbi_handle* h, const double* grid, const double* x, const double* base, double sgn, double* out) {
  return launch_limit64_t(h, h->t, grid, x, base, sgn, out);
}

int launch_limit64_t(kfbi_handle* h, const Tables& t, const double* grid, const double* x, const double* base,
                     double sgn, double* out) {
  if (launch_pdl(k_limit<double>, dim3((t.M + 127) / 128), dim3(128), 0, h->stream, t, h->grid, grid, x, base, sgn,
                 out, (const int*)h->skip) != cudaSuccess)
    return launch_failed("interface limit");
  KFBI_CHECK_LAUNCH();
  return KFBI_OK;
}

int launch_limit32_t(kfbi_handle* h, const Tables& t, const float* grid, const double* x, const double* base,
                     double sgn, double* out) {
  if (launch_pdl(k_limit<float>, dim3((t.M + 127) / 128), dim3(128), 0, h->stream, t, h->grid, grid, x, base, sgn,
                 out, (const int*)h->skip) != cudaSuccess)
    return launch_failed("interface limit");
  KFBI_CHECK_LAUNCH();
  return KFBI_OK;
}

int launch_limit32(kfbi_handle* h, const float* grid, const double* x, const double* base, double sgn, double* out) {
  if (launch_pdl(k_limit<float>, dim3((h->t.M + 127) / 128), dim3(128), 0, h->stream, h->t, h->grid, grid, x, base,
                 sgn, out, (const int*)h->skip) != cudaSuccess)
    return launch_failed("interface limit");
  KFBI_CHECK_LAUNCH();
  return KFBI_OK;
}

int launch_limit_user(kfbi_handle* h, const double* u, const double* x, const double* base, double sgn, double* out) {
  return launch_limit_user_t(h, h->t, u, x, base, sgn, out);
}

int launch_limit_user_t(kfbi_handle* h, const Tables& t, const double* u, const double* x, const double* base,
                        double sgn, double* out) {
  k_limit_user<<<(t.M + 127) / 128, 128, 0, h->stream>>>(t, h->grid, u, x, base, sgn, out);
  KFBI_CHECK_LAUNCH();
  return KFBI_OK;
}

int launch_residual(kfbi_handle* h, const double* src, double alpha, const double* corr, const double* u, double lambda,
                    double* res) {
  const int n1 = h->grid.N - 1;
  if (h->grid.bc == KFBI_BOX_NEUMANN) {
    const int P = h->grid.N + 1;
    k_residual_neumann<<<dim3(P, h->grid.dim == 3 ? P : 1), 128, 0, h->stream>>>(h->grid, src, alpha, u, lambda,
                                                                                   res);
  } else {
    k_residual<<<dim3(n1, h->grid.dim == 3 ? n1 : 1), 128, 0, h->stream>>>(h->grid, src, alpha, u, lambda, res);
  }
  if (corr != nullptr && h->t.n_irr > 0)
    k_scatter_add<<<(h->t.n_irr + 127) / 128, 128, 0, h->stream>>>(h->t, corr, res);
  KFBI_CHECK_LAUNCH_N(corr != nullptr && h->t.n_irr > 0 ? 2 : 1);
  return KFBI_OK;
}

int launch_residual_ff(kfbi_handle* h, const double* src, double alpha, const double* corr, const float* u32,
                       const double* u64, double lambda, float* res) {
  const int n1 = h->grid.N - 1;
  const double ih2 = 1.0 / (h->grid.h * h->grid.h);
  const double dg = -2.0 * h->grid.dim * ih2 - lambda;
  const float ih2_hi = (float)ih2, dg_hi = (float)dg;
  const float ih2_lo = (float)(ih2 - (double)ih2_hi), dg_lo = (float)(dg - (double)dg_hi);
  const float al_hi = (float)alpha, al_lo = (float)(alpha - (double)al_hi);
  if (h->grid.bc == KFBI_BOX_NEUMANN) {
    const int P = h->grid.N + 1;
    k_residual_ff_neumann<<<dim3(P, h->grid.dim == 3 ? P : 1), 128, 0, h->stream>>>(
        h->grid, u32, ih2_hi, ih2_lo, dg_hi, dg_lo, src, al_hi, al_lo, res);
    if (corr != nullptr && h->t.n_irr > 0)
      k_residual_irr_neumann<<<(h->t.n_irr + 127) / 128, 128, 0, h->stream>>>(h->grid, h->t, corr, u64, lambda, src,
                                                                              alpha, res);
  } else {
    k_residual_ff<<<dim3(n1, h->grid.dim == 3 ? n1 : 1), 128, 0, h->stream>>>(h->grid, u32, ih2_hi, ih2_lo, dg_hi,
                                                                               dg_lo, src, al_hi, al_lo, res);
    if (corr != nullptr && h->t.n_irr > 0)
      k_residual_irr<<<(h->t.n_irr + 127) / 128, 128, 0, h->stream>>>(h->grid, h->t, corr, u64, lambda, src, alpha,
                                                                      res, u32);
  }
  KFBI_CHECK_LAUNCH_N(corr != nullptr && h->t.n_irr > 0 ? 2 : 1);
  return KFBI_OK;
}

int launch_rank_one(kfbi_handle* h, const double* psi, double* out, double sgn) {
  const int M = h->t.M;
  double* slot = h->w.proj + KFBI_HISTORY * (KFBI_HISTORY + 2) + 4;
  int rc = vec_dots(h, h->t.ds, 1, M, psi, slot);
  if (rc) return rc;
  k_add_scalar<<<(M + 255) / 256, 256, 0, h->stream>>>(out, slot, sgn / h->t.area, M);
  KFBI_CHECK_LAUNCH();
  return KFBI_OK;
}

int launch_stim_source(kfbi_handle* h, const double* V, double lambda, const double* I, double c, double* f,
                       int64_t n) {
  k_stim_source<<<grid_blocks(n, 256), 256, 0, h->stream>>>(V, lambda, I, c, f, n);
  KFBI_CHECK_LAUNCH();
  return KFBI_OK;
}

int launch_ue_S(kfbi_handle* h, const double* V, const double* S, double* ue) {
  const int64_t total = field_count(h->grid);
  const int nb = RED_BLOCKS;
  k_phi_e<<<grid_blocks(total, 256), 256, 0, h->stream>>>(V, S, h->sigma_i, h->sigma_e, ue, total);
  k_masked_sum<<<nb, 256, 0, h->stream>>>(ue, h->t.inside_user, total, h->w.partial);
  k_dots_final<<<1, 256, 0, h->stream>>>(h->w.partial, nb, 1, h->w.partial + nb);
  k_sub_mean<<<grid_blocks(total, 256), 256, 0, h->stream>>>(ue, h->w.partial + nb, 1.0 / (double)h->t.n_inside,
                                                            total);
  KFBI_CHECK_LAUNCH_N(4);
  return KFBI_OK;
}

// out += sgn (1, 1) <(ds, ds), psi> / (2 |Gamma|) over the 2M entries of a
// coupled density pair (ds2 = (ds, ds) / 2 precomputed): the rank-one term
// of the coupled Neumann operator
int launch_rank_one_coupled(kfbi_handle* h, const double* psi, double* out, double sgn) {
  const int n = h->nk;
  double* slot = h->w.proj + KFBI_HISTORY * (KFBI_HISTORY + 2) + 4;
  int rc = vec_dots(h, h->w.ds2, 1, n, psi, slot);
  if (rc) return rc;
  k_add_scalar<<<(n + 255) / 256, 256, 0, h->stream>>>(out, slot, sgn / h->t.area, n);
  KFBI_CHECK_LAUNCH();
  return KFBI_OK;
}

// Float64 residual of the coupled 5/7-point system on the user layout (zero
// Dirichlet data), both components at once (Section 5.2, Eq. FDE):
//   r_i = a_i src_i - (sum_a d_i,a (u_i(+e_a) - 2 u_i + u_i(-e_a)) / h^2 - kappa (u_i - u_e)),
//   r_e = a_e src_e - (sum_a d_e,a (...) / h^2 + kappa (u_i - u_e));
// the corrections are added by a scatter afterwards.  One block row per
// (y, z) grid line.  The conductivities come pre-scaled by 1/h^2 (ci, ce)
// with the diagonals dgi = -2 sum ci - kappa, dge likewise.
struct CoupledStencil {
  double ci[3], ce[3], dgi, dge, kappa;
};

__device__ __forceinline__ double stencil_axes(const double* __restrict__ v, int64_t f, int x, int y, int z, int n1,
                                               int64_t s, int dim, double c0, double c1, double c2) {
  double acc = c0 * ((x > 0 ? v[f - 1] : 0.0) + (x < n1 - 1 ? v[f + 1] : 0.0));
  acc = fma(c1, (y > 0 ? v[f - n1] : 0.0) + (y < n1 - 1 ? v[f + n1] : 0.0), acc);
  if (dim == 3) acc = fma(c2, (z > 0 ? v[f - s] : 0.0) + (z < n1 - 1 ? v[f + s] : 0.0), acc);
  return acc;
}

__global__ void k_residual_coupled(GridParams gr, CoupledStencil cs, const double* __restrict__ src_i, double a_i,
                                   const double* __restrict__ src_e, double a_e, const double* __restrict__ ui,
                                   const double* __restrict__ ue, double* __restrict__ ri, double* __restrict__ re) {
  const int n1 = gr.N - 1;
  const int y = blockIdx.x, z = blockIdx.y;
  const int64_t s = (int64_t)n1 * n1;
  const int64_t base = (int64_t)z * s + (int64_t)y * n1;
  for (int x = threadIdx.x; x < n1; x += blockDim.x) {
    const int64_t f = base + x;
    const double vi = ui[f], ve = ue[f];
    double Li = stencil_axes(ui, f, x, y, z, n1, s, gr.dim, cs.ci[0], cs.ci[1], cs.ci[2]);
    double Le = stencil_axes(ue, f, x, y, z, n1, s, gr.dim, cs.ce[0], cs.ce[1], cs.ce[2]);
    Li = fma(cs.dgi, vi, fma(cs.kappa, ve, Li));
    Le = fma(cs.dge, ve, fma(cs.kappa, vi, Le));
    ri[f] = (src_i != nullptr ? a_i * src_i[f] : 0.0) - Li;
    re[f] = (src_e != nullptr ? a_e * src_e[f] : 0.0) - Le;
  }
}

CoupledStencil coupled_stencil(const kfbi_handle* h, double kappa) {
  CoupledStencil cs;
  const double ih2 = 1.0 / (h->grid.h * h->grid.h);
  double si = 0.0, se = 0.0;
  for (int a = 0; a < 3; ++a) {
    const bool on = a < h->grid.dim;
    cs.ci[a] = on ? h->cpl.di[a] * ih2 : 0.0;
    cs.ce[a] = on ? h->cpl.de[a] * ih2 : 0.0;
    si += cs.ci[a];
    se += cs.ce[a];
  }
  cs.dgi = -2.0 * si - kappa;
  cs.dge = -2.0 * se - kappa;
  cs.kappa = kappa;
  return cs;
}

int launch_residual_coupled(kfbi_handle* h, const double* src_i, double a_i, const double* src_e, double a_e,
                            const double* corr_i, const double* corr_e, const double* ui, const double* ue,
                            double kappa, double* ri, double* re) {
  const int n1 = h->grid.N - 1;
  k_residual_coupled<<<dim3(n1, h->grid.dim == 3 ? n1 : 1), 256, 0, h->stream>>>(
      h->grid, coupled_stencil(h, kappa), src_i, a_i, src_e, a_e, ui, ue, ri, re);
  int n = 1;
  if (h->t.n_irr > 0) {
    if (corr_i) {
      k_scatter_add<<<(h->t.n_irr + 127) / 128, 128, 0, h->stream>>>(h->t, corr_i, ri);
      ++n;
    }
    if (corr_e) {
      k_scatter_add<<<(h->t.n_irr + 127) / 128, 128, 0, h->stream>>>(h->t, corr_e, re);
      ++n;
    }
  }
  KFBI_CHECK_LAUNCH_N(n);
  return KFBI_OK;
}

// float pair (hi + lo) of a float64 constant
struct FPair {
  float hi, lo;
};
FPair fpair(double v) {
  const float hi = (float)v;
  return {hi, (float)(v - (double)hi)};
}

struct CoupledStencilFF {
  FPair ci[3], ce[3], dgi, dge, kappa, ai, ae;
};

// (acc, lo) += (c.hi + c.lo)(s + e) in float-float arithmetic
__device__ __forceinline__ void ff_mac(float& acc, float& lo, FPair c, float s, float e) {
  float p, ep, t;
  two_prod(c.hi, s, p, ep);
  ep = fmaf(c.hi, e, fmaf(c.lo, s, ep));
  two_sum(acc, p, acc, t);
  lo += t + ep;
}

// (s, e) = a + b exactly
__device__ __forceinline__ void ff_pair(float a, float b, float& s, float& e) { two_sum(a, b, s, e); }

// one component's L u in float-float from the padded float grid u (index 0
// of each axis the zero boundary value), plus kappa times the other
// component's value uo at the node
__device__ __forceinline__ void coupled_L_ff(const float* __restrict__ u, size_t p, int x, int y, int z, int n1,
                                             int N, size_t NN, int dim, const FPair* c, FPair dg, FPair kap,
                                             float uo, float& acc, float& lo) {
  float s, e;
  acc = 0.0f;
  lo = 0.0f;
  ff_pair(u[p - 1], x < n1 - 1 ? u[p + 1] : 0.0f, s, e);
  ff_mac(acc, lo, c[0], s, e);
  ff_pair(u[p - N], y < n1 - 1 ? u[p + N] : 0.0f, s, e);
  ff_mac(acc, lo, c[1], s, e);
  if (dim == 3) {
    ff_pair(u[p - NN], z < n1 - 1 ? u[p + NN] : 0.0f, s, e);
    ff_mac(acc, lo, c[2], s, e);
  }
  ff_mac(acc, lo, dg, u[p], 0.0f);
  ff_mac(acc, lo, kap, uo, 0.0f);
}

// r = a src - L u as a float (the float64 source split into a float pair on its bits)
__device__ __forceinline__ float ff_residual(const double* __restrict__ src, size_t f, FPair al, float acc, float lo) {
  if (src == nullptr) return -(acc + lo);
  const double sv = src[f];
  float sh, sl;
      src_pair(sv, sh, sl);
  float q, eq, h2, e4;
  two_prod(al.hi, sh, q, eq);
  eq = fmaf(al.hi, sl, fmaf(al.lo, sh, eq));
  two_sum(q, -acc, h2, e4);
  return h2 + (e4 + eq - lo);
}

// The coupled residual of a first refinement round, when (u_i, u_e) is
// exactly the pair of padded float grids of the float32 coupled solve just
// done: float-float arithmetic as in the scalar case (the float64 pipe is
// 1/64 of the float32 rate here), float32 result.  The irregular nodes are
// redone in float64 with their corrections by k_residual_irr_coupled.
__global__ void k_residual_ff_coupled(GridParams gr, CoupledStencilFF cs, const float* __restrict__ ui32,
                                      const float* __restrict__ ue32, const double* __restrict__ src_i,
                                      const double* __restrict__ src_e, float* __restrict__ ri,
                                      float* __restrict__ re) {
  const int N = gr.N, n1 = N - 1;
  const int y = blockIdx.x, z = blockIdx.y;
  const size_t NN = (size_t)N * N;
  const size_t pbase = gr.dim == 3 ? (size_t)(z + 1) * NN + (size_t)(y + 1) * N : (size_t)(y + 1) * N;
  const size_t ubase = gr.dim == 3 ? ((size_t)z * n1 + y) * n1 : (size_t)y * n1;
  for (int x = threadIdx.x; x < n1; x += blockDim.x) {
    const size_t p = pbase + x + 1;
    const float vi = ui32[p], ve = ue32[p];
    float acc, lo;
    coupled_L_ff(ui32, p, x, y, z, n1, N, NN, gr.dim, cs.ci, cs.dgi, cs.kappa, ve, acc, lo);
    ri[ubase + x] = ff_residual(src_i, ubase + x, cs.ai, acc, lo);
    coupled_L_ff(ue32, p, x, y, z, n1, N, NN, gr.dim, cs.ce, cs.dge, cs.kappa, vi, acc, lo);
    re[ubase + x] = ff_residual(src_e, ubase + x, cs.ae, acc, lo);
  }
}

// the irregular nodes of the coupled residual in float64 from the float64
// copies of (u_i, u_e), with their corrections
__global__ void k_residual_irr_coupled(GridParams gr, Tables t, CoupledStencil cs, const double* __restrict__ corr_i,
                                       const double* __restrict__ corr_e, const double* __restrict__ ui,
                                       const double* __restrict__ ue, const double* __restrict__ src_i, double a_i,
                                       const double* __restrict__ src_e, double a_e, float* __restrict__ ri,
                                       float* __restrict__ re) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.n_irr) return;
  const int n1 = gr.N - 1;
  const int64_t f = t.irr[i];
  const int64_t s = (int64_t)n1 * n1;
  const int x = (int)(f % n1), y = (int)((f / n1) % n1), z = gr.dim == 3 ? (int)(f / s) : 0;
  const double vi = ui[f], ve = ue[f];
  double Li = stencil_axes(ui, f, x, y, z, n1, s, gr.dim, cs.ci[0], cs.ci[1], cs.ci[2]);
  double Le = stencil_axes(ue, f, x, y, z, n1, s, gr.dim, cs.ce[0], cs.ce[1], cs.ce[2]);
  Li = fma(cs.dgi, vi, fma(cs.kappa, ve, Li));
  Le = fma(cs.dge, ve, fma(cs.kappa, vi, Le));
  const double bi = (src_i != nullptr ? a_i * src_i[f] : 0.0) + (corr_i != nullptr ? corr_i[i] : 0.0);
  const double be = (src_e != nullptr ? a_e * src_e[f] : 0.0) + (corr_e != nullptr ? corr_e[i] : 0.0);
  ri[f] = (float)(bi - Li);
  re[f] = (float)(be - Le);
}

int launch_residual_ff_coupled(kfbi_handle* h, const double* src_i, double a_i, const double* src_e, double a_e,
                               const double* corr_i, const double* corr_e, const double* ui, const double* ue,
                               double kappa, float* ri, float* re) {
  const int n1 = h->grid.N - 1;
  const CoupledStencil cs = coupled_stencil(h, kappa);
  CoupledStencilFF cf;
  for (int a = 0; a < 3; ++a) {
    cf.ci[a] = fpair(cs.ci[a]);
    cf.ce[a] = fpair(cs.ce[a]);
  }
  cf.dgi = fpair(cs.dgi);
  cf.dge = fpair(cs.dge);
  cf.kappa = fpair(kappa);
  cf.ai = fpair(a_i);
  cf.ae = fpair(a_e);
  k_residual_ff_coupled<<<dim3(n1, h->grid.dim == 3 ? n1 : 1), 128, 0, h->stream>>>(
      h->grid, cf, h->w.grid32, h->w.grid32b, src_i, src_e, ri, re);
  int n = 1;
  if (h->t.n_irr > 0 && (corr_i != nullptr || corr_e != nullptr)) {
    k_residual_irr_coupled<<<(h->t.n_irr + 127) / 128, 128, 0, h->stream>>>(h->grid, h->t, cs, corr_i, corr_e, ui, ue,
                                                                            src_i, a_i, src_e, a_e, ri, re);
    ++n;
  }
  KFBI_CHECK_LAUNCH_N(n);
  return KFBI_OK;
}

// V <- 2 ((a + b) - (c + d)) - V: the midpoint of the coupled float32 forms
// from both parts of each potential (v_V of the refined volume solve, v_B of
// the last refined residual)
__global__ void k_midpoint4(double* __restrict__ V, const double* __restrict__ a, const double* __restrict__ b,
                            const double* __restrict__ c, const double* __restrict__ d, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    V[i] = 2.0 * ((a[i] + b[i]) - (c[i] + d[i])) - V[i];
}

int launch_midpoint4(kfbi_handle* h, double* V, const double* a, const double* b, const double* c, const double* d,
                     int64_t n) {
  k_midpoint4<<<grid_blocks(n, 256), 256, 0, h->stream>>>(V, a, b, c, d, n);
  KFBI_CHECK_LAUNCH();
  return KFBI_OK;
}

// V <- 2 (a - b) - V (implicit midpoint from the potentials of the coupled
// solve: w = Phi_i - Phi_e)
__global__ void k_midpoint_diff(double* __restrict__ V, const double* __restrict__ a, const double* __restrict__ b,
                                int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    V[i] = 2.0 * (a[i] - b[i]) - V[i];
}

int launch_midpoint_diff(kfbi_handle* h, double* V, const double* a, const double* b, int64_t n) {
  k_midpoint_diff<<<grid_blocks(n, 256), 256, 0, h->stream>>>(V, a, b, n);
  KFBI_CHECK_LAUNCH();
  return KFBI_OK;
}

// dst = src - mean_Omega(src)
int launch_sub_mean(kfbi_handle* h, const double* src, double* dst) {
  const int64_t total = field_count(h->grid);
  const int nb = RED_BLOCKS;
  if (dst != src) KFBI_CUDA(cudaMemcpyAsync(dst, src, sizeof(double) * (size_t)total, cudaMemcpyDeviceToDevice, h->stream));
  k_masked_sum<<<nb, 256, 0, h->stream>>>(dst, h->t.inside_user, total, h->w.partial);
  k_dots_final<<<1, 256, 0, h->stream>>>(h->w.partial, nb, 1, h->w.partial + nb);
  k_sub_mean<<<grid_blocks(total, 256), 256, 0, h->stream>>>(dst, h->w.partial + nb, 1.0 / (double)h->t.n_inside,
                                                             total);
  KFBI_CHECK_LAUNCH_N(3);
  return KFBI_OK;
}

int launch_lincomb(kfbi_handle* h, double* y, double a, const double* x, double b, int64_t n) {
  k_lincomb<<<grid_blocks(n, 256), 256, 0, h->stream>>>(y, a, x, b, n);
  KFBI_CHECK_LAUNCH();
  return KFBI_OK;
}

int launch_scatter_grid(kfbi_handle* h, const double* corr, double* grid_user) {
  const int64_t total = field_count(h->grid);
  k_scatter<<<grid_blocks(total, 256), 256, 0, h->stream>>>(h->t, corr, grid_user, total);
  if (h->t.n_irr > 0) k_scatter2<<<(h->t.n_irr + 127) / 128, 128, 0, h->stream>>>(h->t, corr, grid_user);
  KFBI_CHECK_LAUNCH_N(h->t.n_irr > 0 ? 2 : 1);
  return KFBI_OK;
}

int launch_padded_to_user(kfbi_handle* h, const double* padded, double* user) {
  const int n1 = h->grid.N - 1;
  const int64_t total = h->grid.dim == 3 ? (int64_t)n1 * n1 * n1 : (int64_t)n1 * n1;
  k_pad_to_user<<<grid_blocks(total, 256), 256, 0, h->stream>>>(h->grid, padded, user, total);
  KFBI_CHECK_LAUNCH();
  return KFBI_OK;
}

// G = H H^T (k x k), b = H g, gg = g . g for the k <= KFBI_HISTORY stored
// right-hand sides H (rows of length M), in one launch
int launch_gram(kfbi_handle* h, const double* H, int k, const double* g, double* G, double* b, double* gg) {
  const int n = h->nk;
  int nb = (n + 255) / 256;
  if (nb > RED_BLOCKS) nb = RED_BLOCKS;
  double* pt = h->w.partial;
  unsigned* c = h->w.counter;
  switch (k) {
    case 0: k_gram<0><<<nb, 256, 0, h->stream>>>(H, n, g, n, pt, c, G, b, gg); break;
    case 1: k_gram<1><<<nb, 256, 0, h->stream>>>(H, n, g, n, pt, c, G, b, gg); break;
    case 2: k_gram<2><<<nb, 256, 0, h->stream>>>(H, n, g, n, pt, c, G, b, gg); break;
    case 3: k_gram<3><<<nb, 256, 0, h->stream>>>(H, n, g, n, pt, c, G, b, gg); break;
    case 4: k_gram<4><<<nb, 256, 0, h->stream>>>(H, n, g, n, pt, c, G, b, gg); break;
    case 5: k_gram<5><<<nb, 256, 0, h->stream>>>(H, n, g, n, pt, c, G, b, gg); break;
    case 6: k_gram<6><<<nb, 256, 0, h->stream>>>(H, n, g, n, pt, c, G, b, gg); break;
    case 7: k_gram<7><<<nb, 256, 0, h->stream>>>(H, n, g, n, pt, c, G, b, gg); break;
    case 8: k_gram<8><<<nb, 256, 0, h->stream>>>(H, n, g, n, pt, c, G, b, gg); break;
    default:
      set_error("history length %d above %d", k, KFBI_HISTORY);
      return KFBI_ERR_ARG;
  }
  KFBI_CHECK_LAUNCH();
  return KFBI_OK;
}

int vec_dots(kfbi_handle* h, const double* V, int nvec, int ld, const double* w, double* out_dev) {
  const int n = h->nk;
  int nb = (n + 255) / 256;
  if (nb > RED_BLOCKS) nb = RED_BLOCKS;
  k_dots_partial<<<dim3(nb, nvec), 256, 0, h->stream>>>(V, ld, w, n, h->w.partial);
  k_dots_final<<<nvec, 256, 0, h->stream>>>(h->w.partial, nb, nvec, out_dev);
  KFBI_CHECK_LAUNCH_N(2);
  return KFBI_OK;
}

int vec_update(kfbi_handle* h, double* w, const double* V, int nvec, int ld, const double* coef_dev, double sign) {
  const int n = h->nk;
  k_update<<<grid_blocks(n, 256), 256, 0, h->stream>>>(w, V, nvec, ld, coef_dev, sign, n);
  KFBI_CHECK_LAUNCH();
  return KFBI_OK;
}

int vec_axpby(kfbi_handle* h, double* y, double a, const double* x, double b, int n) {
  k_axpby<<<(n + 255) / 256, 256, 0, h->stream>>>(y, a, x, b, n);
  KFBI_CHECK_LAUNCH();
  return KFBI_OK;
}

int vec_scale_by_norm(kfbi_handle* h, double* v, const double* w, const double* norm_dev, int n) {
  k_scale_norm<<<(n + 255) / 256, 256, 0, h->stream>>>(v, w, norm_dev, n, nullptr);
  KFBI_CHECK_LAUNCH();
  return KFBI_OK;
}

int vec_copy(kfbi_handle* h, double* dst, const double* src, int n) {
  KFBI_CUDA(cudaMemcpyAsync(dst, src, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, h->stream));
  return KFBI_OK;
}

int arnoldi_givens(kfbi_handle* h, double* small, int j, int m) {
  k_givens<<<1, 1, 0, h->stream>>>(small, m, j);
  KFBI_CHECK_LAUNCH();
  return KFBI_OK;
}

int arnoldi_solve(kfbi_handle* h, double* small, int k, int m) {
  k_backsolve<<<1, 1, 0, h->stream>>>(small, m, k);
  KFBI_CHECK_LAUNCH();
  return KFBI_OK;
}

// one CGS2 Arnoldi step on wv = A v_j (basis V, leading dimension ld,
// restart m): H(:, j), the Givens update, v_{j+1}, and at small[res],
// small[res + 1] the residual estimate and the stop flag (also written to
// h->w.stop).  Launches carry h->skip.
int arnoldi_step(kfbi_handle* h, double* V, int ld, double* wv, int j, int m, double gnorm, double tol) {
  const int n = h->nk;
  int nb = (n + 255) / 256;
  if (nb > ARN_BLOCKS) nb = ARN_BLOCKS;
  SmallLayout L{m};
  double* s = h->w.small;
  const int nv = j + 1;
  const int* skip = h->skip;
  cudaStream_t st = h->stream;
  if (launch_pdl(k_arn_gs<false>, dim3(nb), dim3(256), 0, st, wv, (const double*)V, ld, n, nv, (const double*)nullptr,
                 h->w.partial, h->w.counter, s + L.hcol(), skip) != cudaSuccess ||
      launch_pdl(k_arn_gs<true>, dim3(nb), dim3(256), 0, st, wv, (const double*)V, ld, n, nv,
                 (const double*)(s + L.hcol()), h->w.partial, h->w.counter, s + L.y(), skip) != cudaSuccess ||
      launch_pdl(k_arn_close, dim3(nb), dim3(256), 0, st, wv, (const double*)V, ld, n, nv, s, m, j, h->w.partial,
                 h->w.counter, gnorm, tol, h->w.stop, skip) != cudaSuccess ||
      launch_pdl(k_scale_norm, dim3((n + 255) / 256), dim3(256), 0, st, V + (size_t)(j + 1) * ld, (const double*)wv,
                 (const double*)(s + L.nrm2()), n, skip) != cudaSuccess)
    return launch_failed("Arnoldi step");
  KFBI_CHECK_LAUNCH_N(4);
  return KFBI_OK;
}

int arnoldi_add(kfbi_handle* h, double* small, int m, int n) {
  k_add_small<<<1, 128, 0, h->stream>>>(small, m, n);
  KFBI_CHECK_LAUNCH();
  return KFBI_OK;
}

int launch_init_arnoldi(kfbi_handle* h, double* small, int m) {
  k_init_arnoldi<<<1, 128, 0, h->stream>>>(small, m);
  KFBI_CHECK_LAUNCH();
  return KFBI_OK;
}

int launch_react_fe(const kfbi_fhn* p, double k, double* V, double* w, int64_t n, cudaStream_t s) {
  k_react_fe<<<grid_blocks(n, 256), 256, 0, s>>>(*p, k, V, w, n);
  KFBI_CHECK_LAUNCH();
  return KFBI_OK;
}

static ffl::ff to_pair(double x) {
  const float h = (float)x;
  return ffl::ff{h, (float)(x - (double)h)};
}

int launch_react_be(const kfbi_fhn* p, double k, double* V, double* w, int64_t n, int* err, cudaStream_t s,
                    const double* vV, const double* vB, bool fe_next) {
  BeConsts K;
  K.c = k * p->H / p->Cm;
  const double den = 1.0 + k * p->zeta, ka = k * p->alpha;
  K.inv_den = 1.0 / den;
  K.e2 = -K.c * (1.0 + p->theta);
  K.e1 = 1.0 + K.c * p->theta + K.c * ka * K.inv_den;
  K.cid = K.c * K.inv_den;
  K.kid = ka * K.inv_den;
  K.cf = (float)K.c;
  K.rf = (float)(ka / den);
  K.thf = (float)p->theta;
  K.kaf = (float)ka;
  K.idf = (float)K.inv_den;
  K.th1 = 2.0f * (1.0f + K.thf);
  K.c3f = (float)std::fabs(K.c);
  K.e2f = (float)std::fabs(K.e2);
  K.e1f = (float)std::fabs(K.e1);
  K.e2x2 = (float)(2.0 * K.e2);
  K.cP = to_pair(K.c);
  K.e2P = to_pair(K.e2);
  K.e1P = to_pair(K.e1);
  K.cidP = to_pair(K.cid);
  K.kaP = to_pair(ka);
  K.idP = to_pair(K.inv_den);
  // the next step's forward Euler: the constants of k_react_fe
  K.fa = k * p->H / p->Cm;
  K.fka = k * p->alpha;
  K.fkz1 = 1.0 - k * p->zeta;
  K.fp1 = K.fa * (1.0 + p->theta);
  K.fp0 = -K.fa * p->theta;
  const int nb = grid_blocks(n, 256);
  if (vV != nullptr) {
    if (fe_next)
      k_react_be<true, true><<<nb, 256, 0, s>>>(K, V, w, vV, vB, n, err);
    else
      k_react_be<true, false><<<nb, 256, 0, s>>>(K, V, w, vV, vB, n, err);
  } else if (fe_next) {
    k_react_be<false, true><<<nb, 256, 0, s>>>(K, V, w, nullptr, nullptr, n, err);
  } else {
    k_react_be<false, false><<<nb, 256, 0, s>>>(K, V, w, nullptr, nullptr, n, err);
  }
  KFBI_CHECK_LAUNCH();
  return KFBI_OK;
}

int launch_ue(kfbi_handle* h, const double* V, double* ue) {
  const int64_t total = field_count(h->grid);
  const int nb = RED_BLOCKS;
  k_masked_sum<<<nb, 256, 0, h->stream>>>(V, h->t.inside_user, total, h->w.partial);
  k_dots_final<<<1, 256, 0, h->stream>>>(h->w.partial, nb, 1, h->w.partial + nb);
  k_ue<<<grid_blocks(total, 256), 256, 0, h->stream>>>(V, h->w.partial + nb, 1.0 / (double)h->t.n_inside,
                                                       h->sigma_i, h->sigma_e, ue, total);
  KFBI_CHECK_LAUNCH_N(3);
  return KFBI_OK;
}

}  // namespace kfbi
