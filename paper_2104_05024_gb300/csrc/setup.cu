// Setup of the KFBI tables (Section 6: classify the grid nodes, locate the
// crossings of the interface with grid lines, compute normals, tangents and
// curvatures there and at the interface nodes).
//
// This translation unit is compiled with -fmad=false: level sets, node
// coordinates, cell indices and bisection midpoints use only correctly rounded
// +, -, *, / and sqrt in a fixed order, so classification, crossings and
// interface-to-cell indexing are reproducible bit for bit by any IEEE
// implementation that evaluates the same expressions.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

namespace kfbi {
namespace {

constexpr int BISECT_ITERS = 64;

// ------------------------------------------------------------ level sets
__host__ __device__ inline double phi_ellipse2(double x, double y, const double* p) {
  const double xr = p[2] * x + p[3] * y;
  const double yr = p[2] * y - p[3] * x;
  const double u = xr / p[0];
  const double v = yr / p[1];
  return (u * u + v * v) - 1.0;
}

__host__ __device__ inline double phi_ellipsoid(double x, double y, double z, double a, double b, double c) {
  const double u = x / a;
  const double v = y / b;
  const double w = z / c;
  return ((u * u + v * v) + w * w) - 1.0;
}

__host__ __device__ inline double phi_star(double x, double y, double z, double A, double B) {
  const double x2 = x * x;
  const double y2 = y * y;
  const double z2 = z * z;
  const double s2 = x2 + y2;
  const double r2 = s2 + z2;
  const double rho = sqrt(r2);
  double g = 0.0;
  if (s2 > 0.0) {
    const double s = sqrt(s2);
    g = ((x2 - y2) / s2) * ((s / rho) * (3.0 - 4.0 * (s2 / r2)));
  }
  return (rho - A) - B * g;
}

__host__ __device__ inline double comp_phi(const GeomParams& g, int comp, double x, double y, double z) {
  switch (g.kind) {
    case KFBI_ELLIPSE2: return phi_ellipse2(x, y, g.p);
    case KFBI_ELLIPSOID3: return phi_ellipsoid(x, y, z, g.p[0], g.p[1], g.p[2]);
    case KFBI_STAR3: return phi_star(x, y, z, g.p[0], g.p[1]);
    default: {
      const int o = comp == 0 ? 0 : 3;
      return phi_ellipsoid(x, y, z, g.p[o], g.p[o + 1], g.p[o + 2]);
    }
  }
}

// enclosed side of one surface: Phi <= 0, except the hole of the shell (Phi < 0)
__host__ __device__ inline bool comp_pred(const GeomParams& g, int comp, double x, double y, double z) {
  const double ph = comp_phi(g, comp, x, y, z);
  if (g.kind == KFBI_SHELL3 && comp == 1) return ph < 0.0;
  return ph <= 0.0;
}

__host__ __device__ inline bool inside_pt(const GeomParams& g, double x, double y, double z) {
  if (g.kind == KFBI_SHELL3) return comp_pred(g, 0, x, y, z) && !comp_pred(g, 1, x, y, z);
  return comp_pred(g, 0, x, y, z);
}

__host__ __device__ inline double node_coord(const GridParams& gr, int k) { return gr.lo + (double)k * gr.h; }

// --------------------------------------------------------------- 2-jets
struct Jet {
  double v, g[3], H[3][3];
};

__host__ __device__ inline Jet jconst(double c) {
  Jet r;
  r.v = c;
  for (int i = 0; i < 3; ++i) {
    r.g[i] = 0.0;
    for (int j = 0; j < 3; ++j) r.H[i][j] = 0.0;
  }
  return r;
}
__host__ __device__ inline Jet jvar(double x, int k) {
  Jet r = jconst(x);
  r.g[k] = 1.0;
  return r;
}
__host__ __device__ inline Jet jadd(const Jet& a, const Jet& b) {
  Jet r;
  r.v = a.v + b.v;
  for (int i = 0; i < 3; ++i) {
    r.g[i] = a.g[i] + b.g[i];
    for (int j = 0; j < 3; ++j) r.H[i][j] = a.H[i][j] + b.H[i][j];
  }
  return r;
}
__host__ __device__ inline Jet jscale(const Jet& a, double s) {
  Jet r;
  r.v = a.v * s;
  for (int i = 0; i < 3; ++i) {
    r.g[i] = a.g[i] * s;
    for (int j = 0; j < 3; ++j) r.H[i][j] = a.H[i][j] * s;
  }
  return r;
}
__host__ __device__ inline Jet jaddc(const Jet& a, double c) {
  Jet r = a;
  r.v = a.v + c;
  return r;
}
__host__ __device__ inline Jet jmul(const Jet& a, const Jet& b) {
  Jet r;
  r.v = a.v * b.v;
  for (int i = 0; i < 3; ++i) {
    r.g[i] = a.g[i] * b.v + b.g[i] * a.v;
    for (int j = 0; j < 3; ++j)
      r.H[i][j] = a.H[i][j] * b.v + b.H[i][j] * a.v + a.g[i] * b.g[j] + b.g[i] * a.g[j];
  }
  return r;
}
__host__ __device__ inline Jet jrecip(const Jet& a) {
  Jet r;
  const double q = 1.0 / a.v;
  r.v = q;
  for (int i = 0; i < 3; ++i) {
    r.g[i] = -a.g[i] * q * q;
    for (int j = 0; j < 3; ++j) r.H[i][j] = -a.H[i][j] * q * q + 2.0 * a.g[i] * a.g[j] * q * q * q;
  }
  return r;
}
__host__ __device__ inline Jet jdiv(const Jet& a, const Jet& b) { return jmul(a, jrecip(b)); }
__host__ __device__ inline Jet jsqrt(const Jet& a) {
  Jet r;
  const double s = sqrt(a.v);
  r.v = s;
  for (int i = 0; i < 3; ++i) {
    r.g[i] = a.g[i] / (2.0 * s);
    for (int j = 0; j < 3; ++j) r.H[i][j] = a.H[i][j] / (2.0 * s) - a.g[i] * a.g[j] / (4.0 * s * s * s);
  }
  return r;
}

__host__ __device__ Jet phi_jet(const GeomParams& gp, int comp, const double* P) {
  const int d = gp.dim;
  Jet X = jvar(P[0], 0), Y = jvar(P[1], 1);
  Jet Z = d == 3 ? jvar(P[2], 2) : jconst(0.0);
  const double* p = gp.p;
  if (gp.kind == KFBI_ELLIPSE2) {
    Jet u = jscale(jadd(jscale(X, p[2]), jscale(Y, p[3])), 1.0 / p[0]);
    Jet v = jscale(jadd(jscale(Y, p[2]), jscale(X, -p[3])), 1.0 / p[1]);
    return jaddc(jadd(jmul(u, u), jmul(v, v)), -1.0);
  }
  if (gp.kind == KFBI_ELLIPSOID3 || gp.kind == KFBI_SHELL3) {
    const int o = (gp.kind == KFBI_SHELL3 && comp == 1) ? 3 : 0;
    Jet u = jscale(X, 1.0 / p[o]), v = jscale(Y, 1.0 / p[o + 1]), w = jscale(Z, 1.0 / p[o + 2]);
    return jaddc(jadd(jadd(jmul(u, u), jmul(v, v)), jmul(w, w)), -1.0);
  }
  // star body; the B term is dropped on the polar axis (see the oracle's reading)
  const double A = p[0], B = p[1];
  Jet x2 = jmul(X, X), y2 = jmul(Y, Y), z2 = jmul(Z, Z);
  Jet s2 = jadd(x2, y2);
  Jet r2 = jadd(s2, z2);
  Jet out = jaddc(jsqrt(r2), -A);
  if (s2.v > 0.0) {
    Jet t1 = jdiv(jadd(x2, jscale(y2, -1.0)), s2);
    Jet t2 = jdiv(jsqrt(s2), jsqrt(r2));
    Jet t3 = jaddc(jscale(jdiv(s2, r2), -4.0), 3.0);
    Jet gterm = jmul(t1, jmul(t2, t3));
    out = jadd(out, jscale(gterm, -B));
  }
  return out;
}

// outward normal of Omega and shape operator S = P Hess P / |grad| at P
__host__ __device__ void normal_shape(const GeomParams& gp, int comp, const double* P, double* n, double S[3][3]) {
  const int d = gp.dim;
  Jet J = phi_jet(gp, comp, P);
  double gn = 0.0;
  for (int i = 0; i < d; ++i) gn += J.g[i] * J.g[i];
  gn = sqrt(gn);
  for (int i = 0; i < 3; ++i) n[i] = i < d ? J.g[i] / gn : 0.0;
  double Pm[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Pm[i][j] = (i < d && j < d) ? ((i == j ? 1.0 : 0.0) - n[i] * n[j]) : 0.0;
  double T[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double a = 0.0;
      for (int k = 0; k < 3; ++k) a += Pm[i][k] * J.H[k][j];
      T[i][j] = a;
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double a = 0.0;
      for (int k = 0; k < 3; ++k) a += T[i][k] * Pm[k][j];
      S[i][j] = a / gn;
    }
  if (gp.kind == KFBI_SHELL3 && comp == 1) {
    for (int i = 0; i < 3; ++i) {
      n[i] = -n[i];
      for (int j = 0; j < 3; ++j) S[i][j] = -S[i][j];
    }
  }
}

// Gaussian elimination with partial pivoting: solve A x = b in place (n <= 10)
__host__ __device__ bool gauss_solve(double* A, double* b, int n, int lda) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    double best = fabs(A[c * lda + c]);
    for (int r = c + 1; r < n; ++r) {
      const double v = fabs(A[r * lda + c]);
      if (v > best) {
        best = v;
        piv = r;
      }
    }
    if (best == 0.0) return false;
    if (piv != c) {
      for (int k = 0; k < n; ++k) {
        const double t = A[c * lda + k];
        A[c * lda + k] = A[piv * lda + k];
        A[piv * lda + k] = t;
      }
      const double t = b[c];
      b[c] = b[piv];
      b[piv] = t;
    }
    for (int r = c + 1; r < n; ++r) {
      const double f = A[r * lda + c] / A[c * lda + c];
      if (f != 0.0) {
        for (int k = c; k < n; ++k) A[r * lda + k] -= f * A[c * lda + k];
        b[r] -= f * b[c];
      }
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double a = b[r];
    for (int k = r + 1; k < n; ++k) a -= A[r * lda + k] * b[k];
    b[r] = a / A[r * lda + r];
  }
  return true;
}

// ------------------------------------------------------------- kernels
__global__ void k_classify(GeomParams gp, GridParams gr, uint8_t* inside, int64_t total) {
  const int n1 = gr.N - 1;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < total; f += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(f % n1) + 1;
    const int y = (int)((f / n1) % n1) + 1;
    const int z = gr.dim == 3 ? (int)(f / ((int64_t)n1 * n1)) + 1 : 0;
    const double X = node_coord(gr, x), Y = node_coord(gr, y), Z = gr.dim == 3 ? node_coord(gr, z) : 0.0;
    inside[f] = inside_pt(gp, X, Y, Z) ? 1 : 0;
  }
}

__host__ __device__ inline int64_t axis_stride(int a, int n1) {
  return a == 0 ? 1 : (a == 1 ? (int64_t)n1 : (int64_t)n1 * n1);
}
__host__ __device__ inline int axis_index(int64_t f, int a, int n1) {
  return (int)((f / axis_stride(a, n1)) % n1);
}

// flags: irregular (mode 0) or crossing edges along axis `a` (mode 1)
__global__ void k_flags(GridParams gr, const uint8_t* inside, int64_t total, int mode, int a, uint8_t* flag, int* err) {
  const int n1 = gr.N - 1;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < total; f += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t me = inside[f];
    if (mode == 0) {
      bool irr = false;
      for (int ax = 0; ax < gr.dim; ++ax) {
        const int k = axis_index(f, ax, n1);
        const int64_t st = axis_stride(ax, n1);
        const uint8_t lo = k > 0 ? inside[f - st] : 0;
        const uint8_t hi = k < n1 - 1 ? inside[f + st] : 0;
        if (lo != me || hi != me) irr = true;
        if (me && (k == 0 || k == n1 - 1)) atomicOr(err, DEVERR_GEOMETRY);
      }
      flag[f] = irr ? 1 : 0;
    } else {
      const int k = axis_index(f, a, n1);
      flag[f] = (k < n1 - 1 && inside[f + axis_stride(a, n1)] != me) ? 1 : 0;
    }
  }
}

// two-pass ordered compaction of flags into increasing indices
constexpr int CB = 1024;
__global__ void k_count(const uint8_t* flag, int64_t total, int* counts) {
  __shared__ int s;
  if (threadIdx.x == 0) s = 0;
  __syncthreads();
  const int64_t f = blockIdx.x * (int64_t)CB + threadIdx.x;
  const int c = __syncthreads_count(f < total && flag[f]);
  if (threadIdx.x == 0) counts[blockIdx.x] = c;
}
__global__ void k_write(const uint8_t* flag, int64_t total, const int* offsets, int32_t* out) {
  __shared__ int warp_tot[CB / 32];
  const int64_t f = blockIdx.x * (int64_t)CB + threadIdx.x;
  const bool on = f < total && flag[f];
  const unsigned bal = __ballot_sync(0xffffffffu, on);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) warp_tot[wid] = __popc(bal);
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int w = 0; w < CB / 32; ++w) {
      const int t = warp_tot[w];
      warp_tot[w] = acc;
      acc += t;
    }
  }
  __syncthreads();
  if (on) {
    const int pos = offsets[blockIdx.x] + warp_tot[wid] + __popc(bal & ((1u << lane) - 1u));
    out[pos] = (int32_t)f;
  }
}

// crossing points by bisection on the surface whose predicate changes
__global__ void k_bisect(GeomParams gp, GridParams gr, const int32_t* c_lo, const int32_t* c_axis, int n, double* c_z,
                         int8_t* c_comp, int* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int n1 = gr.N - 1;
  const int64_t f = c_lo[i];
  const int a = c_axis[i];
  int k[3] = {(int)(f % n1) + 1, (int)((f / n1) % n1) + 1, gr.dim == 3 ? (int)(f / ((int64_t)n1 * n1)) + 1 : 0};
  double X[3] = {node_coord(gr, k[0]), node_coord(gr, k[1]), gr.dim == 3 ? node_coord(gr, k[2]) : 0.0};
  double Xh[3] = {X[0], X[1], X[2]};
  Xh[a] = node_coord(gr, k[a] + 1);
  const int ncomp = gp.kind == KFBI_SHELL3 ? 2 : 1;
  int comp = -1;
  for (int c = 0; c < ncomp; ++c) {
    if (comp_pred(gp, c, X[0], X[1], X[2]) != comp_pred(gp, c, Xh[0], Xh[1], Xh[2])) {
      if (comp >= 0) atomicOr(err, DEVERR_GEOMETRY);
      comp = c;
    }
  }
  if (comp < 0) {
    atomicOr(err, DEVERR_GEOMETRY);
    comp = 0;
  }
  double lo = X[a], hi = Xh[a];
  const bool plo = comp_pred(gp, comp, X[0], X[1], X[2]);
  double P[3] = {X[0], X[1], X[2]};
  for (int it = 0; it < BISECT_ITERS; ++it) {
    const double mid = 0.5 * (lo + hi);
    P[a] = mid;
    if (comp_pred(gp, comp, P[0], P[1], P[2]) == plo) lo = mid;
    else hi = mid;
  }
  c_z[i] = 0.5 * (lo + hi);
  c_comp[i] = (int8_t)comp;
}

// ---- local quadratic surface fit (3-D) ----
__host__ __device__ void tangent_basis(const double* n, double* t1, double* t2) {
  int k = 0;
  double best = fabs(n[0]);
  for (int ax = 1; ax < 3; ++ax)
    if (fabs(n[ax]) < best) {
      best = fabs(n[ax]);
      k = ax;
    }
  double e[3] = {0.0, 0.0, 0.0};
  e[k] = 1.0;
  t1[0] = e[1] * n[2] - e[2] * n[1];
  t1[1] = e[2] * n[0] - e[0] * n[2];
  t1[2] = e[0] * n[1] - e[1] * n[0];
  const double l = sqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
  for (int i = 0; i < 3; ++i) t1[i] /= l;
  t2[0] = n[1] * t1[2] - n[2] * t1[1];
  t2[1] = n[2] * t1[0] - n[0] * t1[2];
  t2[2] = n[0] * t1[1] - n[1] * t1[0];
}

// weights w0[K] (value) and wg[3][K] (surface gradient) of the quadratic fit at z
__host__ __device__ bool fit_weights(const double* nodes, const int* ids, int K, const double* z, const double* n, double* w0,
                            double (*wg)[PATCH_MAX]) {
  double t1[3], t2[3];
  tangent_basis(n, t1, t2);
  double s[PATCH_MAX], t[PATCH_MAX];
  double ell = 0.0;
  for (int k = 0; k < K; ++k) {
    const double* X = nodes + 3 * (size_t)ids[k];
    const double D0 = X[0] - z[0], D1 = X[1] - z[1], D2 = X[2] - z[2];
    ell = fmax(ell, sqrt(D0 * D0 + D1 * D1 + D2 * D2));
    s[k] = D0 * t1[0] + D1 * t1[1] + D2 * t1[2];
    t[k] = D0 * t2[0] + D1 * t2[1] + D2 * t2[2];
  }
  for (int k = 0; k < K; ++k) {
    s[k] /= ell;
    t[k] /= ell;
  }
  double V[PATCH_MAX][6];
  for (int k = 0; k < K; ++k) {
    V[k][0] = 1.0;
    V[k][1] = s[k];
    V[k][2] = t[k];
    V[k][3] = s[k] * s[k];
    V[k][4] = s[k] * t[k];
    V[k][5] = t[k] * t[k];
  }
  // rows r = 0, 1, 2 of the (pseudo-)inverse
  double rows[3][PATCH_MAX];
  if (K == 6) {
    for (int r = 0; r < 3; ++r) {
      double A[36], b[6];
      for (int i = 0; i < 6; ++i) {
        for (int j = 0; j < 6; ++j) A[i * 6 + j] = V[j][i];  // V^T
        b[i] = i == r ? 1.0 : 0.0;
      }
      if (!gauss_solve(A, b, 6, 6)) return false;
      for (int k = 0; k < 6; ++k) rows[r][k] = b[k];
    }
  } else {
    double Gm[36];
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) {
        double a = 0.0;
        for (int k = 0; k < K; ++k) a += V[k][i] * V[k][j];
        Gm[i * 6 + j] = a;
      }
    for (int r = 0; r < 3; ++r) {
      double A[36], b[6];
      for (int i = 0; i < 36; ++i) A[i] = Gm[i];
      for (int i = 0; i < 6; ++i) b[i] = i == r ? 1.0 : 0.0;
      if (!gauss_solve(A, b, 6, 6)) return false;
      for (int k = 0; k < K; ++k) {
        double a = 0.0;
        for (int l = 0; l < 6; ++l) a += V[k][l] * b[l];
        rows[r][k] = a;
      }
    }
  }
  for (int k = 0; k < K; ++k) {
    w0[k] = rows[0][k];
    for (int i = 0; i < 3; ++i) wg[i][k] = (t1[i] * rows[1][k] + t2[i] * rows[2][k]) / ell;
  }
  return true;
}

__host__ __device__ int locate_tri(const GeomParams& gp, const double* cube_t, int comp, const double* P) {
  double q[3] = {P[0], P[1], P[2]};
  if (gp.comp_map[comp] == KFBI_MAP_ELLIPSOID) {
    q[0] = P[0] / gp.comp_axes[comp][0];
    q[1] = P[1] / gp.comp_axes[comp][1];
    q[2] = P[2] / gp.comp_axes[comp][2];
  }
  int k = 0;
  double best = fabs(q[0]);
  for (int ax = 1; ax < 3; ++ax)
    if (fabs(q[ax]) > best) {
      best = fabs(q[ax]);
      k = ax;
    }
  const int face = 2 * k + (q[k] < 0.0 ? 1 : 0);
  const double u = q[(k + 1) % 3] / best;
  const double v = q[(k + 2) % 3] / best;
  const int n = gp.cube_n;
  int i = 0, j = 0;
  for (int m = 1; m < n; ++m) {
    if (cube_t[m] <= u) i = m;
    if (cube_t[m] <= v) j = m;
  }
  const double fu = (u - cube_t[i]) / (cube_t[i + 1] - cube_t[i]);
  const double fv = (v - cube_t[j]) / (cube_t[j + 1] - cube_t[j]);
  const int half = (fu + fv > 1.0) ? 1 : 0;
  return gp.comp_tri_offset[comp] + (((face * n + j) * n + i) * 2 + half);
}

struct DensityInputs {
  const double* nodes;      // [M][dim]
  const int32_t* patch_ids; // [n_tri][PATCH_MAX]
  const int32_t* patch_cnt; // [n_tri]
  const double* cube_t;
  int M;
  // mesh-only domains: each node's fit triangle and every triangle's local
  // surface (see below)
  const int32_t* vtri = nullptr;
  const double* tri_fit = nullptr;
};

// ---- domains given only by a closed triangle mesh (KFBI_MESH3) ----
// Section 5.3 / Example 4: the triangles are all there is.  Classification is
// the parity of ray crossings along x; every edge is evaluated once, in its
// canonical direction (lower vertex index first), as
//   E(p) = (Q_u - P_u)(p_v - P_v) - (Q_v - P_v)(p_u - P_u)
// (u, v the axes after the ray's axis), so the two triangles of an edge see
// the same value; E = 0 takes the sign of the symbolic perturbation
// p + (eps, eps^2).  A line meets a triangle iff the three signs, taken in
// the triangle's winding direction, agree; the crossing coordinate is the
// barycentric combination of the vertices' coordinates along the ray (the
// centroid's for a triangle degenerate in projection), clamped to the
// triangle.  A node is inside iff an odd number of its x-line's crossings lie
// beyond it.  Crossing points are then moved onto the triangle's local
// surface w = h(s, t): the quadratic height over the triangle's plane (frame:
// centroid, unit face normal, tangents as for the density fit; coordinates
// scaled by the patch radius ell) through the triangle's fit points.  The
// surface is the zero set of phi = w - h, growing out of Omega, so normals and
// shape operators follow as for the level sets.
constexpr int MESH_NEWTON = 30;
constexpr int TRI_FIT = 19;          // o[3], t1[3], t2[3], nf[3], ell, c[6]
constexpr double MESH_NEAR = 1e-6;   // fallback window of a crossing, units of h

__host__ __device__ inline int canon_sign(double Pu, double Pv, double Qu, double Qv, double pu, double pv,
                                          double* E) {
  const double d1 = Qu - Pu, d2 = pv - Pv, d3 = Qv - Pv, d4 = pu - Pu;
  const double e = d1 * d2 - d3 * d4;
  *E = e;
  if (e > 0.0) return 1;
  if (e < 0.0) return -1;
  if (d3 != 0.0) return d3 < 0.0 ? 1 : -1;
  return d1 > 0.0 ? 1 : -1;
}

// does the line through (pu, pv) along axis a meet triangle t?  *xh: where
__host__ __device__ inline bool tri_hit(const double* X, const int32_t* T, int t, int a, double pu, double pv,
                                        double* xh) {
  const int u = (a + 1) % 3, v = (a + 2) % 3;
  const int id[3] = {T[3 * t], T[3 * t + 1], T[3 * t + 2]};
  double e[3];
  int sg[3];
  for (int k = 0; k < 3; ++k) {
    const int A = id[k], B = id[(k + 1) % 3];
    const double* PA = X + 3 * (size_t)A;
    const double* PB = X + 3 * (size_t)B;
    if (A < B) {
      sg[k] = canon_sign(PA[u], PA[v], PB[u], PB[v], pu, pv, &e[k]);
    } else {
      sg[k] = -canon_sign(PB[u], PB[v], PA[u], PA[v], pu, pv, &e[k]);
      e[k] = -e[k];
    }
  }
  if (sg[0] != sg[1] || sg[1] != sg[2]) return false;
  const double eAB = e[0], eBC = e[1], eCA = e[2];
  const double den = (eBC + eCA) + eAB;
  const double mag = (fabs(eBC) + fabs(eCA)) + fabs(eAB);
  const double Aa = X[3 * (size_t)id[0] + a], Ba = X[3 * (size_t)id[1] + a], Ca = X[3 * (size_t)id[2] + a];
  double x;
  if (fabs(den) <= 1e-12 * mag) x = ((Aa + Ba) + Ca) / 3.0;
  else x = ((eBC * Aa + eCA * Ba) + eAB * Ca) / den;
  x = fmin(fmax(x, fmin(fmin(Aa, Ba), Ca)), fmax(fmax(Aa, Ba), Ca));
  *xh = x;
  return true;
}

// grid-line candidates of triangle t along axis a (interior node indices)
__host__ __device__ inline void tri_lines(const double* X, const int32_t* T, int t, int a, const GridParams& gr,
                                          int* ju0, int* ju1, int* jv0, int* jv1) {
  const int u = (a + 1) % 3, v = (a + 2) % 3;
  double umin = 1e300, umax = -1e300, vmin = 1e300, vmax = -1e300;
  for (int k = 0; k < 3; ++k) {
    const double* P = X + 3 * (size_t)T[3 * t + k];
    umin = fmin(umin, P[u]);
    umax = fmax(umax, P[u]);
    vmin = fmin(vmin, P[v]);
    vmax = fmax(vmax, P[v]);
  }
  const int n1 = gr.N - 1;
  *ju0 = max(1, (int)floor((umin - gr.lo) / gr.h) - 1);
  *ju1 = min(n1, (int)ceil((umax - gr.lo) / gr.h) + 1);
  *jv0 = max(1, (int)floor((vmin - gr.lo) / gr.h) - 1);
  *jv1 = min(n1, (int)ceil((vmax - gr.lo) / gr.h) + 1);
}

// per triangle: count its crossings with the lines along a (offs == nullptr)
// or write them from offs[t] on: line (interior numbering k_v, k_u), x, t
__global__ void k_mesh_hits(const double* X, const int32_t* T, int n_tri, GridParams gr, int a, const int* offs,
                            int* counts, int32_t* line, double* xh, int32_t* tri) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tri) return;
  int ju0, ju1, jv0, jv1;
  tri_lines(X, T, t, a, gr, &ju0, &ju1, &jv0, &jv1);
  const int n1 = gr.N - 1;
  int c = 0;
  for (int ju = ju0; ju <= ju1; ++ju)
    for (int jv = jv0; jv <= jv1; ++jv) {
      double x;
      if (!tri_hit(X, T, t, a, node_coord(gr, ju), node_coord(gr, jv), &x)) continue;
      if (offs != nullptr) {
        const int o = offs[t] + c;
        line[o] = (jv - 1) * n1 + (ju - 1);
        xh[o] = x;
        tri[o] = t;
      }
      ++c;
    }
  if (offs == nullptr) counts[t] = c;
}

// inside flags of the interior nodes from the sorted crossings of their
// x-line: odd count beyond the node
__global__ void k_mesh_classify(GridParams gr, const int32_t* ptr, const double* hx, uint8_t* inside) {
  const int n1 = gr.N - 1;
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n1 * n1) return;
  const int j0 = ptr[l], j1 = ptr[l + 1];
  int j = j0;
  uint8_t* row = inside + (size_t)l * n1;
  for (int k = 1; k <= n1; ++k) {
    const double xk = node_coord(gr, k);
    while (j < j1 && hx[j] <= xk) ++j;
    row[k - 1] = (uint8_t)((j1 - j) & 1);
  }
}

__host__ __device__ inline void fit_height(const double* f, double s, double q, double* hs, double* hq,
                                           double* hh) {
  const double* c = f + 13;
  *hh = c[0] + c[1] * s + c[2] * q + c[3] * s * s + c[4] * s * q + c[5] * q * q;
  *hs = c[1] + 2.0 * c[3] * s + c[4] * q;
  *hq = c[2] + c[4] * s + 2.0 * c[5] * q;
}

__host__ __device__ inline void fit_local(const double* f, const double* P, double* s, double* q, double* w) {
  const double D0 = P[0] - f[0], D1 = P[1] - f[1], D2 = P[2] - f[2];
  const double ell = f[12];
  *s = (D0 * f[3] + D1 * f[4] + D2 * f[5]) / ell;
  *q = (D0 * f[6] + D1 * f[7] + D2 * f[8]) / ell;
  *w = (D0 * f[9] + D1 * f[10] + D2 * f[11]) / ell;
}

// outward normal and shape operator of triangle tri's local surface at P
__host__ __device__ void mesh_normal_shape(const double* tri_fit, int tri, const double* P, double* n,
                                           double S[3][3]) {
  const double* f = tri_fit + (size_t)tri * TRI_FIT;
  const double *t1 = f + 3, *t2 = f + 6, *nf = f + 9;
  const double ell = f[12];
  const double* c = f + 13;
  double s, q, w, hs, hq, hh;
  fit_local(f, P, &s, &q, &w);
  fit_height(f, s, q, &hs, &hq, &hh);
  double g[3];
  for (int i = 0; i < 3; ++i) g[i] = (nf[i] - hs * t1[i] - hq * t2[i]) / ell;
  const double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
  for (int i = 0; i < 3; ++i) n[i] = g[i] / gn;
  double H[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      H[i][j] = -(2.0 * c[3] * t1[i] * t1[j] + c[4] * (t1[i] * t2[j] + t2[i] * t1[j]) + 2.0 * c[5] * t2[i] * t2[j]) /
                (ell * ell);
  double Pm[3][3], Tm[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Pm[i][j] = (i == j ? 1.0 : 0.0) - n[i] * n[j];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0.0;
      for (int k = 0; k < 3; ++k) acc += Pm[i][k] * H[k][j];
      Tm[i][j] = acc;
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0.0;
      for (int k = 0; k < 3; ++k) acc += Tm[i][k] * Pm[k][j];
      S[i][j] = acc / gn;
    }
}

// per triangle: frame and height coefficients of its local surface
__global__ void k_tri_fit(const double* X, const int32_t* T, int n_tri, const int32_t* patch_ids,
                          const int32_t* patch_cnt, double* tri_fit, int* err) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tri) return;
  const double* A = X + 3 * (size_t)T[3 * t];
  const double* B = X + 3 * (size_t)T[3 * t + 1];
  const double* C = X + 3 * (size_t)T[3 * t + 2];
  double* f = tri_fit + (size_t)t * TRI_FIT;
  double o[3], nf[3], t1[3], t2[3];
  for (int i = 0; i < 3; ++i) o[i] = ((A[i] + B[i]) + C[i]) / 3.0;
  const double u[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
  const double v[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
  nf[0] = u[1] * v[2] - u[2] * v[1];
  nf[1] = u[2] * v[0] - u[0] * v[2];
  nf[2] = u[0] * v[1] - u[1] * v[0];
  const double ln = sqrt(nf[0] * nf[0] + nf[1] * nf[1] + nf[2] * nf[2]);
  for (int i = 0; i < 3; ++i) nf[i] /= ln;
  tangent_basis(nf, t1, t2);
  const int K = patch_cnt[t];
  double s[PATCH_MAX], q[PATCH_MAX], w[PATCH_MAX];
  double ell = 0.0;
  for (int k = 0; k < K; ++k) {
    const double* P = X + 3 * (size_t)patch_ids[(size_t)t * PATCH_MAX + k];
    const double D0 = P[0] - o[0], D1 = P[1] - o[1], D2 = P[2] - o[2];
    ell = fmax(ell, sqrt(D0 * D0 + D1 * D1 + D2 * D2));
    s[k] = D0 * t1[0] + D1 * t1[1] + D2 * t1[2];
    q[k] = D0 * t2[0] + D1 * t2[1] + D2 * t2[2];
    w[k] = D0 * nf[0] + D1 * nf[1] + D2 * nf[2];
  }
  double Gm[36], rhs[6];
  for (int i = 0; i < 36; ++i) Gm[i] = 0.0;
  for (int i = 0; i < 6; ++i) rhs[i] = 0.0;
  for (int k = 0; k < K; ++k) {
    const double sk = s[k] / ell, qk = q[k] / ell, wk = w[k] / ell;
    const double r[6] = {1.0, sk, qk, sk * sk, sk * qk, qk * qk};
    if (K == 6) {
      for (int j = 0; j < 6; ++j) Gm[k * 6 + j] = r[j];
      rhs[k] = wk;
    } else {
      for (int i = 0; i < 6; ++i) {
        for (int j = 0; j < 6; ++j) Gm[i * 6 + j] += r[i] * r[j];
        rhs[i] += r[i] * wk;
      }
    }
  }
  if (!gauss_solve(Gm, rhs, 6, 6)) atomicOr(err, DEVERR_SINGULAR);
  for (int i = 0; i < 3; ++i) {
    f[i] = o[i];
    f[3 + i] = t1[i];
    f[6 + i] = t2[i];
    f[9 + i] = nf[i];
  }
  f[12] = ell;
  for (int i = 0; i < 6; ++i) f[13 + i] = rhs[i];
}

// per crossing edge: its triangle (the line's single crossing in
// (x_lo, x_hi], or the nearest within MESH_NEAR h) and the point where the
// edge meets that triangle's local surface (Newton along the edge)
struct MeshHits {
  const int32_t* ptr[3];
  const double* x[3];
  const int32_t* tri[3];
};

__global__ void k_mesh_cross(GridParams gr, MeshHits mh, const double* tri_fit, const int32_t* c_lo,
                             const int32_t* c_axis, int n, double* c_z, int8_t* c_comp, int32_t* c_tri, int* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int n1 = gr.N - 1;
  const int64_t f = c_lo[i];
  const int a = c_axis[i];
  const int k[3] = {(int)(f % n1) + 1, (int)((f / n1) % n1) + 1, (int)(f / ((int64_t)n1 * n1)) + 1};
  const int u = (a + 1) % 3, v = (a + 2) % 3;
  const int line = (k[v] - 1) * n1 + (k[u] - 1);
  const double xl = node_coord(gr, k[a]), xhi = node_coord(gr, k[a] + 1);
  const int j0 = mh.ptr[a][line], j1 = mh.ptr[a][line + 1];
  int cnt = 0, pick = -1, near = -1;
  double best = 1e300;
  for (int j = j0; j < j1; ++j) {
    const double x = mh.x[a][j];
    if (x > xl && x <= xhi) {
      ++cnt;
      pick = j;
    }
    const double d = fmax(xl - x, x - xhi);
    if (d < best) {
      best = d;
      near = j;
    }
  }
  if (cnt == 0 && near >= 0 && best <= MESH_NEAR * gr.h) pick = near;
  c_comp[i] = 0;
  if (cnt > 1 || pick < 0) {
    atomicOr(err, DEVERR_GEOMETRY);
    c_z[i] = 0.5 * (xl + xhi);
    c_tri[i] = 0;
    return;
  }
  const int t = mh.tri[a][pick];
  c_tri[i] = t;
  const double* fr = tri_fit + (size_t)t * TRI_FIT;
  const double X0[3] = {node_coord(gr, k[0]), node_coord(gr, k[1]), node_coord(gr, k[2])};
  double s0, q0, w0;
  fit_local(fr, X0, &s0, &q0, &w0);
  const double ell = fr[12];
  const double ds = gr.h * fr[3 + a] / ell, dq = gr.h * fr[6 + a] / ell, dw = gr.h * fr[9 + a] / ell;
  double tau = (mh.x[a][pick] - xl) / gr.h;
  for (int it = 0; it < MESH_NEWTON; ++it) {
    double hs, hq, hh;
    const double s = s0 + tau * ds, q = q0 + tau * dq, w = w0 + tau * dw;
    fit_height(fr, s, q, &hs, &hq, &hh);
    const double fv = w - hh;
    const double fp = dw - (hs * ds + hq * dq);
    tau = tau - fv / fp;
  }
  c_z[i] = xl + tau * gr.h;
}

// Coefficients of the single layer's jump polynomial of one component with
// diagonal conductivity D at the displacement xi from a surface point with
// outward normal n and shape operator S (d n / d t = S t):
//   J(xi) = [grad v].xi + xi^T [D^2 v] xi / 2 = Apsi psi + Bg . grad_G psi,
// from [grad v] = alpha n, alpha = psi / q, q = n.D n,
//   grad_G alpha = grad_G psi / q - psi m,   m = 2 S D n / q^2,
//   [D^2 v] = alpha S + n grad_G alpha^T + grad_G alpha n^T + c n n^T,
//   c = -(alpha tr(D S) + 2 n.D grad_G alpha) / q
// ([v] = 0 differentiated twice along the surface, n.D[grad v] = psi, and
// the PDE jump tr(D [D^2 v]) = 0).  With D = I this is the isotropic
// J = psi (n.xi + xi^T (S - tr S n n^T) xi / 2) + (n.xi)(xi . grad_G psi).
__host__ __device__ void jump_poly(const double* n, const double (*S)[3], const double* D, int d, const double* xi,
                                   double* Apsi, double* Bg) {
  double Dn[3] = {0.0, 0.0, 0.0}, SDn[3] = {0.0, 0.0, 0.0};
  double q = 0.0, nx = 0.0, xSx = 0.0, trDS = 0.0;
  for (int a = 0; a < d; ++a) {
    Dn[a] = D[a] * n[a];
    q += n[a] * Dn[a];
    nx += n[a] * xi[a];
    trDS += D[a] * S[a][a];
  }
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) {
      SDn[a] += S[a][b] * Dn[b];
      xSx += xi[a] * S[a][b] * xi[b];
    }
  // u = xi - (n.xi) D n / q: J's grad_G alpha part is (n.xi) u . grad_G alpha
  double um = 0.0;
  for (int a = 0; a < 3; ++a) {
    const double u = a < d ? xi[a] - nx * Dn[a] / q : 0.0;
    Bg[a] = nx * u / q;
    um += u * (a < d ? 2.0 * SDn[a] / (q * q) : 0.0);
  }
  *Apsi = (nx + 0.5 * xSx - 0.5 * nx * nx * trDS / q) / q - nx * um;
}

// per crossing: density row (psi at z and its surface gradient) folded with
// the jump polynomial of the component (conductivity t.cond) into correction
// weights for both end nodes
__host__ __device__ int crossing_row(const GeomParams& gp, const GridParams& gr, const DensityInputs& di,
                                     const uint8_t* inside, const Tables& t, int i) {
  int errbits = 0;
  const int n1 = gr.N - 1, d = gr.dim;
  const int64_t f = t.c_lo[i];
  const int a = t.c_axis[i];
  const int comp = t.c_comp[i];
  int k[3] = {(int)(f % n1) + 1, (int)((f / n1) % n1) + 1, d == 3 ? (int)(f / ((int64_t)n1 * n1)) + 1 : 0};
  double P[3] = {node_coord(gr, k[0]), node_coord(gr, k[1]), d == 3 ? node_coord(gr, k[2]) : 0.0};
  const double xl = P[a], xh = node_coord(gr, k[a] + 1);
  const double z = t.c_z[i];
  P[a] = z;
  double n[3], S[3][3];
  if (gp.kind == KFBI_MESH3) mesh_normal_shape(di.tri_fit, t.c_tri[i], P, n, S);
  else normal_shape(gp, comp, P, n, S);
  // density row: psi(z) = sum w0 x[pid], grad_G psi(z) = sum wg[.] x[pid]
  int pid[PATCH_MAX];
  double w0[PATCH_MAX], wg[3][PATCH_MAX];
  int K = 0;
  if (d == 2) {
    const double* p = gp.p;
    const double xr = p[2] * P[0] + p[3] * P[1];
    const double yr = p[2] * P[1] - p[3] * P[0];
    const double twopi = 6.283185307179586476925286766559;
    double tt = atan2(yr / p[1], xr / p[0]);
    if (tt < 0.0) tt += twopi;
    if (tt >= twopi) tt -= twopi;
    const int M = di.M;
    const double D = twopi / M;
    int s = (int)floor(tt / D);
    if (s > M - 1) s = M - 1;
    if (s < 0) s = 0;
    const double u = (tt - s * D) / D, w = 1.0 - u;
    const int sp = (s + 1) % M;
    const double speed = sqrt((p[0] * yr / p[1]) * (p[0] * yr / p[1]) + (p[1] * xr / p[0]) * (p[1] * xr / p[0]));
    // grad_G psi = psi_s tau, tau = (-n_y, n_x), psi_s = psi_t / speed
    const double tau[2] = {-n[1], n[0]};
    const double dw[4] = {-1.0 / D, 1.0 / D, -(D / 6.0) * (3.0 * w * w - 1.0), (D / 6.0) * (3.0 * u * u - 1.0)};
    K = 4;
    pid[0] = s;
    pid[1] = sp;
    pid[2] = M + s;
    pid[3] = M + sp;
    w0[0] = w;
    w0[1] = u;
    w0[2] = (D * D / 6.0) * (w * w * w - w);
    w0[3] = (D * D / 6.0) * (u * u * u - u);
    for (int q = 0; q < 4; ++q) {
      wg[0][q] = tau[0] / speed * dw[q];
      wg[1][q] = tau[1] / speed * dw[q];
      wg[2][q] = 0.0;
    }
  } else {
    const int tri = gp.kind == KFBI_MESH3 ? t.c_tri[i] : locate_tri(gp, di.cube_t, comp, P);
    K = di.patch_cnt[tri];
    int ids[PATCH_MAX];
    for (int q = 0; q < K; ++q) ids[q] = di.patch_ids[(size_t)tri * PATCH_MAX + q];
    if (!fit_weights(di.nodes, ids, K, P, n, w0, wg)) errbits |= DEVERR_SINGULAR;
    for (int q = 0; q < K; ++q) pid[q] = ids[q];
  }
  // correction of end node e: -+ d_a J(x_other - z) / h^2 (- inside Omega)
  const double ih2 = 1.0 / (gr.h * gr.h);
  const int64_t fh = f + axis_stride(a, n1);
  const double sl = (inside[f] ? -ih2 : ih2) * t.cond[a];
  const double sh = (inside[fh] ? -ih2 : ih2) * t.cond[a];
  double xil[3] = {0.0, 0.0, 0.0}, xih[3] = {0.0, 0.0, 0.0};
  xil[a] = xh - z;
  xih[a] = xl - z;
  double Apl, Bgl[3], Aph, Bgh[3];
  jump_poly(n, S, t.cond, d, xil, &Apl, Bgl);
  jump_poly(n, S, t.cond, d, xih, &Aph, Bgh);
  t.c_cnt[i] = K;
  for (int q = 0; q < PATCH_MAX; ++q) {
    const bool on = q < K;
    double gl = 0.0, gh = 0.0;
    if (on)
      for (int b = 0; b < d; ++b) {
        gl += Bgl[b] * wg[b][q];
        gh += Bgh[b] * wg[b][q];
      }
    t.c_pid[(size_t)i * PATCH_MAX + q] = on ? pid[q] : 0;
    t.c_wlo[(size_t)i * PATCH_MAX + q] = on ? sl * (Apl * w0[q] + gl) : 0.0;
    t.c_whi[(size_t)i * PATCH_MAX + q] = on ? sh * (Aph * w0[q] + gh) : 0.0;
  }
  return errbits;
}

__global__ void k_crossing_rows(GeomParams gp, GridParams gr, DensityInputs di, const uint8_t* inside, Tables t,
                                int* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.n_int) return;
  const int e = crossing_row(gp, gr, di, inside, t, i);
  if (e) atomicOr(err, e);
}

// per interface node: stencil centre/signs, Taylor weights of dv/dn, and the
// coefficients A_i, B_i of the node's own jump terms (AB [M][4])
__host__ __device__ int node_stencil_row(const GeomParams& gp, const GridParams& gr, const DensityInputs& di,
                                         const uint8_t* inside, double* AB, const Tables& t, int i) {
  int errbits = 0;
  const int d = gr.dim, N = gr.N, n1 = N - 1;
  double q[3] = {di.nodes[(size_t)i * d], di.nodes[(size_t)i * d + 1], d == 3 ? di.nodes[(size_t)i * d + 2] : 0.0};
  int c[3] = {0, 0, 0}, sg[3] = {1, 1, 1};
  for (int ax = 0; ax < d; ++ax) {
    const double tt = (q[ax] - gr.lo) / gr.h;
    c[ax] = (int)floor(tt + 0.5);
    const double xc = gr.lo + (double)c[ax] * gr.h;
    sg[ax] = q[ax] >= xc ? 1 : -1;
    if (c[ax] < 2 || c[ax] > N - 2) errbits |= DEVERR_GEOMETRY;
    t.n_center[(size_t)i * d + ax] = c[ax];
    t.n_sign[(size_t)i * d + ax] = (int8_t)sg[ax];
  }
  if (errbits) return errbits;
  const int wn = work_n(gr);  // work-grid row length; node k sits at index k on both layouts
  t.n_base[i] = (int32_t)(((int64_t)(d == 3 ? c[2] : 0) * wn + c[1]) * wn + c[0]);
  int comp = 0;
  for (int cc = 1; cc < gp.n_comp; ++cc)
    if (i >= gp.comp_vert_offset[cc]) comp = cc;
  double n[3], S[3][3];
  if (gp.kind == KFBI_MESH3) mesh_normal_shape(di.tri_fit, di.vtri[i], q, n, S);
  else normal_shape(gp, comp, q, n, S);
  // stencil offsets in the oracle's order
  const int P = d == 2 ? 6 : 10;
  int off[10][3];
  int np = 0;
  off[np][0] = off[np][1] = off[np][2] = 0;
  ++np;
  for (int a = 0; a < d; ++a)
    for (int st = -1; st <= 1; st += 2) {
      off[np][0] = off[np][1] = off[np][2] = 0;
      off[np][a] = st;
      ++np;
    }
  for (int a = 0; a < d; ++a)
    for (int b = a + 1; b < d; ++b) {
      off[np][0] = off[np][1] = off[np][2] = 0;
      off[np][a] = sg[a];
      off[np][b] = sg[b];
      ++np;
    }
  double A[100], rhs[10];
  double xi[10][3];
  bool out[10];
  for (int j = 0; j < P; ++j) {
    double sx[3];
    for (int a = 0; a < 3; ++a) {
      xi[j][a] = a < d ? (gr.lo + (double)(c[a] + off[j][a]) * gr.h) - q[a] : 0.0;
      sx[a] = xi[j][a] / gr.h;
    }
    double* row = A + j * P;  // row j of the Taylor matrix (stored transposed below)
    int col = 0;
    row[col++] = 1.0;
    for (int a = 0; a < d; ++a) row[col++] = sx[a];
    for (int a = 0; a < d; ++a) row[col++] = 0.5 * sx[a] * sx[a];
    for (int a = 0; a < d; ++a)
      for (int b = a + 1; b < d; ++b) row[col++] = sx[a] * sx[b];
    int64_t f = (int64_t)(c[0] + off[j][0] - 1) + (int64_t)(c[1] + off[j][1] - 1) * n1;
    if (d == 3) f += (int64_t)(c[2] + off[j][2] - 1) * n1 * n1;
    out[j] = inside[f] == 0;
  }
  // wn solves A^T wn = c / h with c = (0, n_1 D_1 .. n_d D_d, 0...): the
  // conormal limit n.D grad v^+ of the component (D = t.cond)
  double At[100];
  for (int r = 0; r < P; ++r)
    for (int cc = 0; cc < P; ++cc) At[r * P + cc] = A[cc * P + r];
  for (int r = 0; r < P; ++r) rhs[r] = (r >= 1 && r <= d) ? n[r - 1] * t.cond[r - 1] / gr.h : 0.0;
  if (!gauss_solve(At, rhs, P, P)) errbits |= DEVERR_SINGULAR;
  double Ai = 0.0, Bi[3] = {0.0, 0.0, 0.0};
  for (int j = 0; j < P; ++j) {
    t.n_wn[(size_t)i * P + j] = rhs[j];
    if (!out[j]) continue;
    double Ap, Bg[3];
    jump_poly(n, S, t.cond, d, xi[j], &Ap, Bg);
    Ai += rhs[j] * Ap;
    for (int a = 0; a < d; ++a) Bi[a] += rhs[j] * Bg[a];
  }
  AB[(size_t)i * 4 + 0] = Ai;
  for (int a = 0; a < 3; ++a) AB[(size_t)i * 4 + 1 + a] = Bi[a];
  return errbits;
}

// the node's jump row on x = psi (3-D) or [psi; m] (2-D):
//   A_i psi_i + B_i . grad_Gamma psi(q_i)
__host__ __device__ int node_density_row(const GeomParams& gp, const GridParams& gr, const DensityInputs& di,
                                         const int32_t* vtri, const double* AB, const Tables& t, int i) {
  int errbits = 0;
  const int d = gr.dim;
  double q[3] = {di.nodes[(size_t)i * d], di.nodes[(size_t)i * d + 1], d == 3 ? di.nodes[(size_t)i * d + 2] : 0.0};
  int comp = 0;
  for (int cc = 1; cc < gp.n_comp; ++cc)
    if (i >= gp.comp_vert_offset[cc]) comp = cc;
  double n[3], S[3][3];
  if (gp.kind == KFBI_MESH3) mesh_normal_shape(di.tri_fit, di.vtri[i], q, n, S);
  else normal_shape(gp, comp, q, n, S);
  for (int k = 0; k < 3; ++k) t.n_normal[(size_t)i * 3 + k] = n[k];
  const double Ai = AB[(size_t)i * 4];
  const double Bi[3] = {AB[(size_t)i * 4 + 1], AB[(size_t)i * 4 + 2], AB[(size_t)i * 4 + 3]};
  const size_t o = (size_t)i * (PATCH_MAX + 1);
  if (d == 2) {
    const int M = di.M;
    const double twopi = 6.283185307179586476925286766559;
    const double D = twopi / M;
    const double* p = gp.p;
    const double xr = p[2] * q[0] + p[3] * q[1];
    const double yr = p[2] * q[1] - p[3] * q[0];
    const double speed = sqrt((p[0] * yr / p[1]) * (p[0] * yr / p[1]) + (p[1] * xr / p[0]) * (p[1] * xr / p[0]));
    const double tau0 = -n[1], tau1 = n[0];
    const double b = (Bi[0] * tau0 + Bi[1] * tau1) / speed;
    const int ip = (i + 1) % M;
    t.n_dcnt[i] = 4;
    t.n_dpid[o + 0] = i;
    t.n_dw[o + 0] = Ai - b / D;
    t.n_dpid[o + 1] = ip;
    t.n_dw[o + 1] = b / D;
    t.n_dpid[o + 2] = M + i;
    t.n_dw[o + 2] = -b * D / 3.0;
    t.n_dpid[o + 3] = M + ip;
    t.n_dw[o + 3] = -b * D / 6.0;
    for (int k = 4; k < PATCH_MAX + 1; ++k) {
      t.n_dpid[o + k] = 0;
      t.n_dw[o + k] = 0.0;
    }
  } else {
    const int tri = vtri[i];
    const int K = di.patch_cnt[tri];
    int ids[PATCH_MAX];
    for (int k = 0; k < K; ++k) ids[k] = di.patch_ids[(size_t)tri * PATCH_MAX + k];
    double w0[PATCH_MAX], wg[3][PATCH_MAX];
    if (!fit_weights(di.nodes, ids, K, q, n, w0, wg)) errbits |= DEVERR_SINGULAR;
    t.n_dcnt[i] = K + 1;
    t.n_dpid[o] = i;
    t.n_dw[o] = Ai;
    for (int k = 0; k < PATCH_MAX; ++k) {
      const bool on = k < K;
      t.n_dpid[o + 1 + k] = on ? ids[k] : 0;
      t.n_dw[o + 1 + k] = on ? Bi[0] * wg[0][k] + Bi[1] * wg[1][k] + Bi[2] * wg[2][k] : 0.0;
    }
  }
  return errbits;
}

__global__ void k_node_stencil(GeomParams gp, GridParams gr, DensityInputs di, const uint8_t* inside, double* AB,
                               Tables t, int* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.M) return;
  const int e = node_stencil_row(gp, gr, di, inside, AB, t, i);
  if (e) atomicOr(err, e);
}

__global__ void k_node_density(GeomParams gp, GridParams gr, DensityInputs di, const int32_t* vtri, const double* AB,
                               Tables t, int* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.M) return;
  const int e = node_density_row(gp, gr, di, vtri, AB, t, i);
  if (e) atomicOr(err, e);
}

// interior flat index -> field-layout flat index (Neumann box: all nodes)
__host__ __device__ inline int64_t interior_to_field(const GridParams& gr, int64_t f) {
  const int n1 = gr.N - 1, P = gr.N + 1;
  const int x = (int)(f % n1) + 1, y = (int)((f / n1) % n1) + 1;
  const int z = gr.dim == 3 ? (int)(f / ((int64_t)n1 * n1)) + 1 : 0;
  return ((int64_t)z * P + y) * P + x;
}

// the inside mask and the irregular nodes on the field layout of the Neumann
// box (box-boundary nodes are outside Omega)
__global__ void k_field_mask(GridParams gr, const uint8_t* inside, int64_t total, uint8_t* inside_user) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < total; f += (int64_t)gridDim.x * blockDim.x)
    inside_user[interior_to_field(gr, f)] = inside[f];
}
__global__ void k_field_irr(GridParams gr, const int32_t* irr, int n, int32_t* irr_user) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) irr_user[i] = (int32_t)interior_to_field(gr, irr[i]);
}

// per irregular node: its crossing arms (binary search in the per-axis lists)
__global__ void k_irr_arms(GridParams gr, const uint8_t* inside, Tables t, const int* axis_off, int* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.n_irr) return;
  const int n1 = gr.N - 1;
  const int64_t f = t.irr[i];
  const uint8_t me = inside[f];
  int na = 0;
  for (int a = 0; a < gr.dim; ++a) {
    const int k = axis_index(f, a, n1);
    const int64_t st = axis_stride(a, n1);
    for (int side = 0; side < 2; ++side) {
      int64_t lo;
      if (side == 0) {
        if (k == 0 || inside[f - st] == me) continue;
        lo = f - st;
      } else {
        if (k == n1 - 1 || inside[f + st] == me) continue;
        lo = f;
      }
      int b = axis_off[a], e = axis_off[a + 1];
      while (b < e) {
        const int m = (b + e) / 2;
        if (t.c_lo[m] < lo) b = m + 1;
        else e = m;
      }
      if (b >= axis_off[a + 1] || t.c_lo[b] != lo) {
        atomicOr(err, DEVERR_GEOMETRY);
        continue;
      }
      // end 0 = lower node of the crossing, end 1 = upper node
      t.irr_arm[(size_t)i * 6 + na] = b * 2 + (side == 0 ? 1 : 0);
      ++na;
    }
  }
  t.irr_narm[i] = (int8_t)na;
}

// CSR correction rows of the irregular nodes: the arms' crossing rows
// concatenated, entries with the same density index merged (in order of first
// appearance; neighbouring crossings share most of their surface-fit points).
// count: the merged length only (pointers are then scanned on the host).
__device__ int corr_row(const Tables& t, int i, int32_t* pid, double* w) {
  const int na = t.irr_narm[i];
  int n = 0;
  for (int a = 0; a < na; ++a) {
    const int code = t.irr_arm[(size_t)i * 6 + a];
    const int c = code >> 1;
    const double* wc = (code & 1) ? t.c_whi : t.c_wlo;
    const int K = t.c_cnt[c];
    for (int q = 0; q < K; ++q) {
      const int32_t p = t.c_pid[(size_t)c * PATCH_MAX + q];
      const double v = wc[(size_t)c * PATCH_MAX + q];
      int j = 0;
      while (j < n && pid[j] != p) ++j;
      if (j == n) {
        pid[n] = p;
        w[n] = v;
        ++n;
      } else {
        w[j] += v;
      }
    }
  }
  return n;
}

__global__ void k_corr_count(Tables t, int32_t* count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.n_irr) return;
  int32_t pid[6 * PATCH_MAX];
  double w[6 * PATCH_MAX];
  count[i] = corr_row(t, i, pid, w);
}

__global__ void k_corr_rows(Tables t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.n_irr) return;
  int32_t pid[6 * PATCH_MAX];
  double w[6 * PATCH_MAX];
  const int n = corr_row(t, i, pid, w);
  const int o = t.cr_ptr[i];
  for (int k = 0; k < n; ++k) {
    t.cr_pid[o + k] = pid[k];
    t.cr_w[o + k] = w[k];
  }
}

__global__ void k_line_start(const int32_t* irr, int n_irr, int n1, int n_lines, int32_t* line_start) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n_irr) return;
  const int li = i < n_irr ? irr[i] / n1 : n_lines;
  const int prev = i == 0 ? -1 : irr[i - 1] / n1;
  for (int l = prev + 1; l <= li; ++l) line_start[l] = i;
}

int blocks_for(int64_t n, int bs) { return (int)std::min<int64_t>((n + bs - 1) / bs, 1 << 20); }

// ordered compaction of flag[0..total) -> out (device), returns count
int compact(kfbi_handle* h, const uint8_t* flag, int64_t total, int32_t** out, int* count) {
  const int nb = (int)((total + CB - 1) / CB);
  int* counts = nullptr;
  KFBI_CUDA(cudaMalloc(&counts, sizeof(int) * (size_t)nb));
  k_count<<<nb, CB, 0, h->stream>>>(flag, total, counts);
  std::vector<int> hc(nb);
  KFBI_CUDA(cudaMemcpyAsync(hc.data(), counts, sizeof(int) * (size_t)nb, cudaMemcpyDeviceToHost, h->stream));
  KFBI_CUDA(cudaStreamSynchronize(h->stream));
  int acc = 0;
  for (int b = 0; b < nb; ++b) {
    const int c = hc[b];
    hc[b] = acc;
    acc += c;
  }
  *count = acc;
  int rc = dalloc(h, out, (size_t)acc);
  if (rc) {
    cudaFree(counts);
    return rc;
  }
  KFBI_CUDA(cudaMemcpyAsync(counts, hc.data(), sizeof(int) * (size_t)nb, cudaMemcpyHostToDevice, h->stream));
  k_write<<<nb, CB, 0, h->stream>>>(flag, total, counts, *out);
  KFBI_CUDA(cudaStreamSynchronize(h->stream));
  cudaFree(counts);
  KFBI_CHECK_LAUNCH();
  return KFBI_OK;
}

// surface-fit point lists of every triangle (six-point patch, or the vertex
// ring of the triangle when one of its points has valence other than 6)
int host_patches(const kfbi_geometry* g, std::vector<int32_t>& ids, std::vector<int32_t>& cnt,
                 std::vector<int32_t>& vtri) {
  const int nt = g->n_tri, nv = g->n_nodes;
  const int32_t* T = g->tri;
  std::unordered_map<int64_t, std::vector<std::pair<int, int>>> edges;
  edges.reserve((size_t)nt * 2);
  auto key = [](int u, int v) { return (int64_t)std::min(u, v) * (int64_t)(1 << 30) + std::max(u, v); };
  std::vector<int> val(nv, 0);
  std::vector<std::vector<int>> vt(nv);
  for (int t = 0; t < nt; ++t) {
    const int a = T[3 * t], b = T[3 * t + 1], c = T[3 * t + 2];
    edges[key(a, b)].push_back({t, c});
    edges[key(b, c)].push_back({t, a});
    edges[key(c, a)].push_back({t, b});
    for (int k = 0; k < 3; ++k) {
      val[T[3 * t + k]]++;
      vt[T[3 * t + k]].push_back(t);
    }
  }
  ids.assign((size_t)nt * PATCH_MAX, 0);
  cnt.assign(nt, 0);
  vtri.assign(nv, 0);
  for (int v = 0; v < nv; ++v) {
    if (vt[v].empty()) {
      set_error("interface node %d belongs to no triangle", v);
      return KFBI_ERR_ARG;
    }
    vtri[v] = *std::min_element(vt[v].begin(), vt[v].end());
  }
  for (int t = 0; t < nt; ++t) {
    const int a = T[3 * t], b = T[3 * t + 1], c = T[3 * t + 2];
    int six[6] = {a, b, c, -1, -1, -1};
    const int pairs[3][2] = {{a, b}, {b, c}, {c, a}};
    for (int s = 0; s < 3; ++s) {
      auto it = edges.find(key(pairs[s][0], pairs[s][1]));
      if (it == edges.end() || it->second.size() != 2) {
        set_error("surface mesh is not a closed manifold");
        return KFBI_ERR_ARG;
      }
      const auto& l = it->second;
      six[3 + s] = l[0].first != t ? l[0].second : l[1].second;
    }
    bool regular = true;
    for (int k = 0; k < 6; ++k)
      if (val[six[k]] != 6) regular = false;
    if (regular) {
      for (int k = 0; k < 6; ++k) ids[(size_t)t * PATCH_MAX + k] = six[k];
      cnt[t] = 6;
    } else {
      std::vector<int> ring;
      for (int k = 0; k < 3; ++k)
        for (int tt : vt[T[3 * t + k]])
          for (int m = 0; m < 3; ++m) ring.push_back(T[3 * tt + m]);
      std::sort(ring.begin(), ring.end());
      ring.erase(std::unique(ring.begin(), ring.end()), ring.end());
      if (ring.size() > (size_t)PATCH_MAX || ring.size() < 6) {
        set_error("unsupported vertex ring of %zu points", ring.size());
        return KFBI_ERR_ARG;
      }
      for (size_t k = 0; k < ring.size(); ++k) ids[(size_t)t * PATCH_MAX + k] = ring[k];
      cnt[t] = (int)ring.size();
    }
  }
  return KFBI_OK;
}

// first column of G = C^{-1} (6/D^2) second-difference, C = circulant(4, 1, 1)
void host_spline_column(int M, std::vector<double>& gcol) {
  const double D = 2.0 * M_PI / M;
  std::vector<double> rhs(M, 0.0);
  rhs[0] = -2.0 * 6.0 / (D * D);
  rhs[1 % M] += 6.0 / (D * D);
  rhs[(M - 1) % M] += 6.0 / (D * D);
  // cyclic tridiagonal solve (Sherman-Morrison) of  x_{i-1} + 4 x_i + x_{i+1} = rhs_i
  const double gam = -4.0;
  std::vector<double> bb(M, 4.0), u(M, 0.0), y(M), z(M), cp(M);
  bb[0] = 4.0 - gam;
  bb[M - 1] = 4.0 - 1.0 * 1.0 / gam;
  auto thomas = [&](const std::vector<double>& r, std::vector<double>& x) {
    cp[0] = 1.0 / bb[0];
    x[0] = r[0] / bb[0];
    for (int i = 1; i < M; ++i) {
      const double m = bb[i] - cp[i - 1];
      cp[i] = 1.0 / m;
      x[i] = (r[i] - x[i - 1]) / m;
    }
    for (int i = M - 2; i >= 0; --i) x[i] -= cp[i] * x[i + 1];
  };
  thomas(rhs, y);
  u[0] = gam;
  u[M - 1] = 1.0;
  thomas(u, z);
  const double fact = (y[0] + y[M - 1] / gam) / (1.0 + z[0] + z[M - 1] / gam);
  gcol.resize(M);
  for (int i = 0; i < M; ++i) gcol[i] = y[i] - fact * z[i];
}

template <typename T>
int upload(kfbi_handle* h, T** dst, const T* src, size_t n) {
  int rc = dalloc(h, dst, n);
  if (rc) return rc;
  KFBI_CUDA(cudaMemcpyAsync(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice, h->stream));
  return KFBI_OK;
}

// Mesh-only domain: every triangle's local surface, the ray crossings of
// the grid lines along each axis sorted by (line, coordinate, triangle) into
// per-line lists (the sort runs on the host), and the inside flags of the
// interior nodes from the x-lines.
int mesh_setup(kfbi_handle* h, const kfbi_geometry* geom, const double* X, const int32_t* T, const int32_t* ids,
               const int32_t* cnt, double** tri_fit, MeshHits* mh) {
  const GridParams gr = h->grid;
  cudaStream_t st = h->stream;
  const int nt = geom->n_tri, n1 = gr.N - 1, n_lines = n1 * n1;
  int rc;
  if ((rc = dalloc(h, tri_fit, (size_t)nt * TRI_FIT))) return rc;
  k_tri_fit<<<(nt + 127) / 128, 128, 0, st>>>(X, T, nt, ids, cnt, *tri_fit, h->w.err);
  KFBI_CHECK_LAUNCH();
  int* counts = nullptr;
  KFBI_CUDA(cudaMalloc((void**)&counts, sizeof(int) * 2 * (size_t)nt));
  int* offs = counts + nt;
  std::vector<int> hc(nt), ho(nt);
  for (int a = 0; a < 3; ++a) {
    k_mesh_hits<<<(nt + 127) / 128, 128, 0, st>>>(X, T, nt, gr, a, nullptr, counts, nullptr, nullptr, nullptr);
    KFBI_CHECK_LAUNCH();
    KFBI_CUDA(cudaMemcpyAsync(hc.data(), counts, sizeof(int) * (size_t)nt, cudaMemcpyDeviceToHost, st));
    KFBI_CUDA(cudaStreamSynchronize(st));
    int total = 0;
    for (int t = 0; t < nt; ++t) {
      ho[t] = total;
      total += hc[t];
    }
    const size_t nb = (size_t)std::max(total, 1);
    int32_t *line_d = nullptr, *tri_d = nullptr;
    double* x_d = nullptr;
    KFBI_CUDA(cudaMalloc((void**)&line_d, sizeof(int32_t) * nb));
    KFBI_CUDA(cudaMalloc((void**)&tri_d, sizeof(int32_t) * nb));
    KFBI_CUDA(cudaMalloc((void**)&x_d, sizeof(double) * nb));
    KFBI_CUDA(cudaMemcpyAsync(offs, ho.data(), sizeof(int) * (size_t)nt, cudaMemcpyHostToDevice, st));
    k_mesh_hits<<<(nt + 127) / 128, 128, 0, st>>>(X, T, nt, gr, a, offs, counts, line_d, x_d, tri_d);
    std::vector<int32_t> hl((size_t)total), ht((size_t)total);
    std::vector<double> hx((size_t)total);
    KFBI_CUDA(cudaMemcpyAsync(hl.data(), line_d, sizeof(int32_t) * (size_t)total, cudaMemcpyDeviceToHost, st));
    KFBI_CUDA(cudaMemcpyAsync(ht.data(), tri_d, sizeof(int32_t) * (size_t)total, cudaMemcpyDeviceToHost, st));
    KFBI_CUDA(cudaMemcpyAsync(hx.data(), x_d, sizeof(double) * (size_t)total, cudaMemcpyDeviceToHost, st));
    KFBI_CUDA(cudaStreamSynchronize(st));
    cudaFree(line_d);
    cudaFree(tri_d);
    cudaFree(x_d);
    KFBI_CHECK_LAUNCH();
    std::vector<int> order((size_t)total);
    for (int j = 0; j < total; ++j) order[j] = j;
    std::sort(order.begin(), order.end(), [&](int p, int q) {
      if (hl[p] != hl[q]) return hl[p] < hl[q];
      if (hx[p] != hx[q]) return hx[p] < hx[q];
      return ht[p] < ht[q];
    });
    std::vector<int32_t> ptr((size_t)n_lines + 1, 0), st_tri((size_t)nb, 0);
    std::vector<double> st_x((size_t)nb, 0.0);
    for (int j = 0; j < total; ++j) {
      st_x[j] = hx[order[j]];
      st_tri[j] = ht[order[j]];
      ptr[hl[order[j]] + 1]++;
    }
    for (int l = 0; l < n_lines; ++l) ptr[l + 1] += ptr[l];
    int32_t* ptr_d = nullptr;
    int32_t* stri_d = nullptr;
    double* sx_d = nullptr;
    if ((rc = upload(h, &ptr_d, ptr.data(), ptr.size()))) break;
    if ((rc = upload(h, &stri_d, st_tri.data(), st_tri.size()))) break;
    if ((rc = upload(h, &sx_d, st_x.data(), st_x.size()))) break;
    mh->ptr[a] = ptr_d;
    mh->tri[a] = stri_d;
    mh->x[a] = sx_d;
    KFBI_CUDA(cudaStreamSynchronize(st));
  }
  cudaFree(counts);
  if (rc) return rc;
  k_mesh_classify<<<(n_lines + 127) / 128, 128, 0, st>>>(gr, mh->ptr[0], mh->x[0], h->t.inside);
  KFBI_CHECK_LAUNCH();
  return KFBI_OK;
}

}  // namespace

// the CSR correction rows of t (new_pattern: also the pointers and indices;
// else they are shared with h->t and only the weights are built)
int build_corr_csr(kfbi_handle* h, Tables& t, bool new_pattern) {
  cudaStream_t st = h->stream;
  int rc;
  if (new_pattern) {
    std::vector<int32_t> cnt((size_t)t.n_irr), ptr((size_t)t.n_irr + 1, 0);
    if (t.n_irr > 0) {
      int32_t* cnt_d = nullptr;
      KFBI_CUDA(cudaMalloc((void**)&cnt_d, sizeof(int32_t) * (size_t)t.n_irr));
      k_corr_count<<<(t.n_irr + 127) / 128, 128, 0, st>>>(t, cnt_d);
      const cudaError_t e = cudaMemcpyAsync(cnt.data(), cnt_d, sizeof(int32_t) * cnt.size(), cudaMemcpyDeviceToHost, st);
      const cudaError_t e2 = cudaStreamSynchronize(st);
      cudaFree(cnt_d);
      KFBI_CUDA(e);
      KFBI_CUDA(e2);
      KFBI_COUNT(1);
    }
    for (int i = 0; i < t.n_irr; ++i) ptr[i + 1] = ptr[i] + cnt[i];
    if ((rc = upload(h, &t.cr_ptr, ptr.data(), ptr.size()))) return rc;
    if ((rc = dalloc(h, &t.cr_pid, (size_t)ptr[t.n_irr]))) return rc;
    h->cr_nnz = ptr[t.n_irr];
  }
  if ((rc = dalloc(h, &t.cr_w, (size_t)h->cr_nnz))) return rc;
  if (t.n_irr > 0) k_corr_rows<<<(t.n_irr + 127) / 128, 128, 0, st>>>(t);
  KFBI_CHECK_LAUNCH();
  return KFBI_OK;
}

int setup_build(kfbi_handle* h, const kfbi_geometry* geom) {
  const GridParams gr = h->grid;
  GeomParams& gp = h->gp;
  const int d = gr.dim, N = gr.N, n1 = N - 1;
  const int64_t total = d == 3 ? (int64_t)n1 * n1 * n1 : (int64_t)n1 * n1;
  Tables& t = h->t;
  cudaStream_t st = h->stream;
  int rc;

  int* err = h->w.err;
  KFBI_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  if ((rc = dalloc(h, &t.inside, (size_t)total))) return rc;
  // interface nodes and (3-D) the point lists of every triangle's surface
  // fit: the density fits, and the local surfaces of a mesh-only domain
  t.M = geom->n_nodes;
  double* nodes_d = nullptr;
  if ((rc = upload(h, &nodes_d, geom->nodes, (size_t)t.M * d))) return rc;
  int32_t *ids_d = nullptr, *cnt_d = nullptr, *vtri_d = nullptr, *tri_d = nullptr;
  if (d == 3) {
    std::vector<int32_t> ids, cnt, vtri;
    if ((rc = host_patches(geom, ids, cnt, vtri))) return rc;
    if ((rc = upload(h, &ids_d, ids.data(), ids.size()))) return rc;
    if ((rc = upload(h, &cnt_d, cnt.data(), cnt.size()))) return rc;
    if ((rc = upload(h, &vtri_d, vtri.data(), vtri.size()))) return rc;
    if ((rc = upload(h, &tri_d, geom->tri, (size_t)geom->n_tri * 3))) return rc;
  }
  const bool mesh = gp.kind == KFBI_MESH3;
  double* tri_fit = nullptr;
  MeshHits mh{};
  if (mesh) {
    if ((rc = mesh_setup(h, geom, nodes_d, tri_d, ids_d, cnt_d, &tri_fit, &mh))) return rc;
  } else {
    k_classify<<<blocks_for(total, 256), 256, 0, st>>>(gp, gr, t.inside, total);
  }
  uint8_t* flag = nullptr;
  KFBI_CUDA(cudaMalloc(&flag, (size_t)total));
  k_flags<<<blocks_for(total, 256), 256, 0, st>>>(gr, t.inside, total, 0, 0, flag, err);
  KFBI_CHECK_LAUNCH();
  if ((rc = compact(h, flag, total, &t.irr, &t.n_irr))) {
    cudaFree(flag);
    return rc;
  }
  // crossings along each axis, concatenated in axis order
  std::vector<int32_t*> parts(d, nullptr);
  std::vector<int> pc(d, 0);
  int axis_off_h[4] = {0, 0, 0, 0};
  for (int a = 0; a < d; ++a) {
    k_flags<<<blocks_for(total, 256), 256, 0, st>>>(gr, t.inside, total, 1, a, flag, err);
    if ((rc = compact(h, flag, total, &parts[a], &pc[a]))) {
      cudaFree(flag);
      return rc;
    }
    axis_off_h[a + 1] = axis_off_h[a] + pc[a];
  }
  cudaFree(flag);
  t.n_int = axis_off_h[d];
  if ((rc = dalloc(h, &t.c_lo, (size_t)t.n_int))) return rc;
  if ((rc = dalloc(h, &t.c_axis, (size_t)t.n_int))) return rc;
  {
    std::vector<int32_t> ax(t.n_int);
    for (int a = 0; a < d; ++a) {
      KFBI_CUDA(cudaMemcpyAsync(t.c_lo + axis_off_h[a], parts[a], sizeof(int32_t) * pc[a], cudaMemcpyDeviceToDevice, st));
      for (int i = axis_off_h[a]; i < axis_off_h[a + 1]; ++i) ax[i] = a;
    }
    KFBI_CUDA(cudaMemcpyAsync(t.c_axis, ax.data(), sizeof(int32_t) * t.n_int, cudaMemcpyHostToDevice, st));
    KFBI_CUDA(cudaStreamSynchronize(st));
  }
  int* axis_off = nullptr;
  if ((rc = upload(h, &axis_off, axis_off_h, 4))) return rc;
  if ((rc = dalloc(h, &t.c_z, (size_t)t.n_int))) return rc;
  if ((rc = dalloc(h, &t.c_comp, (size_t)t.n_int))) return rc;
  if (mesh) {
    if ((rc = dalloc(h, &t.c_tri, (size_t)std::max(t.n_int, 1)))) return rc;
    if (t.n_int > 0)
      k_mesh_cross<<<(t.n_int + 127) / 128, 128, 0, st>>>(gr, mh, tri_fit, t.c_lo, t.c_axis, t.n_int, t.c_z,
                                                          t.c_comp, t.c_tri, err);
  } else if (t.n_int > 0) {
    k_bisect<<<(t.n_int + 127) / 128, 128, 0, st>>>(gp, gr, t.c_lo, t.c_axis, t.n_int, t.c_z, t.c_comp, err);
  }
  KFBI_CHECK_LAUNCH();

  // the mask and the irregular list on the field layout
  if (gr.bc == KFBI_BOX_NEUMANN) {
    const int64_t nf = field_count(gr);
    if ((rc = dalloc(h, &t.inside_user, (size_t)nf))) return rc;
    if ((rc = dalloc(h, &t.irr_user, (size_t)t.n_irr))) return rc;
    KFBI_CUDA(cudaMemsetAsync(t.inside_user, 0, (size_t)nf, st));
    k_field_mask<<<blocks_for(total, 256), 256, 0, st>>>(gr, t.inside, total, t.inside_user);
    if (t.n_irr > 0) k_field_irr<<<(t.n_irr + 127) / 128, 128, 0, st>>>(gr, t.irr, t.n_irr, t.irr_user);
    KFBI_CHECK_LAUNCH_N(2);
  } else {
    t.inside_user = t.inside;
    t.irr_user = t.irr;
  }

  // irregular arms and x-line offsets
  if ((rc = dalloc(h, &t.irr_arm, (size_t)t.n_irr * 6))) return rc;
  if ((rc = dalloc(h, &t.irr_narm, (size_t)t.n_irr))) return rc;
  if (t.n_irr > 0) k_irr_arms<<<(t.n_irr + 127) / 128, 128, 0, st>>>(gr, t.inside, t, axis_off, err);
  const int n_lines = d == 3 ? n1 * n1 : n1;
  if ((rc = dalloc(h, &t.line_start, (size_t)n_lines + 1))) return rc;
  k_line_start<<<(t.n_irr + 1 + 127) / 128, 128, 0, st>>>(t.irr, t.n_irr, n1, n_lines, t.line_start);
  KFBI_CHECK_LAUNCH();

  // density inputs
  t.P = d == 2 ? 6 : 10;
  DensityInputs di{};
  di.M = t.M;
  di.nodes = nodes_d;
  t.nodes = nodes_d;
  if (d == 3) {
    double* ct_d = nullptr;
    if (!mesh && (rc = upload(h, &ct_d, geom->cube_t, (size_t)geom->cube_n + 1))) return rc;
    di.patch_ids = ids_d;
    di.patch_cnt = cnt_d;
    di.cube_t = ct_d;
    di.vtri = vtri_d;
    di.tri_fit = tri_fit;
  } else {
    std::vector<double> gcol;
    host_spline_column(t.M, gcol);
    if ((rc = upload(h, &t.spline_G, gcol.data(), gcol.size()))) return rc;
  }
  if (h->coupled)
    for (int a = 0; a < 3; ++a) t.cond[a] = a < d ? h->cpl.di[a] : 1.0;
  if ((rc = dalloc(h, &t.c_cnt, (size_t)t.n_int))) return rc;
  if ((rc = dalloc(h, &t.c_pid, (size_t)t.n_int * PATCH_MAX))) return rc;
  if ((rc = dalloc(h, &t.c_wlo, (size_t)t.n_int * PATCH_MAX))) return rc;
  if ((rc = dalloc(h, &t.c_whi, (size_t)t.n_int * PATCH_MAX))) return rc;
  if (t.n_int > 0) k_crossing_rows<<<(t.n_int + 63) / 64, 64, 0, st>>>(gp, gr, di, t.inside, t, err);
  KFBI_CHECK_LAUNCH();
  if ((rc = dalloc(h, &t.n_base, (size_t)t.M))) return rc;
  if ((rc = dalloc(h, &t.n_sign, (size_t)t.M * d))) return rc;
  if ((rc = dalloc(h, &t.n_center, (size_t)t.M * d))) return rc;
  if ((rc = dalloc(h, &t.n_wn, (size_t)t.M * t.P))) return rc;
  if ((rc = dalloc(h, &t.n_dcnt, (size_t)t.M))) return rc;
  if ((rc = dalloc(h, &t.n_dpid, (size_t)t.M * (PATCH_MAX + 1)))) return rc;
  if ((rc = dalloc(h, &t.n_dw, (size_t)t.M * (PATCH_MAX + 1)))) return rc;
  if ((rc = dalloc(h, &t.n_normal, (size_t)t.M * 3))) return rc;
  {
    double* AB = nullptr;
    KFBI_CUDA(cudaMalloc(&AB, sizeof(double) * 4 * (size_t)t.M));
    k_node_stencil<<<(t.M + 63) / 64, 64, 0, st>>>(gp, gr, di, t.inside, AB, t, err);
    int herr = 0;
    KFBI_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    KFBI_CUDA(cudaStreamSynchronize(st));
    if (!(herr & DEVERR_GEOMETRY))
      k_node_density<<<(t.M + 63) / 64, 64, 0, st>>>(gp, gr, di, vtri_d, AB, t, err);
    KFBI_CUDA(cudaStreamSynchronize(st));
    cudaFree(AB);
    KFBI_CHECK_LAUNCH();
  }

  // CSR correction rows of the irregular nodes
  if ((rc = build_corr_csr(h, t, true))) return rc;
  // coupled system: the extracellular component's correction and limit rows
  // (conductivity D_e) in t2; everything else is shared with t
  if (h->coupled) {
    Tables& t2 = h->t2;
    t2 = t;
    for (int a = 0; a < 3; ++a) t2.cond[a] = a < d ? h->cpl.de[a] : 1.0;
    if ((rc = dalloc(h, &t2.c_wlo, (size_t)t.n_int * PATCH_MAX))) return rc;
    if ((rc = dalloc(h, &t2.c_whi, (size_t)t.n_int * PATCH_MAX))) return rc;
    if ((rc = dalloc(h, &t2.n_wn, (size_t)t.M * t.P))) return rc;
    if ((rc = dalloc(h, &t2.n_dw, (size_t)t.M * (PATCH_MAX + 1)))) return rc;
    if (t.n_int > 0) k_crossing_rows<<<(t.n_int + 63) / 64, 64, 0, st>>>(gp, gr, di, t.inside, t2, err);
    double* AB = nullptr;
    KFBI_CUDA(cudaMalloc(&AB, sizeof(double) * 4 * (size_t)t.M));
    k_node_stencil<<<(t.M + 63) / 64, 64, 0, st>>>(gp, gr, di, t.inside, AB, t2, err);
    int herr = 0;
    KFBI_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    KFBI_CUDA(cudaStreamSynchronize(st));
    if (!(herr & DEVERR_GEOMETRY))
      k_node_density<<<(t.M + 63) / 64, 64, 0, st>>>(gp, gr, di, vtri_d, AB, t2, err);
    KFBI_CUDA(cudaStreamSynchronize(st));
    cudaFree(AB);
    KFBI_CHECK_LAUNCH_N(3);
    if ((rc = build_corr_csr(h, t2, false))) return rc;
  }

  // boundary quadrature weights (the rank-one term of the Poisson operator):
  // 2-D half the lengths of the two chords at a node, 3-D a third of the
  // areas of the incident triangles
  {
    const int M = t.M;
    const double* X = geom->nodes;
    std::vector<double> ds((size_t)M, 0.0);
    if (d == 2) {
      std::vector<double> seg((size_t)M);
      for (int i = 0; i < M; ++i) {
        const int j = (i + 1) % M;
        const double dx = X[2 * j] - X[2 * i], dy = X[2 * j + 1] - X[2 * i + 1];
        seg[i] = std::sqrt(dx * dx + dy * dy);
      }
      for (int i = 0; i < M; ++i) ds[i] = 0.5 * (seg[i] + seg[(i + M - 1) % M]);
    } else {
      for (int k = 0; k < geom->n_tri; ++k) {
        const int32_t* v = geom->tri + 3 * (size_t)k;
        const double* a = X + 3 * (size_t)v[0];
        const double* b = X + 3 * (size_t)v[1];
        const double* c = X + 3 * (size_t)v[2];
        const double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        const double w[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        const double cr[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
        const double area = 0.5 * std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
        for (int q = 0; q < 3; ++q) ds[v[q]] += area / 3.0;
      }
    }
    t.area = 0.0;
    for (int i = 0; i < M; ++i) t.area += ds[i];
    if ((rc = upload(h, &t.ds, ds.data(), ds.size()))) return rc;
    h->t2.ds = t.ds;
    h->t2.area = t.area;
    if (h->coupled) {
      std::vector<double> ds2(2 * (size_t)M);
      for (int i = 0; i < M; ++i) ds2[i] = ds2[M + i] = 0.5 * ds[i];
      if ((rc = upload(h, &h->w.ds2, ds2.data(), ds2.size()))) return rc;
    }
  }

  // transform tables
  {
    // mu1[p], p = 0..N (the cosine modes of the Neumann box use all of
    // them, the sine modes p = 1..N-1)
    std::vector<double> mu(N + 1), tw(4 * (size_t)N);
    for (int k = 0; k <= N; ++k) {
      const double s = std::sin(M_PI * k / (2.0 * N));
      mu[k] = -(4.0 / (gr.h * gr.h)) * s * s;
    }
    for (int j = 0; j < 2 * N; ++j) {
      tw[2 * j] = std::cos(M_PI * j / N);
      tw[2 * j + 1] = std::sin(M_PI * j / N);
    }
    std::vector<float> mu32(mu.begin(), mu.end()), tw32(tw.begin(), tw.end());
    if ((rc = upload(h, &t.mu, mu.data(), mu.size()))) return rc;
    if ((rc = upload(h, &t.tw64, tw.data(), tw.size()))) return rc;
    if ((rc = upload(h, &t.mu32, mu32.data(), mu32.size()))) return rc;
    if ((rc = upload(h, &t.tw32, tw32.data(), tw32.size()))) return rc;
    h->t2.mu = t.mu;
    h->t2.tw64 = t.tw64;
    h->t2.mu32 = t.mu32;
    h->t2.tw32 = t.tw32;
  }
  // inside count
  {
    std::vector<uint8_t> ins((size_t)total);
    KFBI_CUDA(cudaMemcpyAsync(ins.data(), t.inside, (size_t)total, cudaMemcpyDeviceToHost, st));
    int herr = 0;
    KFBI_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    KFBI_CUDA(cudaStreamSynchronize(st));
    int64_t cnt = 0;
    for (auto v : ins) cnt += v;
    t.n_inside = (int)cnt;
    if (herr & DEVERR_GEOMETRY) {
      set_error("geometry: the domain touches the box boundary, a grid edge crosses two surfaces, or an "
                "interpolation stencil leaves the interior grid");
      return KFBI_ERR_GEOMETRY;
    }
    if (herr & DEVERR_SINGULAR) {
      set_error("singular local system in the surface fit or the Taylor stencil");
      return KFBI_ERR_GEOMETRY;
    }
  }
  return KFBI_OK;
}

}  // namespace kfbi
